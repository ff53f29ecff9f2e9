"""Throughput benchmark of the lane-detection path on GB300.

One step = one pass of the whole path (all stages) over one batch of 64 synthetic 1242x375 frames
(the KITTI-shaped throughput workload).  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the only other program of the method here) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "frames/s @1242x375 batch 64 (plain vs learned proposal @≥99% agree); p99 ms"
UNIT = "frames/s"
WORKLOAD = "batch64_1242x375"
STEREO_BASE = 5_000_000   # frame indices of the stereo pairs
DTYPE = "u8/i32 (f32 decisions, f64 solves)"
# Integer operations of one bilateral tap as the method defines it (Eq. 15-16 in Q15 integers): the weight
# product ws * wr, its rounding add and shift, the accumulation of w * I (one multiply-add) and of w.  The
# kernel does the same work in fewer instructions (one table load replaces the weight's three operations).
INT_OPS_PER_TAP = 5


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------------------------------
# oracle arm (host cores)
# ----------------------------------------------------------------------------------------------------
_BARRIER = None


def _init_worker(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_chunk(args):
    """Render a chunk of frames, wait until every process of the pool has rendered its own chunk, then run
    the oracle on each frame.  Returns the process id, the start and the end of the oracle section
    (time.perf_counter: the system-wide monotonic clock, comparable across processes) and the summed
    per-frame oracle time; rendering stays outside all of them.  The barrier holds each process on its one
    chunk, so no process renders a second chunk while others are timed."""
    cfg_name, frames, pdict = args
    import oracle
    from paper_1807_02752_gb300 import scenes

    cfg, _ = scenes.WORKLOADS[cfg_name]
    inputs = [scenes.make_frame(cfg, f)[:2] for f in frames]
    p = oracle.default_params(**pdict)
    if _BARRIER is not None:
        _BARRIER.wait(timeout=900)
    t_start = time.perf_counter()
    cpu = 0.0
    for d, im in inputs:
        t0 = time.perf_counter()
        oracle.detect(d, im, p, dumps=False)
        cpu += time.perf_counter() - t0
    return os.getpid(), t_start, time.perf_counter(), cpu


def _stereo_worker(k):
    """One stereo pair of the workload's recipe and what scoring it needs (no detector arithmetic)."""
    from paper_1807_02752_gb300 import scenes

    cfg, _ = scenes.WORKLOADS[WORKLOAD]
    left, right, clean, truth = scenes.make_stereo_frame(cfg, STEREO_BASE + k)
    disp, _, _ = scenes.make_frame(cfg, STEREO_BASE + k)
    return left, right, clean, disp, (truth.v_horizon, truth.lane_starts, truth.lane_widths, truth.lane_visible_rows)


def oracle_pool(n_workers):
    """A spawned pool of n_workers processes that share one barrier of n_workers parties."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    return ctx.Pool(n_workers, initializer=_init_worker, initargs=(ctx.Barrier(n_workers),))


def run_oracle_frames(pool, frames, pdict, n_chunks):
    """The oracle over `frames` split into n_chunks tasks, n_chunks being the size of an oracle_pool (at
    least one frame per task).  The pool's barrier puts every task on its own process.  Returns the wall
    time of the oracle sections (latest end - earliest start; each task renders its frames before its
    section) and the summed single-thread time per frame."""
    chunks = [frames[k::n_chunks] for k in range(n_chunks)]
    if any(not c for c in chunks):
        raise ValueError("fewer frames than processes")
    res = pool.map(_oracle_chunk, [(WORKLOAD, c, pdict) for c in chunks], chunksize=1)
    if len({r[0] for r in res}) != len(res):
        raise RuntimeError("two oracle chunks ran on one process")
    return max(r[2] for r in res) - min(r[1] for r in res), sum(r[3] for r in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        inside = [s for s in self.samples if t0 - 0.1 <= s[0] <= t1 + 0.1]
        used = inside or [min(self.samples, key=lambda s: min(abs(s[0] - t0), abs(s[0] - t1)))]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(s[1][0]) for s in used if num(s[1][0]) is not None]
        mx = [num(s[1][1]) for s in used if num(s[1][1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in used for i in range(4) if "Active" in s[1][3 + i] and "Not" not in s[1][3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


# ----------------------------------------------------------------------------------------------------
def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, or None when the
    summary is missing or was taken on another version of the kernel source (its sha256 is recorded)."""
    import hashlib
    import re

    md = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    src = os.path.join(ROOT, "paper_1807_02752_gb300", "csrc", f"{kernel}.cu")
    if not (os.path.exists(md) and os.path.exists(src)):
        return None
    text = open(md).read()
    sha = re.search(r"sha256 ([0-9a-f]{64})", text)
    val = re.search(r"dram_bytes_per_launch: (\d+)", text)
    if not sha or not val:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != sha.group(1):
        return None
    return int(val.group(1))


def bilateral_pixels(det, W, H, n):
    """Pixels whose bilateral output the gradient kernel computes on the last call's frames (each counted
    once): read from the stage capture (LD_STAGE_IBF >= 0), so the road pixels the kernel proves flat and
    leaves out are not counted as work."""
    from paper_1807_02752_gb300 import ld

    return int(sum(int((det.debug(f, ld.STAGE_IBF, W, H) >= 0).sum()) for f in range(n)))


WEIGHTS = os.path.join(ROOT, "paper_1807_02752_gb300", "proposal_weights.npy")


def _recall(lanes, truths, W, S0):
    tp = fn = 0
    for r, (_, starts, widths, vis) in zip(lanes, truths):
        det = np.asarray(r["start_u"])
        used = np.zeros(len(det), bool)
        for s_, w_, v_ in sorted(zip(starts, widths, vis), key=lambda x: x[0]):
            if v_ < 40 or not -S0 <= s_ < W + S0:
                continue
            free = np.where(~used)[0]
            k = free[np.argmin(np.abs(det[free] - s_))] if len(free) else -1
            if k >= 0 and abs(det[k] - s_) <= w_ / 2 + 3:
                tp += 1
                used[k] = True
            else:
                fn += 1
    return tp / max(1, tp + fn)


def measure_stereo(args, pairs_async, det, stream, n):
    """Stereo (Sec. 2.1) on n rendered pairs of the workload: the disparity alone and the whole path from
    the pairs, timed with CUDA events on the handle's stream; the disparity against the planted one and
    the lanes against the planted markings (beside the lanes from the generator's own disparity)."""
    import torch

    from paper_1807_02752_gb300 import ld

    if pairs_async is None:
        return None
    pairs = pairs_async.get()
    W, H = pairs[0][0].shape[1], pairs[0][0].shape[0]
    L = torch.from_numpy(np.stack([p_[0] for p_ in pairs])).cuda()
    R = torch.from_numpy(np.stack([p_[1] for p_ in pairs])).cuda()
    G = torch.from_numpy(np.stack([p_[3] for p_ in pairs])).cuda()
    clean = np.stack([p_[2] for p_ in pairs])
    truths = [p_[4] for p_ in pairs]
    reps = max(5, min(args.steps, 50))
    with torch.cuda.stream(stream):
        st = ld.Stereo(det)
        disp = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
        lanes = det.alloc_lanes(n)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        for _ in range(3):
            st.run(L, R, disp)
            st.detect(L, R, lanes)
        ev[0].record(stream)
        for _ in range(reps):
            st.run(L, R, disp)
        ev[1].record(stream)
        for _ in range(reps):
            st.detect(L, R, lanes)
        ev[2].record(stream)
        stream.synchronize()
        d = disp.cpu().numpy()
        from_pairs = ld.lanes_to_dicts(ld.Detector.lanes(lanes))
        given = ld.lanes_to_dicts(ld.Detector.lanes(det.detect(G, L)))
        stream.synchronize()
        st.close()
    ms_st, ms_all = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
    road = np.zeros(d.shape, bool)
    for f, t in enumerate(truths):
        road[f, int(t[0]) + 6:] = True
    ok = road & (d > 0)
    S0 = (det.n_starts(W) - W) // 2
    return {"value": round(n / ms_st * 1e3, 1), "unit": UNIT, "ms_per_batch": round(ms_st, 4), "frames": n,
            "from_pairs": {"value": round(n / ms_all * 1e3, 1), "ms_per_batch": round(ms_all, 4)},
            "road_valid_fraction": round(float(ok.sum() / max(1, road.sum())), 4),
            "road_within_1px": round(float(np.mean(np.abs(d[ok] - clean[ok]) <= 1.0)), 4),
            "lane_recall_from_pairs": round(_recall(from_pairs, truths, W, S0), 4),
            "lane_recall_given_disparity": round(_recall(given, truths, W, S0), 4),
            "rho": 3, "tau": 1, "tr_lrc": 3}


def measure_single(args, stream):
    """Latency of one frame of the single-frame 1242x375 workload (5 % outlier disparities) on a one-frame
    handle: the captured graph timed with CUDA events on the handle's stream, L2 flushed by a 160 MiB write
    before each call, and end to end through ld_detect_host from pinned host buffers (host clock: the
    copies, the kernels, the result copy and the wait)."""
    import torch

    from paper_1807_02752_gb300 import ld, scenes

    if args.no_single:
        return None
    cfg, _ = scenes.WORKLOADS["single_1242x375"]
    d, i, _ = scenes.make_frame(cfg, 0)
    W, H = cfg.width, cfg.height
    reps = max(20, min(args.steps, 200))
    with torch.cuda.stream(stream):
        det = ld.Detector(W, H, 1, ld.default_params(n_disp=cfg.n_disp), stream=stream)
        dd, ii = torch.from_numpy(d[None]).cuda(), torch.from_numpy(i[None]).cuda()
        out = det.alloc_lanes(1)
        flush = torch.empty(40 * 2 ** 20, dtype=torch.float32, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(5):
            det.detect(dd, ii, out)
        dev = []
        for _ in range(reps):
            flush.fill_(1.0)
            a.record(stream)
            det.detect(dd, ii, out)
            b.record(stream)
            stream.synchronize()
            dev.append(a.elapsed_time(b))
        hd, hi = torch.from_numpy(d[None]).pin_memory(), torch.from_numpy(i[None]).pin_memory()
        res = np.zeros(1, ld.LANES_DTYPE)
        for _ in range(5):
            det.detect_host_ptr(hd.data_ptr(), hi.data_ptr(), W, H, 1, res)
        host = []
        for _ in range(reps):
            flush.fill_(1.0)
            stream.synchronize()
            t = time.perf_counter()
            det.detect_host_ptr(hd.data_ptr(), hi.data_ptr(), W, H, 1, res)
            host.append((time.perf_counter() - t) * 1e3)
        det.close()
    pct = lambda x, q: round(float(np.percentile(x, q)), 4)
    return {"workload": "single_1242x375 (one frame, 5 % outlier disparities)", "calls": reps,
            "p50_ms": pct(dev, 50), "p99_ms": pct(dev, 99), "e2e_p50_ms": pct(host, 50), "e2e_p99_ms": pct(host, 99),
            "l2": "flushed before each call (160 MiB write)"}


def measure_learned(args, dets, streams, disp, img, n, world):
    """The learned form (network-ranked starts, exact energies of the top-k) on the same handles, streams,
    inputs and step count as the plain form; agreement of its lanes with the plain lanes on both input
    batches.  None when the trained weights are absent."""
    import torch

    from paper_1807_02752_gb300 import ld, replicas

    if args.no_learned or not os.path.exists(WEIGHTS):
        return None
    S, K = len(dets), args.top_k
    theta = torch.from_numpy(np.load(WEIGHTS).astype(np.float32)).cuda()
    nets = [ld.Net(d) for d in dets]
    louts = [[d.alloc_lanes(n), d.alloc_lanes(n)] for d in dets]
    for k in range(S):
        with torch.cuda.stream(streams[k]):
            nets[k].set_params(theta)
    torch.cuda.synchronize()
    for s in range(max(args.warmup, 3) * S):
        k = s % S
        with torch.cuda.stream(streams[k]):
            nets[k].detect(disp[s & 1], img[s & 1], K, out=louts[k][s & 1])
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(main)
    for st in streams:
        st.wait_event(ev0)
    for s in range(args.steps):
        k = s % S
        with torch.cuda.stream(streams[k]):
            nets[k].detect(disp[s & 1], img[s & 1], K, out=louts[k][s & 1])
    for st in streams:
        main.wait_stream(st)
    ev1.record(main)
    torch.cuda.synchronize()
    total_ms = replicas.max_over_ranks(ev0.elapsed_time(ev1))
    # agreement with the plain form on both batches (exact start positions), fallbacks, evaluated starts
    agree, fallback, evaluated = [], 0, 0
    ns = dets[0].n_starts(disp[0].shape[2])
    with torch.cuda.stream(streams[0]):
        for b in range(2):
            plain = ld.Detector.lanes(dets[0].detect(disp[b], img[b]))
            got = ld.Detector.lanes(nets[0].detect(disp[b], img[b], K))
            for f in range(n):
                a = set(got[f]["start_u"][:got[f]["n_lanes"]])
                c = set(plain[f]["start_u"][:plain[f]["n_lanes"]])
                agree.append(1.0 if not a and not c else 2.0 * len(a & c) / (len(a) + len(c)))
                fallback += bool(got[f]["flags"] & ld.F_FALLBACK)
                evaluated += int(np.count_nonzero(nets[0].debug(f, ld.NET_STAGE_CFLAG) & 2))
    for x in nets:
        x.close()
    value = world * n * args.steps / (total_ms * 1e-3)
    return {"value": round(value, 2), "unit": UNIT, "ms_per_step": round(total_ms / args.steps, 4), "top_k": K,
            "agreement": round(float(np.mean(agree)), 5),
            "frames_at_99pct_agreement": round(float(np.mean(np.asarray(agree) >= 0.99)), 5),
            "fallback_frames": fallback, "frames_compared": len(agree),
            "evaluated_start_fraction": round(evaluated / (len(agree) * ns), 5),
            "weights": os.path.relpath(WEIGHTS, ROOT)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1807_02752_gb300 import ld, replicas, scenes
    from paper_1807_02752_gb300 import build as ldbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0 or local == 0:
        ldbuild.build()
    if world > 1:
        dist.barrier()

    # the oracle pool starts before the first CUDA work so no process forks after it
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    pool = oracle_pool(host_cores()) if want_cpu else None
    # stereo pairs render on host cores while the GPU runs (a spawn pool, started before any CUDA work)
    spool = mp.get_context("spawn").Pool(host_cores()) if rank == 0 and not args.no_stereo else None
    pairs_async = spool.map_async(_stereo_worker, range(64), chunksize=2) if spool else None

    cfg, n = scenes.WORKLOADS[WORKLOAD]
    W, H = cfg.width, cfg.height
    # two input batches (frames of this rank), alternated so the inputs (2 x 149 MB) exceed the 129 MB L2
    # this rank's frames: its round-robin share of a sequence of world x 2 batches (replicas, no collective)
    mine = replicas.frames_of_rank(world * 2 * n, rank, world)

    def batch(frames):
        fr = [scenes.make_frame(cfg, k) for k in frames]
        return np.stack([x[0] for x in fr]), np.stack([x[1] for x in fr])

    d0, i0 = batch(mine[:n])
    d1, i1 = batch(mine[n:])
    base = mine[0]
    disp = [torch.from_numpy(d0).cuda(), torch.from_numpy(d1).cuda()]
    img = [torch.from_numpy(i0).cuda(), torch.from_numpy(i1).cuda()]
    p = ld.default_params(n_disp=cfg.n_disp)
    # S streams, one library handle each; consecutive batches alternate between them so one batch's
    # per-frame serial stages overlap the next batch's dense stages
    S = max(1, args.streams)
    streams = [torch.cuda.Stream() for _ in range(S)]
    dets = [ld.Detector(W, H, n, p, stream=st) for st in streams]
    det = dets[0]
    stream = streams[0]
    outs = [[d.alloc_lanes(n), d.alloc_lanes(n)] for d in dets]
    torch.cuda.synchronize()
    # autotuned tile shapes: each handle times its candidates on the first input batch (results unchanged)
    tiles = None
    if not args.no_tune:
        for k in range(S):
            with torch.cuda.stream(streams[k]):
                tiles = dets[k].tune(disp[0], img[0], outs[k][0])
        torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    for s in range(max(args.warmup, 3) * S):
        k = s % S
        with torch.cuda.stream(streams[k]):
            dets[k].detect(disp[s & 1], img[s & 1], outs[k][s & 1])
    torch.cuda.synchronize()
    ev_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_end = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    main = torch.cuda.current_stream()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0.record(main)
    for st in streams:
        st.wait_event(ev0)
    for s in range(args.steps):
        k = s % S
        with torch.cuda.stream(streams[k]):
            ev_start[s].record(streams[k])
            dets[k].detect(disp[s & 1], img[s & 1], outs[k][s & 1])
            ev_end[s].record(streams[k])
    for st in streams:
        main.wait_stream(st)
    ev1.record(main)
    torch.cuda.synchronize()
    t_wall1 = time.time()
    if world > 1:
        dist.barrier()
    total_ms = ev0.elapsed_time(ev1)
    step_ms = np.array([ev_start[s].elapsed_time(ev_end[s]) for s in range(args.steps)])
    total_ms = replicas.max_over_ranks(total_ms)
    clk = clocks.summary(t_wall0, t_wall1) if clocks else None

    # per-kernel durations: eager launches with an event around every kernel, same stream
    names = ld.launch_names()
    kp_steps = max(5, min(args.steps, 40))
    per = np.zeros(len(names))
    with torch.cuda.stream(stream):
        for s in range(kp_steps):
            per += det.detect_timed(disp[s & 1], img[s & 1], outs[0][s & 1])
    per /= kp_steps
    if clocks:
        clocks.stop()
    # bilateral pixels per launch of the gradient kernel, averaged over the two input batches the timed
    # launches alternate between, counted on a capture handle of its own (outside every timed region)
    npx_batches = []
    with torch.cuda.stream(stream):
        cdet = ld.Detector(W, H, n, p, stream=stream)
        cdet.capture(True)
        for b in (0, 1):
            cdet.detect(disp[b], img[b], outs[0][b])
            stream.synchronize()
            npx_batches.append(bilateral_pixels(cdet, W, H, n))
        cdet.close()

    # end to end through the C-ABI with host buffers (pinned), copies inside the timed region; one host
    # thread per handle, so one batch's copies overlap another batch's kernels
    hd = [torch.from_numpy(d0).pin_memory(), torch.from_numpy(d1).pin_memory()]
    hi = [torch.from_numpy(i0).pin_memory(), torch.from_numpy(i1).pin_memory()]
    e2e_steps = max(2 * S, min(args.steps, 40))
    res = [np.zeros(n, ld.LANES_DTYPE) for _ in range(S)]
    for k in range(S):
        dets[k].detect_host_ptr(hd[k & 1].data_ptr(), hi[k & 1].data_ptr(), W, H, n, res[k])

    def e2e_worker(k):
        for s in range(k, e2e_steps, S):
            dets[k].detect_host_ptr(hd[s & 1].data_ptr(), hi[s & 1].data_ptr(), W, H, n, res[k])

    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    ths = [threading.Thread(target=e2e_worker, args=(k,)) for k in range(S)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    e2e_s = time.perf_counter() - t0
    e2e_s = replicas.max_over_ranks(e2e_s)

    learned = measure_learned(args, dets, streams, disp, img, n, world)
    stereo = measure_stereo(args, pairs_async, dets[0], streams[0], n) if rank == 0 else None
    single = measure_single(args, streams[0]) if rank == 0 else None
    if spool:
        spool.close()

    # roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    dom = int(np.argmax(per))
    dom_name = names[dom]
    dom_ms = float(per[dom])
    roof = None
    if dom_name == "k_grad":
        npx = int(round(sum(npx_batches) / len(npx_batches)))
        taps = (2 * p.bf_rho + 1) ** 2
        ops = INT_OPS_PER_TAP * taps * npx
        achieved = ops / (dom_ms * 1e-3) / 1e12
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = sms * 128 * sm_mhz * 1e6 / 1e12  # INT32 lanes x SMs x clock
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
                "frac": round(achieved / peak, 4), "traffic": profiled_traffic(dom_name, WORKLOAD), "kernel": dom_name,
                "units_per_launch": {"bilateral_pixels": npx, "taps_per_pixel": taps, "int_ops_per_tap": INT_OPS_PER_TAP},
                "peak_source": f"{sms} SMs x 128 INT32 lanes x {sm_mhz:.0f} MHz ({peak_src} clock)"}
    else:
        in_bytes = n * H * W * 5
        achieved = in_bytes / (dom_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": dom_name, "peak_source": peak_src}

    cpu = None
    if pool is not None:
        # a bounded sample: 16 frames per process on every host core (about 1.3 s of work per process)
        workers = host_cores()
        frames = list(range(base, base + 16 * workers))
        run_oracle_frames(pool, frames[:workers], p.as_dict(), workers)  # warm the workers
        wall, cpu_s = run_oracle_frames(pool, frames, p.as_dict(), workers)
        pool.close()
        cpu = {"value": round(len(frames) / wall, 3), "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{len(frames)} frames of the {WORKLOAD} workload, {len(frames) // workers} per process, "
                         f"rendered before the timed section ({cpu_s:.1f} s of CPU work, {wall:.1f} s wall)",
               "single_thread_ms_per_frame": round(1e3 * cpu_s / len(frames), 2)}

    if rank == 0:
        frames_total = world * n * args.steps
        value = frames_total / (total_ms * 1e-3)
        # the whole path against HBM: algorithmic input bytes (float32 disparity + uint8 image per pixel)
        path_gbs = value * H * W * 5 / 1e9
        roof["path"] = {"bound": "hbm", "achieved": round(path_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": round(path_gbs / peaks["hbm_gbs"], 4), "bytes_per_frame": H * W * 5,
                        "peak_source": peak_src}
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "p50_ms": round(float(np.percentile(step_ms, 50)), 4), "p99_ms": round(float(np.percentile(step_ms, 99)), 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE,
            "data": "synthetic (seeded KITTI-shaped scenes; KITTI is not available)",
            "config": {"workload": f"{WORKLOAD} plain form", "frames_per_step": n, "width": W, "height": H,
                       "streams": S, "tile_rows": tiles if tiles is not None else "built-in",
                       "n_disp": cfg.n_disp, "outliers": cfg.outlier_frac, "invalid": cfg.invalid_frac,
                       "l2": "inputs larger than L2 (two alternating 149 MB input batches)",
                       "parallelism": f"replicas x{world}"},
            "per_kernel_ms": {nm: round(float(x), 4) for nm, x in zip(names, per)},
            "roofline": roof,
            "hbm_frac": roof["path"]["frac"],
            "cpu_baseline": cpu,
            "e2e": {"value": round(world * n * e2e_steps / e2e_s, 2), "unit": UNIT,
                    "h2d_bytes_per_step": int(n * H * W * 5), "d2h_bytes_per_step": int(n * ld.LANES_DTYPE.itemsize)},
            "gpu_launches": int(ld.load().ld_launches_per_detect() * args.steps),
            "learned": None if learned is None else dict(learned, vs_plain=round(learned["value"] / value, 4)),
            "stereo": stereo,
            "single_frame": single,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    for d in dets:
        d.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1807_02752_gb300 import scenes

    import oracle
    oracle.build()
    cores = host_cores()
    pool = oracle_pool(cores)
    cfg, n = scenes.WORKLOADS[WORKLOAD]
    pdict = oracle.default_params(n_disp=cfg.n_disp).as_dict()
    per_step = cores  # one frame per process per step
    for s in range(max(args.warmup, 1)):
        run_oracle_frames(pool, [(s * per_step + k) % n for k in range(per_step)], pdict, cores)
    wall = cpu_total = 0.0   # each step's oracle sections; every process renders its frame before its section
    for s in range(args.steps):
        w, cpu_s = run_oracle_frames(pool, [(s * per_step + k) % n for k in range(per_step)], pdict, cores)
        wall += w
        cpu_total += cpu_s
    pool.close()
    value = args.steps * per_step / wall
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64/i64 (CPU)",
        "data": "synthetic (seeded KITTI-shaped scenes; KITTI is not available)",
        "config": {"workload": f"{WORKLOAD} plain form", "frames_per_step": per_step, "width": cfg.width,
                   "height": cfg.height, "n_disp": cfg.n_disp, "parallelism": "host processes"},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} frames of the {WORKLOAD} workload per step, one frame per process, "
                                   f"rendered before the timed section ({cpu_total:.1f} s of CPU work)",
                         "single_thread_ms_per_frame": round(1e3 * cpu_total / (args.steps * per_step), 2)},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in tile shapes")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal form")
    ap.add_argument("--no-stereo", action="store_true", help="skip the stereo stage measurement")
    ap.add_argument("--no-single", action="store_true", help="skip the single-frame latency measurement")
    ap.add_argument("--top-k", type=int, default=96, help="coarse starts the learned form evaluates per frame")
    ap.add_argument("--streams", type=int, default=4, help="library handles on separate streams, batches rotate over them")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
