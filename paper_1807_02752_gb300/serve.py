"""Serving measurement: camera streams with Poisson frame arrivals at mixed sizes through one server.

    python -m paper_1807_02752_gb300.serve --streams 8 --fps 60 --seconds 10
    python -m paper_1807_02752_gb300.serve --streams 8 --saturate --seconds 5
    python -m paper_1807_02752_gb300.serve --streams 8 --fps 60 --seconds 10 --learned 96
    python -m paper_1807_02752_gb300.serve --streams 8 --saturate --pinned --batch-submit 8 --producers 3

Each camera stream has a fixed resolution (stream k takes size k mod the number of sizes) and submits
frames at exponential inter-arrival times of mean 1/fps (or back to back with --saturate, a closed loop
that resubmits as soon as the server admits a frame).  Frames are seeded synthetic scenes of the size's
workload, generated before the clock starts and reused round-robin.  One JSON line reports the frames/s
completed, p50/p99 latency from submit to result in host memory (overall and per size), the mean batch
size and the admissions refused (a refused frame is retried after the next poll).  --pinned keeps the
frames in page-locked memory that the device reads directly; --batch-submit K hands the closed loop's
frames over K at a time; --producers P splits the streams over P threads; --hbm-budget-mb lets the server
add slots while their device memory stays within the budget.  --learned K runs
every batch in the learned form with top_k = K and the package's trained network weights; the line then
also counts the frames that fell back to the exhaustive search.
"""
from __future__ import annotations

import argparse
import json
import time


def scene_config(w: int, h: int, n_disp: int):
    from . import scenes

    if (w, h) == (1920, 1080):
        return scenes.with_size(scenes.HD_1920x1080, n_disp=n_disp)
    if h >= 600:
        return scenes.with_size(scenes.HD_1920x1080, width=w, height=h, n_disp=n_disp)
    return scenes.with_size(scenes.BATCH64_1242x375, width=w, height=h, n_disp=n_disp)


def main(argv=None):
    import numpy as np

    from . import ld, scenes

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--fps", type=float, default=60.0, help="mean frames/s per stream (Poisson arrivals)")
    ap.add_argument("--saturate", action="store_true", help="closed loop: submit as fast as admission allows")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--sizes", default="1242x375,1280x720,1920x1080")
    ap.add_argument("--n-disp", type=int, default=256)
    ap.add_argument("--max-batch", type=int, default=8)
    ap.add_argument("--slots", type=int, default=2, help="slots per size class")
    ap.add_argument("--max-wait-us", type=int, default=2000)
    ap.add_argument("--frames-per-size", type=int, default=8)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--learned", type=int, default=0, metavar="TOP_K",
                    help="learned form with this top_k (0: plain form)")
    ap.add_argument("--pinned", action="store_true",
                    help="frames in page-locked memory, read by the device directly (no host copy)")
    ap.add_argument("--batch-submit", type=int, default=1, metavar="K",
                    help="closed loop: submit K frames of one size per call")
    ap.add_argument("--producers", type=int, default=1, help="producer threads (streams split among them)")
    ap.add_argument("--hbm-budget-mb", type=int, default=0,
                    help="add slots on demand while their device memory stays within this budget (0: fixed slots)")
    args = ap.parse_args(argv)

    sizes = [tuple(int(x) for x in s.split("x")) for s in args.sizes.split(",")]
    frames = {}
    for (w, h) in sizes:
        cfg = scene_config(w, h, args.n_disp)
        frames[(w, h)] = [scenes.make_frame(cfg, 1000 + k)[:2] for k in range(args.frames_per_size)]
    p = ld.default_params(n_disp=args.n_disp)
    srv = ld.Server(sizes, p, slots_per_size=args.slots, max_batch=args.max_batch, max_wait_us=args.max_wait_us,
                    n_streams=args.streams, hbm_budget_bytes=args.hbm_budget_mb << 20)
    if args.learned > 0:
        import os

        import torch

        theta = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_weights.npy"))
        srv.set_learned(torch.from_numpy(theta.astype(np.float32)).cuda(), args.learned)
    size_of = [sizes[k % len(sizes)] for k in range(args.streams)]
    if args.pinned:   # the frames in page-locked memory, one [frames_per_size][h][w] tensor pair per size
        import torch

        frames = {sz: (torch.from_numpy(np.stack([f[0] for f in fr])).pin_memory(),
                       torch.from_numpy(np.stack([f[1] for f in fr])).pin_memory()) for sz, fr in frames.items()}
    else:
        frames = {sz: (np.stack([f[0] for f in fr]), np.stack([f[1] for f in fr])) for sz, fr in frames.items()}
    nf = args.frames_per_size
    t0 = time.perf_counter()
    t_end = t0 + args.seconds

    def submit(sids, sz, j):
        """Frames j, j+1, ... of size sz for the streams sids (fewer when the run would wrap): the number
        the server accepted."""
        d, i = frames[sz]
        k = min(len(sids), nf - j)
        if k == 1 and args.batch_submit == 1:
            if args.pinned:
                return int(srv.submit_pinned(sids[0], d[j], i[j], sids[0]))
            return int(srv.submit(sids[0], d[j], i[j], sids[0]))
        return srv.submit_batch(sids[:k], d[j:j + k], i[j:j + k], sids[:k], pinned=args.pinned)

    def producer(t, out):
        """Producer thread t drives the streams sid = t mod producers (ctypes drops the GIL in the calls, so
        the threads' copies run in parallel)."""
        mine = [sid for sid in range(args.streams) if sid % args.producers == t]
        res, refused = [], 0
        if not mine:
            out[t] = (res, refused)
            return
        by_size = {}
        for sid in mine:
            by_size.setdefault(size_of[sid], []).append(sid)
        cursor = {sz: 0 for sz in by_size}
        if args.saturate:
            order = list(by_size)
            q = 0
            while time.perf_counter() < t_end:
                sz = order[q % len(order)]
                ids = by_size[sz]
                sids = [ids[(cursor[sz] + r) % len(ids)] for r in range(args.batch_submit)]
                acc = submit(sids, sz, cursor[sz] % nf)
                if acc:
                    cursor[sz] += acc
                    q += 1
                else:
                    refused += 1
                    res.extend(srv.poll(timeout_ms=1))
                res.extend(srv.poll())
        else:
            rng = np.random.default_rng(args.seed + t)
            due = {sid: t0 + rng.exponential(1.0 / args.fps) for sid in mine}
            sent = {sid: 0 for sid in mine}
            while True:
                now = time.perf_counter()
                sid = min(due, key=due.get)
                if due[sid] >= t_end:
                    break
                if due[sid] > now:
                    res.extend(srv.poll(timeout_ms=max(0, int((due[sid] - now) * 1e3) - 1)))
                    continue
                if submit([sid], size_of[sid], sent[sid] % nf):
                    sent[sid] += 1
                    due[sid] += rng.exponential(1.0 / args.fps)
                else:
                    refused += 1
                    res.extend(srv.poll(timeout_ms=1))
                res.extend(srv.poll())
        out[t] = (res, refused)

    import threading

    outs = [None] * args.producers
    threads = [threading.Thread(target=producer, args=(t, outs)) for t in range(args.producers)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    results = [r for res, _ in outs for r in res]
    refused = sum(rf for _, rf in outs)
    srv.drain()
    while True:
        r = srv.poll()
        if len(r) == 0:
            break
        results.extend(r)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array([float(r["latency_ms"]) for r in results])
    per_size = {}
    for (w, h) in sizes:
        m = np.array([int(r["w"]) == w and int(r["h"]) == h for r in results], bool)
        if m.any():
            per_size[f"{w}x{h}"] = {"frames": int(m.sum()), "p50_ms": round(float(np.percentile(lat[m], 50)), 3),
                                    "p99_ms": round(float(np.percentile(lat[m], 99)), 3)}
    line = {
        "mode": "saturate" if args.saturate else "poisson", "streams": args.streams,
        "offered_fps": None if args.saturate else args.fps * args.streams,
        "frames": len(results), "seconds": round(wall, 3), "fps": round(len(results) / wall, 1),
        "p50_ms": round(float(np.percentile(lat, 50)), 3) if len(lat) else None,
        "p99_ms": round(float(np.percentile(lat, 99)), 3) if len(lat) else None,
        "mean_batch": round(st["mean_batch"], 2), "batches": st["batches"], "refused_submits": refused,
        "sizes": per_size, "n_disp": args.n_disp, "max_batch": args.max_batch, "slots_per_size": args.slots,
        "max_wait_us": args.max_wait_us, "form": f"learned top_k={args.learned}" if args.learned > 0 else "plain",
        "submit": {"pinned": args.pinned, "batch": args.batch_submit, "producers": args.producers},
        "slots": st["slots"], "device_mb": round(st["device_bytes"] / 2**20, 1),
        "hbm_budget_mb": args.hbm_budget_mb,
    }
    if args.learned > 0:
        line["fallback_frames"] = int(sum((int(r["lanes"]["flags"]) & ld.F_FALLBACK) != 0 for r in results))
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
