"""Run the detector on one named synthetic workload a few times, with eager launches (no CUDA graph), so
that a profiler attached to the process sees every kernel of every call as a separate launch.

    python -m paper_1807_02752_gb300.run_workload batch64_1242x375 4
    python -m paper_1807_02752_gb300.run_workload batch64_1242x375 4 learned 64
    python -m paper_1807_02752_gb300.run_workload batch64_1242x375 3 learned 96 fused
    python -m paper_1807_02752_gb300.run_workload batch64_1242x375 3 stereo
    python -m paper_1807_02752_gb300.run_workload mixed 20

Each call launches the nine kernels of the path once, in order, on the handle's stream, and times each
with CUDA events; the per-kernel times of the last call are printed.  With `learned [top_k]` each call is
the learned form instead (the network with the package's trained weights ranks the starts; exact
energies for the top_k coarse starts), timed as a whole; `fused` after top_k runs the network as the one
fused kernel instead of one kernel per layer.  With `stereo` each call is the stereo stage on
the workload's stereo pairs (search range propagation for both maps, then the consistency check).
`mixed` times frames of three camera sizes (16 x 1242x375, 8 x 1280x720, 8 x 1920x1080, D = 256) as one
ld_detect_groups call, as one ld_detect_mixed call (one launch per stage) and as three ld_detect calls in
a row on the same stream (captured graphs, replayed; CUDA events; median of the calls).
"""
from __future__ import annotations

import os
import sys


def mixed(calls: int):
    import numpy as np
    import torch

    from . import ld, scenes

    hd = scenes.HD_1920x1080
    spec = ((scenes.with_size(scenes.BATCH64_1242x375, n_disp=256), 16),
            (scenes.with_size(hd, width=1280, height=720, n_disp=256), 8), (scenes.with_size(hd, n_disp=256), 8))
    groups = []
    for g, (cfg, n) in enumerate(spec):
        fr = [scenes.make_frame(cfg, 900 + 10 * g + k)[:2] for k in range(4)]   # four scenes, repeated
        groups.append((torch.from_numpy(np.stack([fr[k % 4][0] for k in range(n)])).cuda(),
                       torch.from_numpy(np.stack([fr[k % 4][1] for k in range(n)])).cuda()))
    s = torch.cuda.Stream()
    det = ld.Detector(1920, 1080, sum(n for _, n in spec), ld.default_params(n_disp=256), stream=s)
    outs = [det.alloc_lanes(d.shape[0]) for d, _ in groups]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
            ms = []
            for _ in range(calls):
                e0.record(s)
                fn()
                e1.record(s)
                s.synchronize()
                ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    one = timed(lambda: det.detect_groups(groups, outs))
    mixed_ms = timed(lambda: det.detect_groups(groups, outs, mixed=True))
    three = timed(lambda: [det.detect(d, i, o) for (d, i), o in zip(groups, outs)])
    n = sum(n for _, n in spec)
    print({"frames": n, "groups_ms": round(one, 4), "groups_fps": round(n / one * 1e3, 1),
           "mixed_ms": round(mixed_ms, 4), "mixed_fps": round(n / mixed_ms * 1e3, 1),
           "three_calls_ms": round(three, 4), "three_calls_fps": round(n / three * 1e3, 1)})
    det.close()


def main(argv=None):
    import numpy as np
    import torch

    from . import ld, scenes

    argv = sys.argv[1:] if argv is None else argv
    name = argv[0] if argv else "batch64_1242x375"
    calls = int(argv[1]) if len(argv) > 1 else 4
    if name == "mixed":
        return mixed(calls)
    learned = len(argv) > 2 and argv[2] == "learned"
    stereo = len(argv) > 2 and argv[2] == "stereo"
    top_k = int(argv[3]) if len(argv) > 3 else 64
    fused = len(argv) > 4 and argv[4] == "fused"
    if name not in scenes.WORKLOADS:
        raise SystemExit(f"unknown workload {name!r}; known: {', '.join(scenes.WORKLOADS)}")
    cfg, n = scenes.WORKLOADS[name]
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, n, p)
    if stereo:
        pairs = [scenes.make_stereo_frame(cfg, k) for k in range(n)]
        lt = torch.from_numpy(np.stack([x[0] for x in pairs])).cuda()
        rt = torch.from_numpy(np.stack([x[1] for x in pairs])).cuda()
        st = ld.Stereo(det)
        out = torch.empty((n, cfg.height, cfg.width), dtype=torch.float32, device="cuda")
        ms = [st.run_timed(lt, rt, out) for _ in range(calls)]
        print(name, n, "frames, stereo: ms per call (propagation, check):", [list(map(float, m)) for m in ms])
        st.close()
        det.close()
        return
    disp, img, _ = scenes.make_batch(cfg, n)
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    out = det.alloc_lanes(n)
    if learned:
        net = ld.Net(det)
        w = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_weights.npy"))
        net.set_params(torch.from_numpy(w.astype(np.float32)).cuda())
        net.set_fused(fused)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(calls):
            e0.record()
            net.detect(d, i, top_k, out=out)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        print(name, n, "frames, learned form, top_k", top_k, "fused network" if fused else "network per layer",
              "ms per call:", [round(x, 4) for x in ms])
        net.close()
    else:
        ms = None
        for _ in range(calls):
            ms = det.detect_timed(d, i, out)
        torch.cuda.synchronize()
        print(name, n, "frames:", {k: round(float(x), 4) for k, x in zip(ld.launch_names(), np.asarray(ms))})
    det.close()


if __name__ == "__main__":
    main()
