"""A/B of the paper-literal variants on the synthetic suite (GPU library, planted ground truth).

    python -m paper_1807_02752_gb300.ab_variants --frames 256 --hd-frames 64

Each variant is a parameter switch of the same library; every variant runs on the same seeded frames of
two workloads (the 64-frame 1242x375 recipe: 10 % outlier and 10 % invalid disparities; the 1920x1080
stress recipe: dashed lanes, shadow bands, 30 % outliers).  A planted marking counts when at least 40 of
its rows are visible and its start lies in the searched range; it is found when an unused detected start
lies within half its width + 3 px of it (nearest first).  Reported per variant and workload: recall of
planted markings, detections matching no marking per frame, frames whose road or V_px fit failed, and
the batch time (eager launches, CUDA events).  One JSON line per workload and variant.

Variants: the default readings; Sobel on the raw image (no pre-filter); the 11x11 median pre-filter of
the authors' previous system (Sec. 2.3.1); w_g as the Gaussian the Sec. 2.4 text names instead of the
printed exponential; one RANSAC hypothesis per round (the literal loop of Alg. 4 / Alg. 6); an absolute
lane threshold instead of the relative one; Eq. 12 as printed (the road DP linked to the row above);
Alg. 5's listing for the bottom rows of the V_px accumulator.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os

import numpy as np

VARIANTS = {
    "default": {},
    "no_prefilter": {"bilateral": 0},
    "median": {"bilateral": 2},
    "wg_gaussian": {"wg_gaussian": 1},
    "ransac_one_hypothesis": {"ransac_hyps": 1},
    "threshold_absolute": {"thr_abs": -(1 << 26)},
    "dp_literal": {"dp_literal": 1},
    "band_literal_bottom": {"band_literal_bottom": 1},
}


def _render(args):
    from . import scenes

    name, k = args
    cfg, _ = scenes.WORKLOADS[name]
    d, i, t = scenes.make_frame(cfg, k)
    return d, i, (t.lane_starts, t.lane_widths, t.lane_visible_rows)


def score(lanes, truths, W, S0):
    tp = fn = fp = failed = 0
    for r, (starts, widths, vis) in zip(lanes, truths):
        if r["flags"] & (1 | 4 | 16):          # no road, degenerate road fit, degenerate V_px fit
            failed += 1
        det = np.asarray(r["start_u"][:r["n_lanes"]])
        used = np.zeros(len(det), bool)
        for s, w, v in sorted(zip(starts, widths, vis), key=lambda x: x[0]):
            if v < 40 or not -S0 <= s < W + S0:
                continue
            free = np.where(~used)[0]
            k = free[np.argmin(np.abs(det[free] - s))] if len(free) else -1
            if k >= 0 and abs(det[k] - s) <= w / 2 + 3:
                tp += 1
                used[k] = True
            else:
                fn += 1
        fp += int((~used).sum())
    return tp, fn, fp, failed


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--frames", type=int, default=256)
    ap.add_argument("--hd-frames", type=int, default=64)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    args = ap.parse_args(argv)
    pool = mp.get_context("spawn").Pool(args.workers)   # before the first CUDA call
    import torch

    from . import ld, scenes

    for name, count, batch in (("batch64_1242x375", args.frames, 64), ("batch16_1920x1080", args.hd_frames, 16)):
        if count <= 0:
            continue
        cfg, _ = scenes.WORKLOADS[name]
        frames = pool.map(_render, [(name, 3_000_000 + k) for k in range(count)], chunksize=2)
        W, H = cfg.width, cfg.height
        for vname, kw in VARIANTS.items():
            p = ld.default_params(n_disp=cfg.n_disp, **kw)
            det = ld.Detector(W, H, batch, p)
            S0 = (det.n_starts(W) - W) // 2
            tp = fn = fp = failed = 0
            ms = []
            for b0 in range(0, count, batch):
                chunk = frames[b0:b0 + batch]
                d = torch.from_numpy(np.stack([c[0] for c in chunk])).cuda()
                i = torch.from_numpy(np.stack([c[1] for c in chunk])).cuda()
                out = det.alloc_lanes(len(chunk))
                ms.append(float(np.sum(det.detect_timed(d, i, out))))
                lanes = ld.lanes_to_dicts(ld.Detector.lanes(out))
                a, b, c, e = score(lanes, [c[2] for c in chunk], W, S0)
                tp, fn, fp, failed = tp + a, fn + b, fp + c, failed + e
            det.close()
            print(json.dumps({"workload": name, "variant": vname, "params": kw, "frames": count,
                              "recall": round(tp / max(1, tp + fn), 4), "planted": tp + fn,
                              "unmatched_per_frame": round(fp / count, 3), "fit_failed_frames": failed,
                              "ms_per_batch": round(float(np.median(ms)), 3), "batch": batch}), flush=True)
    pool.close()


if __name__ == "__main__":
    main()
