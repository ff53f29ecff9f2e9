"""Train the learned lane-position proposal on the GPU and measure what it gains.

    python -m paper_1807_02752_gb300.train_proposal --train 20000 --test 2000 --epochs 12 \
        --out paper_1807_02752_gb300/proposal_weights.npy

Frames are seeded synthetic 1242x375 scenes (the 64-frame workload's recipe: 10 % outlier and 10 % invalid
disparities), rendered by a process pool while the GPU consumes them.  The plain method labels every
training frame on the GPU (ld_make_training_pairs: its lanes' Eq. 25 tracks give the lane cells), the
network is trained with the library's own forward and backward kernels and Adam (ld_net_train_step), and
the held-out frames compare three rankings of the starts at the same top-k against the exhaustive search:
the trained network, the untrained one (its initial weights), and the raw input map without a network.
Agreement is 2 |P & L| / (|P| + |L|) over exact start positions, averaged over frames; a frame where the
proposal found no lane ran the exhaustive search (fallback) and agrees by construction.  Throughput of the
plain and learned forms on 64-frame batches is timed with CUDA events on one stream.  One JSON line.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

TRAIN_BASE, TEST_BASE = 1_000_000, 2_000_000    # frame-index ranges of the two sets (seeded, disjoint)


def _render(k):
    from . import scenes

    cfg, _ = scenes.WORKLOADS["batch64_1242x375"]
    d, i, _ = scenes.make_frame(cfg, k)
    return d, i


def init_params(seed: int) -> np.ndarray:
    """He-normal convolution weights, biases 0.01, head bias -2 (a lane cell is rare)."""
    rng = np.random.default_rng(seed)
    chans = (1, 16, 32, 32, 16)
    parts = []
    for l in range(4):
        ci, co = chans[l], chans[l + 1]
        parts.append(rng.standard_normal(co * ci * 9) * np.sqrt(2.0 / (ci * 9)))
        parts.append(np.full(co, 0.01))
    parts.append(rng.standard_normal(16) * 0.25)
    parts.append(np.array([-2.0]))
    return np.concatenate(parts).astype(np.float32)


def batches(pool, first: int, count: int, bs: int):
    """Yield (disp [b,H,W], img [b,H,W]) numpy batches of consecutive frame indices, rendered in the pool."""
    buf = []
    for d, i in pool.imap(_render, range(first, first + count), chunksize=4):
        buf.append((d, i))
        if len(buf) == bs:
            yield np.stack([x[0] for x in buf]), np.stack([x[1] for x in buf])
            buf = []
    if buf:
        yield np.stack([x[0] for x in buf]), np.stack([x[1] for x in buf])


def agreement(a, b) -> float:
    a, b = set(a), set(b)
    if not a and not b:
        return 1.0
    return 2.0 * len(a & b) / (len(a) + len(b))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--top-k", type=int, default=32)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--seed", type=int, default=20180706)
    ap.add_argument("--out", default=None, help="where to save the trained weights (.npy)")
    ap.add_argument("--weights", default=None, help="start from these weights (.npy); with --train 0, evaluate only")
    ap.add_argument("--sweep", type=int, nargs="*", default=[16, 48, 64, 96], help="further top-k values to evaluate")
    args = ap.parse_args(argv)

    pool = mp.get_context("spawn").Pool(args.workers)   # before the first CUDA call
    import torch

    from . import ld, scenes

    cfg, _ = scenes.WORKLOADS["batch64_1242x375"]
    W, H, B = cfg.width, cfg.height, args.batch
    mh, mw = (H + 3) // 4, (W + 3) // 4
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(W, H, B, p)
    net = ld.Net(det, training=True)
    theta0 = init_params(args.seed)
    start = np.load(args.weights).astype(np.float32) if args.weights else theta0
    net.set_params(torch.from_numpy(start).cuda())

    # training set: block sums and labels of every frame, kept on the device
    t0 = time.perf_counter()
    xs_all = torch.empty((max(args.train, 1), mh, mw), dtype=torch.int32, device="cuda")
    lb_all = torch.empty((max(args.train, 1), mh, mw), dtype=torch.uint8, device="cuda")
    k = 0
    for d, i in batches(pool, TRAIN_BASE, args.train, B):
        n = len(d)
        net.training_pairs(torch.from_numpy(d).cuda(), torch.from_numpy(i).cuda(), xs_all[k:k + n], lb_all[k:k + n])
        k += n
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    lane_cells = float(lb_all[:args.train].float().mean()) if args.train else None

    # training
    gen = torch.Generator().manual_seed(args.seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    steps = 0
    for ep in range(args.epochs if args.train else 0):
        perm = torch.randperm(args.train // B, generator=gen).tolist()
        lr = args.lr * (0.5 * (1.0 + np.cos(np.pi * ep / args.epochs)))      # cosine decay per epoch
        acc = torch.zeros(1, dtype=torch.float32, device="cuda")
        for b in perm:
            sl = slice(b * B, (b + 1) * B)
            net.train_step(xs_all[sl], lb_all[sl], W, H, float(lr), loss)
            acc += loss
            steps += 1
        losses.append(float(acc.item()) / max(1, len(perm)))
    ev1.record()
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    theta = net.get_params()
    if args.out:
        np.save(args.out, theta.cpu().numpy())
    del xs_all, lb_all

    # evaluation on held-out frames
    inf = ld.Net(det)
    results, fallbacks = {}, {}
    theta0_d = torch.from_numpy(theta0).cuda()

    def runs(theta, theta0, raw_map):
        """(name, weights or None, heatmap or None, top_k) of every ranking compared"""
        yield "trained", theta, None, args.top_k
        yield "untrained", theta0_d, None, args.top_k
        yield "raw_map", None, raw_map, args.top_k
        for k in args.sweep:
            yield f"trained_k{k}", theta, None, k
            yield f"raw_map_k{k}", None, raw_map, k
    frames = 0
    plain_out = det.alloc_lanes(B)
    learned_out = det.alloc_lanes(B)
    timing_batch = None
    for d, i in batches(pool, TEST_BASE, args.test, B):
        n = len(d)
        dd, ii = torch.from_numpy(d).cuda(), torch.from_numpy(i).cuda()
        if n == B and timing_batch is None:
            timing_batch = (dd, ii)
        plain = ld.Detector.lanes(det.detect(dd, ii, plain_out[:n * ld.LANES_DTYPE.itemsize]))
        xs, _, _ = net.training_pairs(dd, ii)
        raw_map = xs.float() * (2.0 ** -22)
        for name, params, hm, k in runs(theta, theta0, raw_map):
            if params is not None:
                inf.set_params(params)
            got = ld.Detector.lanes(inf.detect(dd, ii, k, heatmap=hm, out=learned_out[:n * ld.LANES_DTYPE.itemsize]))
            for f in range(n):
                a = list(got[f]["start_u"][:got[f]["n_lanes"]])
                b_ = list(plain[f]["start_u"][:plain[f]["n_lanes"]])
                results.setdefault(name, []).append(agreement(a, b_))
                fallbacks[name] = fallbacks.get(name, 0) + bool(got[f]["flags"] & ld.F_FALLBACK)
        frames += n
    pool.close()

    # throughput of the two forms, 64-frame batches, one stream, inputs resident
    inf.set_params(theta)
    dd, ii = timing_batch
    raw_t = net.training_pairs(dd, ii)[0].float() * (2.0 ** -22)

    def timed(fn, reps=50):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_plain = timed(lambda: det.detect(dd, ii, plain_out))
    ms_learned = timed(lambda: inf.detect(dd, ii, args.top_k, out=learned_out))
    ms_raw = timed(lambda: inf.detect(dd, ii, args.top_k, heatmap=raw_t, out=learned_out))
    line = {
        "train_frames": args.train, "test_frames": frames, "epochs": args.epochs, "batch": B, "lr": args.lr,
        "top_k": args.top_k, "steps": steps, "data_s": round(t_data, 1), "train_s": round(train_ms / 1e3, 2),
        "ms_per_train_step": round(train_ms / max(1, steps), 3),
        "lane_cell_fraction": None if lane_cells is None else round(lane_cells, 5),
        "loss_per_epoch": [round(x, 5) for x in losses],
        "agreement": {k: round(float(np.mean(v)), 5) for k, v in results.items()},
        "frames_at_99pct": {k: round(float(np.mean(np.asarray(v) >= 0.99)), 5) for k, v in results.items()},
        "fallback_frames": fallbacks,
        "ms_per_batch64": {"plain": round(ms_plain, 4), "learned": round(ms_learned, 4), "raw_map": round(ms_raw, 4)},
        "fps": {"plain": round(B / ms_plain * 1e3, 1), "learned": round(B / ms_learned * 1e3, 1)},
        "weights": args.out,
    }
    print(json.dumps(line), flush=True)
    for x in (inf, net):
        x.close()
    det.close()


if __name__ == "__main__":
    main()
