"""Scoring of one oracle detection against the planted truth of its synthetic scene (test helper).

The scene generator plants the road profile f(v), the vanishing point rows V_p(v) = (V_px, V_py) and the
lane markings in closed form (Eq. 14 and the field lines of Eq. 25).  ``score_frame`` runs the oracle on
one frame and reduces the comparison to a few numbers, so that a process pool can score many seeds and
send back only the summaries.

Error measures:

* road profile: |f(v) - f_true(v)| in disparity units on the road rows;
* V_px: an error d at row v turns every Eq. 25 track through that row by the angle atan(d / (v - V_py)),
  because the track aims at (V_px, V_py); the vote that places V_px (Eq. 17) is made from the Sobel
  direction of an edge with the same lever arm v - V_py.  The error is therefore reported as that angle,
  which makes rows and frame sizes comparable, and the rows are split into those inside the span of the
  final RANSAC set of Alg. 6 (first to last inlier row) and those outside it, where the quartic of
  Eq. 19 extrapolates;
* lanes: a planted marking is matched by a detected start within half its width + 3 px at the bottom row;
* the energy stage alone: Eq. 24-25 evaluated on the frame's own M_1 with the planted V_p, so that the
  lane energies are scored without the error of the V_p estimate.
"""
from __future__ import annotations

import numpy as np

from paper_1807_02752_gb300 import scenes

CONFIGS = {"single_1242x375": scenes.SINGLE_1242x375, "batch16_1920x1080": scenes.HD_1920x1080}
MIN_VISIBLE_ROWS = 40


def _match(det, starts, widths, visible, S0, W, slack):
    """Greedy match of planted markings (visible on MIN_VISIBLE_ROWS rows or more, start inside the start
    range) to detected starts within width/2 + slack.  Returns (hits, misses, unmatched detections,
    errors of the hits relative to half the marking width)."""
    det = np.asarray(det, np.float64)
    used = np.zeros(len(det), bool)
    hits = misses = 0
    rel = []
    for s, w, vis in zip(starts, widths, visible):
        if vis < MIN_VISIBLE_ROWS or not -S0 <= s < W + S0:
            continue
        k = int(np.argmin(np.abs(det - s))) if len(det) else -1
        if k >= 0 and abs(det[k] - s) <= w / 2 + slack and not used[k]:
            hits += 1
            used[k] = True
            rel.append(abs(det[k] - s) / (w / 2))
        else:
            misses += 1
    return hits, misses, int((~used).sum()), rel


def score_frame(cfg_name: str, frame: int) -> dict:
    import oracle

    cfg = CONFIGS[cfg_name]
    W, H = cfg.width, cfg.height
    p = oracle.default_params(n_disp=cfg.n_disp)
    ns = oracle.n_starts(W, p)
    S0 = (ns - W) // 2
    disp, img, t = scenes.make_frame(cfg, frame)
    r = oracle.detect(disp, img, p, dumps=True)
    v = np.arange(H)
    road = (v >= r["v_top"]) & (v > t.v_horizon + 2)
    tau = (v - r["centre"]) / 2.0 ** r["scale_exp"]
    f_err = np.abs(np.polyval(np.array(r["beta"])[::-1], tau) - np.polyval(t.beta[::-1], v))[road]

    inl = np.nonzero(r["inl_x"])[0]
    support = road & (v >= inl.min()) & (v <= inl.max()) if inl.size else np.zeros(H, bool)
    with np.errstate(invalid="ignore", divide="ignore"):
        ang = np.degrees(np.arctan(np.abs(r["Vpx"] - t.vpx) / (v - t.vpy)))
    rows = np.nonzero(road)[0]
    thirds = np.array_split(rows, 3)

    hits, misses, extra, rel = _match(r["start_u"], t.lane_starts, t.lane_widths, t.lane_visible_rows, S0, W, 3.0)

    # the energy stage on the planted V_p
    vpx_t = np.where(road, t.vpx, 0.0).astype(np.float32)
    vpy_t = np.where(road, t.vpy, 0.0).astype(np.float32)
    he = oracle.energy(r["M1"], r["v_top"], vpx_t, vpy_t, S0, ns)
    sel = oracle.select(he, S0, p)
    minima_near = []
    for s, w, vis in zip(t.lane_starts, t.lane_widths, t.lane_visible_rows):
        if vis < MIN_VISIBLE_ROWS or not -S0 <= s < W + S0:
            continue
        i0 = max(1, int(np.floor(s - w / 2 - 2)) + S0)
        i1 = min(ns - 2, int(np.ceil(s + w / 2 + 2)) + S0)
        minima_near.append(any(he[i] < he[i - 1] and he[i] < he[i + 1] for i in range(i0, i1 + 1)))
    t_hits, t_misses, t_extra, t_rel = _match(sel["start_u"], t.lane_starts, t.lane_widths, t.lane_visible_rows,
                                              S0, W, 2.0)
    return {
        "frame": frame,
        "flags": int(r["flags"]),
        "v_top_err": float(abs(r["v_top"] - t.v_horizon)),
        "f_med": float(np.median(f_err)),
        "f_p95": float(np.percentile(f_err, 95)),
        "f_max": float(f_err.max()),
        "vpy_med": float(np.median(np.abs(r["Vpy"] - t.vpy)[road])),
        "ang_support_med": float(np.median(ang[support])) if support.any() else 90.0,
        "ang_thirds_med": [float(np.median(ang[x])) for x in thirds],
        "support_cover": float(support.sum() / road.sum()),
        "hits": hits, "misses": misses, "extra": extra, "rel": rel,
        "minima_near": minima_near,
        "t_hits": t_hits, "t_misses": t_misses, "t_extra": t_extra, "t_rel": t_rel,
    }


def score_many(cfg_name: str, frames, processes: int | None = None) -> list[dict]:
    """score_frame over many frames in a spawned process pool (the oracle is single-threaded)."""
    import multiprocessing as mp
    import os

    frames = list(frames)
    n = processes or max(1, min(8, os.cpu_count() or 1, len(frames)))
    if n == 1:
        return [score_frame(cfg_name, f) for f in frames]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.starmap(score_frame, [(cfg_name, f) for f in frames])
