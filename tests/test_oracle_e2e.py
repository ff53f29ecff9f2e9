"""End-to-end pins of the oracle on scenes with closed-form ground truth.

The scene generator plants the road profile f(v), the vanishing point V_p(v) = (V_px, V_py) and the lane
markings u_i(v) in closed form (Eq. 14 and the field lines of Eq. 25); the oracle must recover them.
"""
import math

import numpy as np
import pytest

from paper_1807_02752_gb300 import scenes


def _flat_road_frame(W=320, H=120, vh=40.0, b=0.35, lines=(), vp_u=150.0, D=48):
    v = np.arange(H, dtype=np.float64)
    f = b * (v - vh)
    disp = np.where(f[:, None] > 0, f[:, None], 0.0) * np.ones((1, W))
    img = np.full((H, W), 100.0)
    uu = np.arange(W)[None, :] + 0.0
    for s in lines:  # straight bright lines from (s, H-1) to (vp_u, vh), anti-aliased by 4 sub-rows
        acc = np.zeros((H, W))
        for dy in (-0.375, -0.125, 0.125, 0.375):
            vv = v + dy
            uc = vp_u + (s - vp_u) * (vv - vh) / (H - 1 - vh)
            half = np.maximum(0.5, 2.5 * (vv - vh) / (H - 1 - vh))
            lo = np.maximum(uu - 0.5, (uc - half)[:, None])
            hi = np.minimum(uu + 0.5, (uc + half)[:, None])
            acc += np.clip(hi - lo, 0, 1) / 4
        acc[v <= vh + 1] = 0
        img += acc * (220 - img)
    return disp.astype(np.float32), np.clip(np.rint(img), 0, 255).astype(np.uint8)


def test_flat_road_gives_constant_vpy(oracle_mod):
    """Eq. 14 on a flat road (beta2 = 0): V_py(v) = -beta0/beta1 = v_h on every road row."""
    for vh, b in [(40.0, 0.35), (33.3, 0.3), (47.6, 0.4)]:
        disp, img = _flat_road_frame(vh=vh, b=b)
        p = oracle_mod.default_params(n_disp=48)
        r = oracle_mod.detect(disp, img, p)
        assert not r["flags"] & (oracle_mod.F_NO_ROAD | oracle_mod.F_DEGEN_Y)
        rows = np.arange(r["v_top"], 120)
        assert r["v_top"] == pytest.approx(vh, abs=2.0)
        # the DP path is quantised to one row per disparity bin, which leaves a slight curvature in the
        # fit; V_py = v - f/f' amplifies it, so the planted value is met to a few rows
        assert np.abs(r["Vpy"][rows] - vh).max() < 3.5
        # and the reported rows are Eq. 14 of the reported road profile
        tau = (rows - r["centre"]) / 2.0 ** r["scale_exp"]
        b0, b1, b2 = r["beta"]
        f = b0 + b1 * tau + b2 * tau * tau
        fp = (b1 + 2 * b2 * tau) / 2.0 ** r["scale_exp"]
        assert np.allclose(r["Vpy"][rows], rows - f / fp, rtol=1e-6, atol=1e-4)
        assert np.allclose(r["F"][rows], f, rtol=1e-6, atol=1e-5)


def test_votes_peak_at_vanishing_point(oracle_mod):
    """Straight lines through a known V_p on a flat road vote (Eq. 17) for V_px on every row."""
    vp_u = 150.0
    disp, img = _flat_road_frame(lines=(30.0, 150.0, 290.0), vp_u=vp_u)
    p = oracle_mod.default_params(n_disp=48)
    r = oracle_mod.detect(disp, img, p)
    votes = r["votes"]
    tot = votes.sum(axis=0)
    assert abs(int(np.argmax(tot)) - round(vp_u)) <= 1
    assert tot[round(vp_u) - 2:round(vp_u) + 3].sum() > 0.3 * tot.sum()
    assert abs(r["Vpx"][r["v_top"]:].mean() - vp_u) < 2.0


def test_wg_applied_to_road_edges(oracle_mod):
    """Eq. 23 on every road edge pixel: w_g from the angle between the edge and the ray to V_p."""
    cfg = scenes.SINGLE_1242x375
    disp, img, _ = scenes.make_frame(cfg, 3)
    p = oracle_mod.default_params(n_disp=cfg.n_disp)
    r = oracle_mod.detect(disp, img, p)
    edge = r["edge"].astype(bool)
    assert (r["Gw"][~edge] == 0).all()
    vv, uu = np.nonzero(edge)
    gx = r["Gx"][vv, uu].astype(np.float64)
    gy = r["Gy"][vv, uu].astype(np.float64)
    t = np.stack([-gy, gx], 1)
    ray = np.stack([r["Vpx"][vv] - uu, r["Vpy"][vv] - vv], 1).astype(np.float64)
    cosang = np.abs((t * ray).sum(1)) / (np.linalg.norm(t, axis=1) * np.linalg.norm(ray, axis=1))
    dth = np.arccos(np.clip(cosang, 0, 1))
    w = np.where(gx != 0, r["Gw"][vv, uu] / np.where(gx == 0, 1, gx), 0)
    inside = dth < math.pi / 6 - 1e-3
    outside = dth > math.pi / 6 + 1e-3
    ref = 4096 * np.exp(-dth * 36 / (math.pi * 3.5 ** 2))
    nz = inside & (gx != 0)
    assert nz.sum() > 500
    assert np.abs(w[nz] - ref[nz]).max() <= 1.0
    assert (w[outside] == 0).all()


def test_end_to_end_recovers_planted_scene(oracle_mod):
    """1242x375 frames: road profile, V_p and lane starts recovered from disparity + image alone."""
    cfg = scenes.SINGLE_1242x375
    p = oracle_mod.default_params(n_disp=cfg.n_disp)
    W, H = cfg.width, cfg.height
    S0 = (oracle_mod.n_starts(W, p) - W) // 2
    tp = fn = fp = 0
    vpx_med = []
    for fr in range(12):
        disp, img, truth = scenes.make_frame(cfg, fr)
        r = oracle_mod.detect(disp, img, p, dumps=True)
        assert r["flags"] & ~(oracle_mod.F_CAP_Y | oracle_mod.F_CAP_X) == 0
        v = np.arange(H)
        road = (v >= r["v_top"]) & (v > truth.v_horizon + 2)
        assert abs(r["v_top"] - truth.v_horizon) <= 2.0
        tau = (v - r["centre"]) / 2.0 ** r["scale_exp"]
        f = np.polyval(np.array(r["beta"])[::-1], tau)
        ft = np.polyval(truth.beta[::-1], v)
        err = np.abs(f - ft)[road]
        assert np.median(err) < 0.25 and err.max() < 1.0            # road profile, in disparity units
        assert np.median(np.abs(r["Vpy"] - truth.vpy)[road]) < 1.5  # Eq. 14 rows
        vpx_med.append(np.median(np.abs(r["Vpx"] - truth.vpx)[road]))
        det = np.array(r["start_u"])
        used = np.zeros(len(det), bool)
        for s, w, vis in zip(truth.lane_starts, truth.lane_widths, truth.lane_visible_rows):
            if vis < 40 or not -S0 <= s < W + S0:
                continue
            k = int(np.argmin(np.abs(det - s))) if len(det) else -1
            if k >= 0 and abs(det[k] - s) <= w / 2 + 3 and not used[k]:
                tp += 1
                used[k] = True
            else:
                fn += 1
        fp += int((~used).sum())
    assert max(vpx_med) < 25 and np.mean(vpx_med) < 10
    assert tp >= 0.75 * (tp + fn)
    assert fp <= 0.75 * 12


def test_stress_frames_recover_road_and_vanishing_point(oracle_mod):
    """1920x1080 stress frames (dashed lanes, shadow bands over 30 % of the road rows, 30 % outlier
    disparities, D = 256): the road profile f(v), v_top and the vanishing-point rows V_py, V_px are
    recovered from disparity + image alone.  Lane starts are pinned on the 1242x375 frames above: on this
    recipe the method finds fewer of the planted markings (about 0.43 recall over 64 frames), so the pin
    here is the road and vanishing-point chain."""
    cfg = scenes.HD_1920x1080
    p = oracle_mod.default_params(n_disp=cfg.n_disp)
    H = cfg.height
    vpx_med = []
    for fr in range(6):
        disp, img, truth = scenes.make_frame(cfg, fr)
        r = oracle_mod.detect(disp, img, p, dumps=True)
        assert r["flags"] & ~(oracle_mod.F_CAP_Y | oracle_mod.F_CAP_X) == 0
        assert abs(r["v_top"] - truth.v_horizon) <= 2.0
        v = np.arange(H)
        road = (v >= r["v_top"]) & (v > truth.v_horizon + 2)
        tau = (v - r["centre"]) / 2.0 ** r["scale_exp"]
        err = np.abs(np.polyval(np.array(r["beta"])[::-1], tau) - np.polyval(truth.beta[::-1], v))[road]
        assert np.median(err) < 0.25 and err.max() < 1.0
        assert np.median(np.abs(r["Vpy"] - truth.vpy)[road]) < 2.0
        vpx_med.append(np.median(np.abs(r["Vpx"] - truth.vpx)[road]))
    assert max(vpx_med) < 25 and np.mean(vpx_med) < 15
