"""Pins of the oracle's dense stages: v-disparity (Sec. 2.2), DPs (Eq. 12, Eq. 18), bilateral filter
(Eq. 15-16), Sobel, band accumulator (Alg. 5), w_g (Eq. 23), M_0/M_1 (Alg. 7), energies (Eq. 24-25)
and lane selection.

Each pin is independent of the oracle's own code: brute force on tiny inputs, scipy/numpy library
routines, closed forms and invariants.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import ndimage

from paper_1807_02752_gb300 import scenes


# ---------------------------------------------------------------------------------------------- a1
def test_vdisparity_counts_valid_pixels(oracle_mod):
    rng = np.random.default_rng(0)
    for D in (8, 32, 128):
        d = rng.uniform(-2, D + 2, size=(13, 29)).astype(np.float32)
        d[rng.random(d.shape) < 0.1] = 0.0
        d[0, 0], d[1, 1], d[2, 2], d[3, 3] = np.nan, np.inf, -np.inf, D - 0.5
        m = oracle_mod.vdisparity(d, D)
        with np.errstate(invalid="ignore"):
            valid = np.isfinite(d) & (d > 0) & (np.floor(d + np.float32(0.5)) < D)
        assert (m.sum(axis=1) == valid.sum(axis=1)).all()
        for v in range(d.shape[0]):
            bins = np.floor(d[v][valid[v]] + np.float32(0.5)).astype(int)
            assert (np.bincount(bins, minlength=D) == m[v]).all()


def test_vdisparity_constant_frame_is_one_spike(oracle_mod):
    d = np.full((20, 40), 17.3, np.float32)
    m = oracle_mod.vdisparity(d, 64)
    assert (m[:, 17] == 40).all() and m.sum() == 20 * 40


# ---------------------------------------------------------------------------------------------- a2
def _brute_dp_vdisp(my, tau, lam):
    H, D = my.shape
    best = None
    for v1 in range(H):
        for steps in itertools.product(range(tau + 1), repeat=D - 2):
            path = [v1]
            ok = True
            for s in steps:
                path.append(path[-1] + s)
                if path[-1] > H - 1:
                    ok = False
                    break
            if not ok:
                continue
            e = sum(-int(my[path[i], i + 1]) for i in range(D - 1)) + lam * sum(steps)
            key = (e, path)
            if best is None or key < best:
                best = key
    return best


def test_dp_vdisp_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(1)
    for trial in range(30):
        H, D, tau = 8, 5, int(rng.integers(1, 4))
        my = rng.integers(0, 4 if trial % 2 else 2, size=(H, D)).astype(np.int32)  # many ties
        e, path = oracle_mod.dp_vdisp(my, tau, 1)
        be, bpath = _brute_dp_vdisp(my, tau, 1)
        assert e == be
        assert path[1:].tolist() == bpath


def test_dp_vdisp_follows_noise_free_road(oracle_mod):
    H, W, D = 120, 64, 48
    v = np.arange(H)
    f = 0.0008 * (v - 30.0) ** 2 + 0.3 * (v - 30.0)
    disp = np.where(f[:, None] > 0, f[:, None], 0.0).astype(np.float32) * np.ones((1, W), np.float32)
    my = oracle_mod.vdisparity(disp, D)
    _, path = oracle_mod.dp_vdisp(my, 6, 1)
    dbin = np.floor(np.maximum(f, 0).astype(np.float32) + np.float32(0.5)).astype(int)
    for d in range(1, int(dbin.max()) + 1):
        rows = np.nonzero(dbin == d)[0]
        if rows.size:
            assert rows[0] <= path[d] <= rows[-1]


# ---------------------------------------------------------------------------------------------- b1
def _bilateral_f64(img, rho, ss, sr):
    """Eq. 15-16 evaluated directly in float64 (clipped window, intensities scaled to [0,1])."""
    H, W = img.shape
    I = img.astype(np.float64)
    num = np.zeros((H, W))
    den = np.zeros((H, W))
    pad = np.pad(I, rho, constant_values=np.nan)
    for dy in range(-rho, rho + 1):
        for dx in range(-rho, rho + 1):
            q = pad[rho + dy:rho + dy + H, rho + dx:rho + dx + W]
            ok = ~np.isnan(q)
            w = math.exp(-(dx * dx + dy * dy) / ss ** 2) * np.exp(-((np.nan_to_num(q) - I) / 255.0) ** 2 / sr ** 2)
            w = np.where(ok, w, 0.0)
            num += w * np.nan_to_num(q)
            den += w
    return num / den


def test_bilateral_within_one_lsb_of_direct_formula(oracle_mod):
    rng = np.random.default_rng(2)
    img = np.clip(rng.normal(110, 30, size=(40, 57)), 0, 255).astype(np.uint8)
    img[:, 30:] = np.clip(img[:, 30:].astype(int) + 90, 0, 255)
    out = oracle_mod.bilateral(img)
    ref = _bilateral_f64(img, 5, 300.0, 0.3)
    assert np.abs(out.astype(np.float64) - ref).max() <= 1.0


def test_bilateral_constant_image_unchanged(oracle_mod):
    for c in (0, 1, 100, 254, 255):
        img = np.full((23, 31), c, np.uint8)
        assert (oracle_mod.bilateral(img) == c).all()


def test_bilateral_large_sigma_r_is_gaussian_blur(oracle_mod):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(30, 44)).astype(np.uint8)
    p = oracle_mod.default_params(sigma_r=1e6, sigma_s=3.0)
    out = oracle_mod.bilateral(img, p)
    k = np.array([[math.exp(-(x * x + y * y) / 9.0) for x in range(-5, 6)] for y in range(-5, 6)])
    num = ndimage.correlate(img.astype(np.float64), k, mode="constant", cval=0.0)
    den = ndimage.correlate(np.ones_like(img, dtype=np.float64), k, mode="constant", cval=0.0)
    assert np.abs(out - num / den).max() <= 1.0


def test_bilateral_preserves_step_edge(oracle_mod):
    img = np.full((21, 40), 50, np.uint8)
    img[:, 20:] = 200
    out = oracle_mod.bilateral(img).astype(int)
    assert abs(out[10, 19] - 50) < 15 and abs(out[10, 20] - 200) < 15
    k = np.ones((11, 11))
    blur = ndimage.correlate(img.astype(float), k, mode="nearest") / k.sum()
    assert abs(blur[10, 19] - 50) > 40


# ---------------------------------------------------------------------------------------------- b2
def test_sobel_matches_scipy_correlate(oracle_mod):
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(17, 23)).astype(np.uint8)
    gx, gy = oracle_mod.sobel(img)
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    ky = kx.T
    rx = ndimage.correlate(img.astype(np.int64), kx, mode="constant")
    ry = ndimage.correlate(img.astype(np.int64), ky, mode="constant")
    assert (gx[1:-1, 1:-1] == rx[1:-1, 1:-1]).all() and (gy[1:-1, 1:-1] == ry[1:-1, 1:-1]).all()
    assert (gx[0] == 0).all() and (gx[:, -1] == 0).all() and (gy[-1] == 0).all() and (gy[:, 0] == 0).all()


def test_sobel_vertical_step(oracle_mod):
    img = np.full((9, 12), 40, np.uint8)
    img[:, 6:] = 40 + 77
    gx, gy = oracle_mod.sobel(img)
    assert (gx[1:-1, 5] == 4 * 77).all() and (gx[1:-1, 6] == 4 * 77).all()
    assert (gy == 0).all() and (gx[1:-1, :5] == 0).all()


def test_edge_map_is_road_mask_and_threshold_on_sobel(oracle_mod):
    """The edge map of a whole detection, rebuilt independently: the road mask (finite l > 0,
    |l - f(v)| <= varpi in float32, interior pixels of rows >= v_top) and G_x^2 + G_y^2 > thr^2 with G from
    scipy's correlation of the bilateral output.  The edge count falls as the threshold rises."""
    cfg = scenes.SMALL_320x120
    d, im, _ = scenes.make_frame(cfg, 3)
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    counts = []
    for thr in (50, 100, 150):
        p = oracle_mod.default_params(n_disp=cfg.n_disp, edge_thresh=thr)
        r = oracle_mod.detect(d, im, p)
        I = r["Ibf"].astype(np.int64)
        gx = ndimage.correlate(I, kx, mode="constant")
        gy = ndimage.correlate(I, kx.T, mode="constant")
        H, W = I.shape
        v, u = np.arange(H)[:, None], np.arange(W)[None, :]
        with np.errstate(invalid="ignore"):
            road = (d > 0) & (np.abs(d - r["F"][:, None]) <= np.float32(p.varpi))
        road &= (v >= r["v_top"]) & (v >= 1) & (v <= H - 2) & (u >= 1) & (u <= W - 2)
        want = road & (gx * gx + gy * gy > thr * thr)
        assert (r["edge"].astype(bool) == want).all()
        assert (r["Gx"][want] == gx[want]).all() and (r["Gy"][want] == gy[want]).all()
        counts.append(int(want.sum()))
    assert counts[0] > counts[1] > counts[2] > 0


# ---------------------------------------------------------------------------------------------- b4
def test_band_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(5)
    for v_top, chi in [(0, 3), (10, 5), (25, 25), (39, 2)]:
        c = rng.integers(0, 5, size=(40, 33)).astype(np.int32)
        m = oracle_mod.band(c, v_top, chi, 2)
        for j in range(40):
            if j < v_top:
                assert (m[j] == 0).all()
                continue
            lo, hi = max(v_top, j - chi), min(39, j + chi)
            assert (m[j] == -2 * c[lo:hi + 1].sum(axis=0)).all()


# ---------------------------------------------------------------------------------------------- c1
def _tau_key(t):
    return (abs(t), 0 if t <= 0 else 1)


def _brute_dp_vpx(mx, v_top, tau, lam):
    H, W = mx.shape
    rows = list(range(v_top, H))
    best = None
    for u0 in range(W):
        for steps in itertools.product(range(-tau, tau + 1), repeat=len(rows) - 1):
            path = [u0]
            ok = True
            for s in steps:
                path.append(path[-1] + s)
                if not 0 <= path[-1] < W:
                    ok = False
                    break
            if not ok:
                continue
            e = sum(int(mx[v, u]) for v, u in zip(rows, path)) + lam * sum(abs(s) for s in steps)
            key = (e, u0, [_tau_key(s) for s in steps])
            if best is None or key < best[0]:
                best = (key, path)
    return best[0][0], best[1]


def test_dp_vpx_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(6)
    for trial in range(25):
        H, W, v_top = 6, 6, int(rng.integers(1, 3))
        tau = int(rng.integers(1, 3))
        mx = -rng.integers(0, 3 if trial % 2 else 2, size=(H, W)).astype(np.int32)
        e, path = oracle_mod.dp_vpx(mx, v_top, tau, 1)
        be, bpath = _brute_dp_vpx(mx, v_top, tau, 1)
        assert e == be
        assert path[v_top:].tolist() == bpath


# ---------------------------------------------------------------------------------------------- d1
def test_wg_table_against_direct_formula(oracle_mod):
    _, _, wg = oracle_mod.tables()
    assert wg[0] == 4096
    dth = np.arcsin(np.arange(16385) / 32768.0)
    ref = np.exp(-(dth / 3.5 ** 2) * 36.0 / math.pi) * 4096
    assert np.abs(wg - ref).max() <= 0.5 + 1e-9
    assert dth[-1] == pytest.approx(math.pi / 6)
    # monotone in the angle, and the value at the cut-off is exp(-(pi/6)*36/(pi*3.5^2))
    assert (np.diff(wg) <= 0).all()
    assert wg[-1] == math.floor(math.exp(-6.0 / 12.25) * 4096 + 0.5)


def test_bilateral_tables(oracle_mod):
    ws, wr, _ = oracle_mod.tables()
    assert ws[5, 5] == 32768 and wr[0] == 32768
    for dy in range(-5, 6):
        for dx in range(-5, 6):
            assert abs(ws[dy + 5, dx + 5] - 32768 * math.exp(-(dx * dx + dy * dy) / 9e4)) <= 0.5
    for k in range(256):
        assert abs(wr[k] - 32768 * math.exp(-((k / 255.0) ** 2) / 0.09)) <= 0.5


# ---------------------------------------------------------------------------------------------- d2
def test_box_sobel_matches_scipy(oracle_mod):
    rng = np.random.default_rng(7)
    gw = rng.integers(-4096 * 200, 4096 * 200, size=(30, 41)).astype(np.int32)
    m0, m1 = oracle_mod.box_sobel(gw, 1, 3)
    r0 = ndimage.correlate(gw.astype(np.int64), np.ones((7, 3), np.int64), mode="constant")
    # convolution with G = [1,2,1]^T [1,0,-1]  (scipy's convolve flips the kernel like the definition)
    G = np.outer([1, 2, 1], [1, 0, -1])
    r1 = ndimage.convolve(r0, G, mode="constant")
    assert (m0 == r0).all() and (m1 == r1).all()


def test_m1_minimum_at_stripe_centre(oracle_mod):
    """A narrow bright vertical stripe (G_x > 0 on its left edge, < 0 on its right) gives M_1 its minimum at the centre."""
    gw = np.zeros((20, 30), np.int32)
    gw[:, 14] = 1000   # dark -> light
    gw[:, 16] = -1000  # light -> dark
    _, m1 = oracle_mod.box_sobel(gw, 1, 3)
    assert int(np.argmin(m1[10])) == 15


# ---------------------------------------------------------------------------------------------- e1
def test_energy_straight_tracks_to_vanishing_point(oracle_mod):
    """On a flat road V_p is a fixed point, so Eq. 25 tracks are straight lines to it (closed form)."""
    H, W, v_top = 60, 80, 20
    vx, vy = 33.0, 12.0
    vpx = np.full(H, vx, np.float32)
    vpy = np.full(H, vy, np.float32)
    S0 = W // 2
    ns = W + 2 * S0
    rng = np.random.default_rng(8)
    m1 = rng.integers(-5, 6, size=(H, W)).astype(np.int32)
    he = oracle_mod.energy(m1, v_top, vpx, vpy, S0, ns, 1)
    checked = 0
    for i in range(ns):
        s = i - S0
        want = 0
        clean = True
        for v in range(v_top, H):
            u = vx + (s - vx) * (v - vy) / (H - 1 - vy)
            if abs((u + 0.5) - round(u + 0.5)) < 1e-3:
                clean = False  # a track passing through a rounding boundary: float32 and exact may differ
            c = math.floor(u + 0.5)
            if 0 <= c < W:
                want += int(m1[v, c])
        if clean:
            assert he[i] == want
            checked += 1
    assert checked > ns // 2


def test_energy_minimum_at_planted_lane(oracle_mod):
    H, W, v_top = 70, 90, 25
    vx, vy = 50.0, 15.0
    vpx = np.full(H, vx, np.float32)
    vpy = np.full(H, vy, np.float32)
    S0 = W // 2
    for s_star in (-20, 7, 44, 89, 110):
        m1 = np.zeros((H, W), np.int32)
        for v in range(v_top, H):
            u = vx + (s_star - vx) * (v - vy) / (H - 1 - vy)
            c = math.floor(u + 0.5)
            if 0 <= c < W:
                m1[v, c] = -100
        he = oracle_mod.energy(m1, v_top, vpx, vpy, S0, W + 2 * S0, 1)
        assert he.min() < 0 and int(np.argmin(he)) - S0 == s_star


# ---------------------------------------------------------------------------------------------- e2
def test_selection_properties_on_random_histograms(oracle_mod):
    rng = np.random.default_rng(9)
    for trial in range(200):
        n = int(rng.integers(3, 300))
        he = rng.integers(-1000, 200, size=n).astype(np.int64)
        if trial % 3 == 0:
            he = np.cumsum(rng.integers(-30, 31, size=n)).astype(np.int64)
        p = oracle_mod.default_params(thr_den=int(rng.choice([1, 4, 32])), near_px=int(rng.integers(0, 20)),
                                      max_lanes=int(rng.integers(1, 9)))
        S0 = 7
        out = oracle_mod.select(he, S0, p)
        mn = he.min()
        if mn >= 0:
            assert out["n_lanes"] == 0
            continue
        t = -((-mn * p.thr_num) // p.thr_den)
        cand = [i for i in range(1, n - 1) if he[i] < he[i - 1] and he[i] < he[i + 1] and he[i] < t]
        acc = [s + S0 for s in out["start_u"]]
        assert acc == sorted(acc) and len(acc) <= p.max_lanes
        assert set(acc) <= set(cand)
        assert [int(he[i]) for i in acc] == out["energy"]
        for a, b in itertools.combinations(acc, 2):
            assert abs(a - b) > p.near_px
        if len(acc) < p.max_lanes:
            # every rejected candidate is within near_px of an accepted one at least as deep
            for c in set(cand) - set(acc):
                assert any(abs(c - a) <= p.near_px and (he[a], a) < (he[c], c) for a in acc)
        if acc:
            best = min(cand, key=lambda i: (he[i], i))
            assert best in acc


# ---------------------------------------------------------------------------------------------- Alg. 7 drawing
def test_track_is_exact_on_straight_lanes(oracle_mod):
    """Flat road, constant V_p: every Eq. 25 step lands on the straight line through (s, H-1) and V_p."""
    H, vh, vp = 120, 40.0, 150.0
    vpx = np.full(H, vp, np.float32)
    vpy = np.full(H, vh, np.float32)
    for s in (-30, 12, 150, 290, 400):
        u = oracle_mod.track(vpx, vpy, 41, s)
        v = np.arange(H, dtype=np.float64)
        line = vp + (s - vp) * (v - vh) / (H - 1 - vh)
        assert np.isnan(u[:41]).all()
        assert np.allclose(u[41:], line[41:], atol=1e-3 * max(1, abs(s - vp)) + 1e-3)


def test_track_follows_planted_lanes(oracle_mod):
    """The planted lanes are field lines of the planted V_p (Eq. 14, Eq. 25): the track from a planted start,
    stepped on the planted V_p rows, stays within half a pixel of the lane curve on every road row."""
    cfg = scenes.SINGLE_1242x375
    H = cfg.height
    for fr in range(4):
        _, _, t = scenes.make_frame(cfg, fr)
        vt = int(np.ceil(t.v_horizon)) + 1
        vpx = np.where(np.isnan(t.vpx), 0, t.vpx).astype(np.float32)
        vpy = np.where(np.isnan(t.vpy), 0, t.vpy).astype(np.float32)
        fm = np.polyval(t.beta[::-1], H - 1)
        v = np.arange(vt, H)
        f = np.polyval(t.beta[::-1], v)
        for s in t.lane_starts:
            si = (s - t.alpha[0] - t.alpha[2] * fm * fm) / fm - t.alpha[1]
            lane = t.alpha[0] + (t.alpha[1] + si) * f + t.alpha[2] * f * f
            u = oracle_mod.track(vpx, vpy, vt, int(round(s)))
            # the start is rounded to a column: the offset scales with f along the field line
            assert np.abs(u[vt:] - (lane + (round(s) - s) * f / fm)).max() < 0.5


def test_track_energy_is_the_histogram_entry(oracle_mod):
    """Summing M_1 at the rounded track columns gives the start's entry of the energy histogram."""
    cfg = scenes.SINGLE_1242x375
    disp, img, _ = scenes.make_frame(cfg, 2)
    p = oracle_mod.default_params(n_disp=cfg.n_disp)
    r = oracle_mod.detect(disp, img, p)
    W, H = cfg.width, cfg.height
    S0 = (oracle_mod.n_starts(W, p) - W) // 2
    for s in list(r["start_u"]) + [-100, 7, 600, 1500]:
        u = oracle_mod.track(r["Vpx"], r["Vpy"], r["v_top"], int(s))
        e = 0
        for v in range(r["v_top"], H):
            c = np.floor(np.float32(u[v]) + np.float32(0.5))
            if 0 <= c < W:
                e += int(r["M1"][v, int(c)])
        assert e == int(r["HE"][int(s) + S0])
