"""End-to-end pins of the oracle on scenes with closed-form ground truth.

The scene generator plants the road profile f(v), the vanishing point V_p(v) = (V_px, V_py) and the lane
markings u_i(v) in closed form (Eq. 14 and the field lines of Eq. 25); the oracle must recover them.
"""
import math

import numpy as np
import pytest

from paper_1807_02752_gb300 import scenes

from e2e_eval import score_many


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


# ---------------------------------------------------------------------------------------------------------
# End to end on the planted scenes, 40 seeds of the 1242x375 recipe and 30 of the 1920x1080 stress recipe.
#
# What limits the accuracy (measured on these seeds; each bound below is the measured figure plus a margin):
# * road profile: the Eq. 12 path holds one row per integer disparity bin, about three rows per bin on
#   these roads, so the points of Eq. 13 are quantised by up to half a bin;
# * V_px: the Eq. 17 vote of an edge pixel is the Sobel direction extended over the lever arm v - V_py
#   (about 250 rows at the bottom of a 375-row frame, 700 at 1080).  The 3x3 Sobel direction of these
#   sharp, anti-aliased markings is off by 1-2 degrees near vertical and 2-6 degrees on markings inclined
#   near 67 degrees, so the votes of one row scatter over tens of pixels at the bottom; the band of Alg. 5
#   and the Eq. 18 path follow that scatter, and the quartic of Alg. 6 follows the path to 2-3 degrees in
#   the median.  The error is therefore measured as the angle atan(|dV_px| / (v - V_py)), on the rows
#   spanned by the final RANSAC set; below that span the quartic extrapolates and is not bounded;
# * lane starts: M_1 = G * M_0 with a 3-column box is zero inside a marking wider than about 5 px, so a
#   marking 8-15 px wide at the bottom rows gives two energy valleys, one at each edge, and the deepest
#   energy lies up to about half the width from the centre even with the planted V_p;
# * faint lanes: a marking inclined near 67 degrees has G_x = |G| cos(theta) and a horizontal cross
#   section stretched by 1 / cos(theta), so its energy is 2-9 % of a vertical marking's, near the 1/32
#   threshold of the selection.
# ---------------------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def scored_1242x375(oracle_mod):
    return score_many("single_1242x375", range(40))


@pytest.fixture(scope="module")
def scored_1920x1080(oracle_mod):
    return score_many("batch16_1920x1080", range(30))


def _arr(rs, key):
    return np.array([r[key] for r in rs])


@pytest.mark.parametrize("which,f_p95,f_max,vpy_med", [("scored_1242x375", 0.75, 1.0, 1.5),
                                                       ("scored_1920x1080", 0.5, 0.6, 2.0)])
def test_planted_road_profile_recovered(request, which, f_p95, f_max, vpy_med):
    """Sec. 2.2: the road profile f(v), its zero f^-1(0) and V_py (Eq. 14) from the disparity alone."""
    rs = request.getfixturevalue(which)
    assert (_arr(rs, "flags") == 0).all()
    assert _arr(rs, "v_top_err").max() <= 2.0
    assert _arr(rs, "f_med").max() <= 0.25          # disparity units
    assert _arr(rs, "f_p95").max() <= f_p95
    assert _arr(rs, "f_max").max() <= f_max
    assert _arr(rs, "vpy_med").max() <= vpy_med     # rows


@pytest.mark.parametrize("which,per_frame,overall,cover", [("scored_1242x375", 10.0, 2.5, 0.6),
                                                           ("scored_1920x1080", 14.0, 3.0, 0.3)])
def test_planted_vanishing_point_within_sobel_angle(request, which, per_frame, overall, cover):
    """Sec. 2.3: V_px(v) (Eq. 22) on the rows spanned by the final RANSAC set of Alg. 6, as the angle by
    which it turns the Eq. 25 tracks: within a few degrees, the angular accuracy of the Sobel directions
    that cast the Eq. 17 votes."""
    rs = request.getfixturevalue(which)
    ang = _arr(rs, "ang_support_med")
    assert ang.max() <= per_frame                  # degrees, median over the frame's rows
    assert np.median(ang) <= overall
    assert _arr(rs, "support_cover").min() >= cover


@pytest.mark.parametrize("which,minima,recall,extra,rel_max", [("scored_1242x375", 0.98, 0.75, 0.3, 1.5),
                                                               ("scored_1920x1080", 1.0, 0.8, 1.2, 1.5)])
def test_planted_lanes_are_energy_minima(request, which, minima, recall, extra, rel_max):
    """Eq. 24-25 and Alg. 7 on the frame's own M_1 with the planted V_p: every visible marking has a strict
    local minimum of the start histogram within half its width + 2 px of its planted start; the selection
    keeps most of them and few others; each kept start lies within the marking (error relative to half
    the marking width)."""
    rs = request.getfixturevalue(which)
    near = np.concatenate([r["minima_near"] for r in rs])
    assert near.mean() >= minima
    hits, misses = _arr(rs, "t_hits").sum(), _arr(rs, "t_misses").sum()
    assert hits >= recall * (hits + misses)
    assert _arr(rs, "t_extra").mean() <= extra
    rel = np.concatenate([r["t_rel"] for r in rs])
    assert rel.max() <= rel_max and np.median(rel) <= 0.6


@pytest.mark.parametrize("which,recall,extra", [("scored_1242x375", 0.78, 0.6), ("scored_1920x1080", 0.3, 5.0)])
def test_end_to_end_lanes(request, which, recall, extra):
    """The whole path from disparity and image: planted markings matched by detected starts (half the
    marking width + 3 px).  At 1920x1080 the V_px error of the bottom third of the road (median 5 degrees,
    up to 78) moves the tracks off the markings, so fewer are found than with the planted V_p above."""
    rs = request.getfixturevalue(which)
    hits, misses = _arr(rs, "hits").sum(), _arr(rs, "misses").sum()
    assert hits >= recall * (hits + misses)
    assert _arr(rs, "extra").mean() <= extra
    rel = np.concatenate([r["rel"] for r in rs])
    assert np.median(rel) <= 0.6
