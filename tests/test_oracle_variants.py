"""Pins of the oracle's paper-literal variants: the median pre-filter of the authors' previous system
(Sec. 2.3.1), the Gaussian form of the w_g weight that Sec. 2.4's text names (Eq. 23 prints an exponential
linear in the angle), and an absolute lane threshold (Alg. 7 gives no value)."""
import math

import numpy as np
import pytest

import oracle


def test_median_interior_matches_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (40, 57), dtype=np.uint8)
    got = oracle.median(img, 5)
    want = ndimage.median_filter(img, size=11, mode="constant")
    assert np.array_equal(got[5:-5, 5:-5], want[5:-5, 5:-5])
    got3 = oracle.median(img, 1)
    assert np.array_equal(got3[1:-1, 1:-1], ndimage.median_filter(img, size=3)[1:-1, 1:-1])


def test_median_clipped_window_hand_cases():
    img = np.array([[9, 1, 5], [3, 7, 2], [8, 4, 6]], np.uint8)
    m = oracle.median(img, 1)
    # corner (0,0): taps 9 1 3 7 -> sorted 1 3 7 9, lower median (2nd) = 3
    assert m[0, 0] == 3
    # edge (0,1): taps 9 1 5 3 7 2 -> 1 2 3 5 7 9, lower median (3rd) = 3
    assert m[0, 1] == 3
    # centre: all nine -> 1 2 3 4 5 6 7 8 9, median 5
    assert m[1, 1] == 5
    # corner (2,2): taps 7 2 4 6 -> 2 4 6 7 -> 4
    assert m[2, 2] == 4
    const = np.full((12, 13), 77, np.uint8)
    assert (oracle.median(const, 5) == 77).all()


def test_wg_gaussian_table_closed_form():
    p = oracle.default_params(wg_gaussian=1)
    _, _, wg = oracle.tables(p)
    s = p.sigma_g ** 2
    assert wg[0] == 4096
    # i = 16384: sin(dtheta) = 1/2, dtheta = pi/6, p = 6
    assert wg[16384] == math.floor(math.exp(-36.0 / s) * 4096 + 0.5)
    # i = round(sin(pi/36) 2^15) is within one index of p = 1
    i1 = int(math.sin(math.pi / 36) * 32768)
    assert abs(wg[i1] - math.exp(-1.0 / s) * 4096) <= 4096 * (math.exp(-0.99 / s) - math.exp(-1.0 / s)) + 1
    assert (np.diff(wg) <= 0).all()
    printed = oracle.tables(oracle.default_params())[2]
    assert printed[16384] == math.floor(math.exp(-6.0 / s) * 4096 + 0.5)
    # the Gaussian falls slower than the printed form near 0 and faster beyond p = 1
    assert wg[i1 // 2] > printed[i1 // 2] and wg[16384] < printed[16384]


def test_absolute_threshold_selection():
    he = np.array([0, -5, -90, -5, 0, -1, -40, -1, 0, -3, -20, -3, 0], np.int64)
    rel = oracle.select(he, 0, oracle.default_params(near_px=1))
    assert rel["start_u"] == [2, 6, 10]                 # t = -(90 // 32) = -2
    ab = oracle.select(he, 0, oracle.default_params(near_px=1, thr_abs=-30))
    assert ab["start_u"] == [2, 6] and ab["energy"] == [-90, -40]
    none = oracle.select(he, 0, oracle.default_params(near_px=1, thr_abs=-100))
    assert none["n_lanes"] == 0 and none["flags"] & oracle.F_NO_LANES


def _brute_dp_literal(my, tau, lam):
    """Every path of Eq. 12 as printed: v_{d+1} = v_d - tau_d, energy sum(-m_y) - lam sum(tau); ties to the
    smaller start row, then the smaller steps in order."""
    import itertools

    H, D = my.shape
    best = None
    for v1 in range(H):
        for steps in itertools.product(range(tau + 1), repeat=D - 2):
            path = [v1]
            for st in steps:
                path.append(path[-1] - st)
            if min(path) < 0:
                continue
            e = sum(-int(my[path[i], i + 1]) for i in range(D - 1)) - lam * sum(steps)
            key = (e, v1, steps)
            if best is None or key < best[0]:
                best = (key, path)
    return best[0][0], best[1]


def test_literal_road_dp_matches_brute_force():
    rng = np.random.default_rng(21)
    for trial in range(30):
        H, D, tau = 7, 5, int(rng.integers(1, 4))
        lam = int(rng.integers(0, 3))
        my = rng.integers(0, 4 if trial % 2 else 2, size=(H, D)).astype(np.int32)
        e, path = oracle.dp_vdisp_literal(my, tau, lam)
        be, bpath = _brute_dp_literal(my, tau, lam)
        assert e == be and path[1:].tolist() == bpath, (trial, e, be, path, bpath)


def test_literal_bottom_band_matches_brute_force():
    """Alg. 5 with the listing's bottom rows: band [j, v_max] for j > v_max - chi - 1, else [j - chi, j + chi],
    clipped to [v_top, v_max]."""
    rng = np.random.default_rng(31)
    for trial in range(20):
        H, W = int(rng.integers(10, 40)), int(rng.integers(5, 20))
        chi, rho, v_top = int(rng.integers(0, 8)), int(rng.integers(1, 4)), int(rng.integers(0, 6))
        votes = rng.integers(0, 3, (H, W)).astype(np.int32)
        got = oracle.band(votes, v_top, chi, rho, literal_bottom=True)
        want = np.zeros((H, W), np.int64)
        for j in range(v_top, H):
            lo, hi = (j, H - 1) if j > H - 1 - chi - 1 else (max(v_top, j - chi), min(H - 1, j + chi))
            want[j] = -rho * votes[lo:hi + 1].sum(axis=0)
        assert np.array_equal(got, want), trial
        assert np.array_equal(oracle.band(votes, v_top, chi, rho)[:max(v_top, H - 1 - chi)],
                              got[:max(v_top, H - 1 - chi)])
