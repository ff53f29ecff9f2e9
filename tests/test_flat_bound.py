"""The exact pruning bound of the gradient kernel (ld_flat_range): a road pixel whose neighbourhood spans
an image range of at most r_max cannot pass the edge test, whatever the values in it.

The bound is a derivation (include/ld.h, ld_flat_range); these tests check it against the oracle's exact
bilateral filter (Eq. 15-16, Q15 weights) and Sobel on adversarial images with values confined to a range
of r_max: steps at many angles and offsets, thin lines, stripes, checkerboards, two-level and uniform noise.
A pixel qualifies when the windows of its 3x3 neighbours lie inside the image (rows and columns
rho + 1 .. size - rho - 2).  They also check that the library's value follows from the oracle's own tables
and that the bound is not vacuous: a clear step does pass the edge test.
"""
import ctypes as C
import math

import numpy as np
import pytest


def _lib_flat_range(p):
    from paper_1807_02752_gb300 import ld
    L = ld.load()
    return int(L.ld_flat_range(C.byref(p)))


def _derived_flat_range(oracle_mod, **kw):
    """The bound from the oracle's Q15 tables, evaluated step by step in exact rationals."""
    from fractions import Fraction
    p = oracle_mod.default_params(**kw)
    if p.bilateral != 1:
        return -1
    ws, wr, _ = oracle_mod.tables(p)
    ws = ws.ravel().astype(np.int64)
    N = 2 * p.bf_rho + 1
    b = int(((ws * int(wr[0]) + 16384) >> 15).max())
    best = -1
    for r in range(255):
        a = int(((ws * int(wr[r]) + 16384) >> 15).min())
        if a <= 0:
            break
        e = Fraction(b - a) * r / (4 * a) + Fraction(1, 2)
        g = 4 * (Fraction(2 * r, N) + 2 * e)
        if 2 * g * g > p.edge_thresh ** 2:
            break
        best = r
    return best


@pytest.mark.parametrize("kw", [{}, {"bf_rho": 3}, {"bf_rho": 1}, {"edge_thresh": 50}, {"sigma_r": 0.2},
                                {"sigma_s": 30.0}, {"bilateral": 0}, {"bilateral": 2}])
def test_library_bound_follows_from_the_tables(oracle_mod, kw):
    from paper_1807_02752_gb300 import ld
    assert _lib_flat_range(ld.default_params(**kw)) == _derived_flat_range(oracle_mod, **kw)


def _patterns(rng, n, m, r):
    """Images of size n x n with every value in [m, m + r]."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    out = []
    for ang in np.linspace(0, math.pi, 13, endpoint=False):
        for off in (0.0, 0.3, 0.5, 0.77):
            d = (xx - n / 2 - off) * math.cos(ang) + (yy - n / 2) * math.sin(ang)
            out.append(np.where(d > 0, m + r, m))                                    # step edge
            out.append(np.where(np.abs(d) < 0.5 + off, m + r, m))                      # thin line
            out.append(np.clip(m + r * (0.5 + d / 6.0), m, m + r))                     # ramp
    for w in (1, 2, 3, 5):
        out.append(np.where((xx // w) % 2 == 0, m + r, m))                             # stripes
        out.append(np.where(((xx // w) + (yy // w)) % 2 == 0, m + r, m))               # checkerboard
    for _ in range(12):
        out.append(m + r * (rng.random((n, n)) < rng.uniform(0.05, 0.95)))              # two-level noise
        out.append(m + rng.integers(0, r + 1, size=(n, n)))                             # uniform noise
    return [np.clip(np.rint(x), m, m + r).astype(np.uint8) for x in out]


@pytest.mark.parametrize("kw", [{}, {"bf_rho": 3}, {"edge_thresh": 50}])
def test_pixels_within_the_range_never_pass_the_edge_test(oracle_mod, kw):
    from paper_1807_02752_gb300 import ld
    p = oracle_mod.default_params(**kw)
    r_max = _lib_flat_range(ld.default_params(**kw))
    assert r_max > 0
    rng = np.random.default_rng(20240)
    n, rho = 40, p.bf_rho
    lo, hi = rho + 1, n - rho - 2
    thr2 = p.edge_thresh ** 2
    worst = 0
    for m in (0, 37, 128, 255 - r_max):
        for img in _patterns(rng, n, m, r_max):
            gx, gy = oracle_mod.sobel(oracle_mod.bilateral(img, p))
            g2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
            worst = max(worst, int(g2[lo:hi + 1, lo:hi + 1].max()))
    assert worst <= thr2, f"a pixel within range {r_max} passed the edge test: G^2 = {worst} > {thr2}"
    assert worst > 0


def test_bound_is_not_vacuous(oracle_mod):
    """A clear step (range 120 at the paper's parameters) passes the edge test: pruning must stop below it."""
    from paper_1807_02752_gb300 import ld
    p = oracle_mod.default_params()
    assert _lib_flat_range(ld.default_params()) < 120
    img = np.full((40, 40), 100, np.uint8)
    img[:, 20:] = 220
    gx, gy = oracle_mod.sobel(oracle_mod.bilateral(img, p))
    assert (gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2).max() > p.edge_thresh ** 2
