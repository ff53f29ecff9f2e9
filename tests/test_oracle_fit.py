"""Pins of the oracle's random numbers, least squares fits and RANSAC loop (Alg. 4, Alg. 6, Eq. 13, 19-20).

Each check compares the oracle with something other than itself: published known-answer vectors, numpy's
least squares routine, exact polynomial data, or brute-force consensus counts.
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = oracle_mod.philox(vals[0:4], vals[4:6])
        assert out.tolist() == vals[6:10]


def _vander(tau, m):
    return np.stack([tau ** k for k in range(m)], axis=1)


@pytest.mark.parametrize("m,H", [(3, 375), (5, 375), (5, 1080), (3, 1080)])
def test_lsf_recovers_planted_polynomial(oracle_mod, m, H):
    rng = np.random.default_rng(m * 1000 + H)
    centre, e = oracle_mod.basis(H)
    for _ in range(20):
        x = np.sort(rng.choice(H, size=60, replace=False)).astype(np.int32)
        # integer-valued data on an exact polynomial: y = sum c_k t^k with t = x - centre, c integer-friendly
        t = (x - centre).astype(np.float64)
        c = rng.integers(-3, 4, size=m).astype(np.float64) / np.array([1, 4, 64, 4096, 262144][:m])
        y = np.rint(_vander(t, m) @ c)
        # keep only exact points so the fit is noise-free
        exact = np.abs(_vander(t, m) @ c - y) == 0
        if exact.sum() < m + 2:
            continue
        rc, coef = oracle_mod.lsf(x[exact], y[exact].astype(np.int32), m, centre, e)
        assert rc == 0
        want = c * (2.0 ** (e * np.arange(m)))  # coefficients of tau = t / 2^e
        assert np.allclose(coef, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


@pytest.mark.parametrize("m", [3, 5])
def test_lsf_matches_numpy_lstsq(oracle_mod, m):
    rng = np.random.default_rng(7 + m)
    H = 375
    centre, e = oracle_mod.basis(H)
    for _ in range(20):
        n = int(rng.integers(m + 3, 300))
        x = rng.integers(0, H, size=n).astype(np.int32)
        y = rng.integers(-50, 1300, size=n).astype(np.int32)
        if len(np.unique(x)) < m:
            continue
        rc, coef = oracle_mod.lsf(x, y, m, centre, e)
        assert rc == 0
        tau = (x - centre) / 2.0 ** e
        ref, *_ = np.linalg.lstsq(_vander(tau, m), y.astype(np.float64), rcond=None)
        assert np.allclose(coef, ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_lsf_rejects_too_few_distinct_rows(oracle_mod):
    x = np.array([10, 10, 10, 20], np.int32)
    y = np.array([1, 2, 3, 4], np.int32)
    rc, _ = oracle_mod.lsf(x, y, 3, 187, 8)
    assert rc == -1
    rc, _ = oracle_mod.lsf(x[:2], y[:2], 3, 187, 8)
    assert rc == -1


def test_ransac_separates_planted_outliers(oracle_mod):
    """Inliers within 0.5 of a parabola, outliers >= 10x the tolerance away: the final set is exactly the inliers."""
    rng = np.random.default_rng(3)
    H = 375
    centre, e = oracle_mod.basis(H)
    p = oracle_mod.default_params()
    for trial in range(10):
        n = 120
        x = np.sort(rng.choice(H, size=n, replace=False)).astype(np.int32)
        f = 0.0004 * (x - 120.0) ** 2 + 0.33 * (x - 120.0)
        y = np.rint(f).astype(np.int32)
        out = rng.random(n) < 0.3
        y[out] += (rng.choice([-1, 1], size=out.sum()) * rng.integers(7, 40, size=out.sum())).astype(np.int32)
        fl, mem, coef, rounds = oracle_mod.ransac(x, y, 3, 4.0, 0, p, centre, e)
        assert fl == 0
        assert mem.astype(bool).tolist() == (~out).tolist()
        tau = (x - centre) / 2.0 ** e
        assert np.abs(_vander(tau, 3) @ coef - f).max() < 0.5


def test_ransac_quartic_with_outliers(oracle_mod):
    rng = np.random.default_rng(4)
    H = 375
    centre, e = oracle_mod.basis(H)
    p = oracle_mod.default_params()
    v = np.arange(120, H).astype(np.int32)
    g = 600 - 3e-7 * (v - 100.0) ** 4 + 0.2 * (v - 100)
    y = np.rint(g).astype(np.int32)
    out = rng.random(v.size) < 0.35
    y[out] = rng.integers(0, 1242, size=out.sum())
    far = np.abs(y - g) > 40
    fl, mem, coef, rounds = oracle_mod.ransac(v, y, 5, 16.0, 1, p, centre, e)
    assert fl == 0
    # every planted inlier stays, every far outlier leaves
    assert mem[~out].all()
    assert not mem[far].any()
    tau = (v - centre) / 2.0 ** e
    assert np.abs(_vander(tau, 5) @ coef - g).max() < 1.0


def test_hypothesis_score_is_brute_force_consensus(oracle_mod):
    """The score of each hypothesis equals the consensus count of the exact polynomial through its sample."""
    rng = np.random.default_rng(5)
    H = 375
    centre, e = oracle_mod.basis(H)
    p = oracle_mod.default_params()
    for m, tr in [(3, 4.0), (5, 16.0)]:
        n = 40
        x = np.sort(rng.choice(np.arange(100, H), size=n, replace=False)).astype(np.int32)
        y = rng.integers(0, 200, size=n).astype(np.int32)
        member = np.ones(n, np.uint8)
        member[rng.random(n) < 0.2] = 0
        checked = 0
        for h in range(64):
            cnt, chosen, inl = oracle_mod.hypothesis(x, y, member, m, tr, 1, 0, h, p, centre, e)
            if cnt < 0:
                continue
            tau = (x - centre) / 2.0 ** e
            A = _vander(tau[chosen], m)
            c = np.linalg.solve(A, y[chosen].astype(np.float64))
            r2 = (y - _vander(tau, m) @ c) ** 2
            if np.any(np.abs(r2 - tr) < 1e-2):
                continue  # a residual on the tolerance: float32 and float64 may legitimately differ
            ref = (r2 < tr) & member.astype(bool)
            assert inl.astype(bool).tolist() == ref.tolist()
            assert cnt == ref.sum()
            assert all(member[chosen]) and len(set(x[chosen].tolist())) == m
            checked += 1
        assert checked > 40


def test_hypothesis_draws_follow_philox_stream(oracle_mod):
    """The sample is the first m distinct-row draws of the Philox stream at (stage<<24|round, hyp, block)."""
    p = oracle_mod.default_params(seed=0x1234_5678_9ABC_DEF0)
    x = np.arange(50, 80, dtype=np.int32)
    x[5] = x[4]  # a repeated row must never be chosen twice
    y = np.zeros(30, np.int32)
    member = np.ones(30, np.uint8)
    member[::7] = 0
    lst = np.nonzero(member)[0]
    key = [p.seed & 0xFFFFFFFF, p.seed >> 32]
    for stage, rnd, hyp, m in [(0, 0, 0, 3), (1, 3, 17, 5), (0, 63, 63, 3)]:
        _, chosen, _ = oracle_mod.hypothesis(x, y, member, m, 4.0, stage, rnd, hyp, p, 187, 8)
        want = []
        for j in range(8 * m):
            if len(want) == m:
                break
            w = oracle_mod.philox([(stage << 24) | rnd, hyp, j >> 2, 0], key)[j & 3]
            pt = int(lst[(int(w) * len(lst)) >> 32])
            if pt not in want and x[pt] not in [x[q] for q in want]:
                want.append(pt)
        assert chosen.tolist() == want


def test_exhaustive_consensus_on_tiny_sets(oracle_mod):
    """With enough hypotheses the first RANSAC round reaches the brute-force maximum consensus."""
    rng = np.random.default_rng(11)
    H = 375
    centre, e = oracle_mod.basis(H)
    p = oracle_mod.default_params(ransac_hyps=4096, ransac_rounds=1)
    for trial in range(4):
        n = 10
        x = np.sort(rng.choice(np.arange(100, H), size=n, replace=False)).astype(np.int32)
        y = np.rint(0.3 * (x - 100) + rng.normal(0, 1.0, n)).astype(np.int32)
        y[rng.random(n) < 0.3] += 30
        tau = (x - centre) / 2.0 ** e
        best = 0
        for comb in itertools.combinations(range(n), 3):
            c = np.linalg.solve(_vander(tau[list(comb)], 3), y[list(comb)].astype(np.float64))
            best = max(best, int(((y - _vander(tau, 3) @ c) ** 2 < 4.0).sum()))
        fl, mem, coef, rounds = oracle_mod.ransac(x, y, 3, 4.0, 0, p, centre, e)
        assert rounds == 1
        assert mem.sum() == best
