"""Pins of the learned-proposal oracle (oracle/proposal.py) against things other than itself: a library's
bf16 conversion, scipy's correlation, adjoint identities, finite differences, torch's Adam, closed-form
straight-line tracks (fixed vanishing point), the C oracle's Alg. 7 selection, and hand-worked cases."""
import math

import numpy as np
import pytest

import oracle
from oracle import proposal as P


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(1e3)
    # exact ties in both parities, and values just above / below a tie
    base = rng.integers(0x3F800000, 0x47000000, 2000, dtype=np.uint64).astype(np.uint32) & np.uint32(0xFFFF0000)
    ties = np.concatenate([base | np.uint32(0x8000), (base + np.uint32(0x10000)) | np.uint32(0x8000),
                           base | np.uint32(0x8001), base | np.uint32(0x7FFF)]).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(P.bf16(x), want)


def test_conv3x3_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 7, 9))
    w = rng.standard_normal((4, 3, 3, 3))
    got = P.conv3x3(x, w)
    want = np.zeros((4, 7, 9))
    for o in range(4):
        for c in range(3):
            want[o] += signal.correlate2d(x[c], w[o, c], mode="same", boundary="fill", fillvalue=0)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_backward_operators_are_adjoints():
    """<conv(x, w), d> = <x, conv_T(d, w)> = <w, wgrad(d, x)> for any x, w, d (ragged sizes)."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((5, 6, 11))
    w = rng.standard_normal((3, 5, 3, 3))
    d = rng.standard_normal((3, 6, 11))
    lhs = float(np.sum(P.conv3x3(x, w) * d))
    assert math.isclose(lhs, float(np.sum(x * P.conv3x3_transpose(d, w))), rel_tol=1e-11)
    assert math.isclose(lhs, float(np.sum(w * P.conv3x3_wgrad(d, x))), rel_tol=1e-11)


def _random_params(seed, scale=0.4):
    rng = np.random.default_rng(seed)
    return {name: rng.standard_normal(shape) * scale for name, shape in P.param_shapes()}


def test_gradient_matches_central_differences():
    """Exact mode (no rounding): the analytic gradient of every parameter group against central differences."""
    rng = np.random.default_rng(4)
    params = _random_params(5)
    params["bh"][:] = -0.5
    X = rng.random((2, 5, 7)) * 2.0
    Y = (rng.random((2, 5, 7)) < 0.2).astype(np.uint8)
    _, g = P.loss_and_grad(params, X, Y, exact=True)
    flat = P.pack(params)
    gflat = P.pack(g)
    h = 1e-6
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in P.param_shapes()])
    picks = []
    for k in range(len(offs) - 1):
        picks += list(rng.choice(np.arange(offs[k], offs[k + 1]), size=min(6, offs[k + 1] - offs[k]), replace=False))
    for i in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = P.loss_and_grad(P.unpack(fp), X, Y, exact=True)
        lm, _ = P.loss_and_grad(P.unpack(fm), X, Y, exact=True)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-5 * max(1e-3, abs(fd)), (i, fd, gflat[i])


def test_rounding_points_keep_representable_values():
    """With small-integer inputs and weights in {-1, 0, 1} every product and sum is exact in bf16/f32
    (activations stay below 2^8), so the rounded forward pass equals the exact one."""
    rng = np.random.default_rng(6)
    params = {name: rng.integers(-1, 2, shape).astype(np.float64) for name, shape in P.param_shapes()}
    for l in range(1, 5):
        params[f"W{l}"] *= (rng.random(params[f"W{l}"].shape) < 0.08)
    X = rng.integers(0, 3, (6, 9)).astype(np.float64)
    ex = P.forward(params, X, exact=True)
    rd = P.forward(params, X, exact=False)
    assert max(float(a.max()) for a in ex["A"]) < 256
    assert all(np.array_equal(a, b) for a, b in zip(ex["A"], rd["A"])) and np.array_equal(ex["z"], rd["z"])


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    t = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    th = theta.copy()
    for k, g in enumerate(grads):
        opt.zero_grad()
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = P.adam(th, g, m, v, k + 1, 3e-3)
    assert np.allclose(th, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_xmap_sums_hand_example_and_total():
    Gw = np.arange(-15, 15, dtype=np.int32).reshape(5, 6)
    s = P.xmap_sums(Gw)
    assert s.shape == (2, 2)
    a = np.abs(np.arange(-15, 15)).reshape(5, 6)
    assert s[0, 0] == a[0:4, 0:4].sum() == 15 + 14 + 13 + 12 + 9 + 8 + 7 + 6 + 3 + 2 + 1 + 0 + 3 + 4 + 5 + 6
    assert s[1, 1] == 13 + 14       # the ragged corner holds row 4 (9..14), columns 4..5
    assert s.sum() == a.sum()
    rng = np.random.default_rng(9)
    big = rng.integers(-2 ** 22, 2 ** 22, (37, 45)).astype(np.int32)
    assert P.xmap_sums(big).sum() == np.abs(big.astype(np.int64)).sum()


def test_xmap_input_values():
    s = np.array([0, 2 ** 22, 3 * 2 ** 22 + 1, 2 ** 24 + 1, 2 ** 26 - 1, 5 * 2 ** 20], np.int64)
    got = P.xmap_input(s)
    # 2^24 + 1 rounds to 2^24 in float32; 2^26 - 1 rounds to 2^26; 5/4 = 1.25 is exact in bf16
    assert list(got) == [0.0, 1.0, 3.0, 4.0, 16.0, 1.25]


def _line(s, c, h0, H, v):
    """Track of start s under a fixed vanishing point (c, h0): the straight line through (s, H-1)."""
    return c + (s - c) * (v - h0) / (H - 1 - h0)


def test_labels_follow_straight_tracks_under_fixed_vanishing_point():
    H, W, v_top = 60, 90, 25
    c, h0 = 47.3, 12.6
    Vpx = np.full(H, c, np.float32)
    Vpy = np.full(H, h0, np.float32)
    starts = [5, 40, 88, 120, -30]
    Y = P.lane_labels(starts, Vpx, Vpy, v_top, H, W)
    sure, maybe = set(), set()
    for s in starts:
        for v in range(v_top, H):
            u = _line(s, np.float64(np.float32(c)), np.float64(np.float32(h0)), H, v) + 0.5
            for col, tgt in ((math.floor(u), sure), (math.floor(u - 1e-2), maybe), (math.floor(u + 1e-2), maybe)):
                if 0 <= col < W:
                    (tgt if abs(u - round(u)) > 1e-2 else maybe).add((v >> 2, col >> 2))
    marked = set(zip(*np.nonzero(Y)))
    assert sure <= marked
    assert marked <= sure | maybe
    assert Y[:v_top >> 2].sum() == 0 or (v_top >> 2) == (v_top - 1) >> 2


def test_coarse_scores_count_steps_on_straight_tracks():
    H, W, v_top = 64, 80, 21
    c, h0 = 33.7, 9.2
    Vpx = np.full(H, c, np.float32)
    Vpy = np.full(H, h0, np.float32)
    S0 = 40
    ns = W + 2 * S0
    h, w = P.map_shape(H, W)
    rng = np.random.default_rng(10)
    z = rng.standard_normal((h, w)).astype(np.float32)
    got = P.coarse_scores(z, Vpx, Vpy, v_top, H, W, S0, ns)
    assert got.shape == ((ns + 3) // 4,)
    cf, hf = np.float64(np.float32(c)), np.float64(np.float32(h0))
    for k in range(len(got)):
        s = 4 * k - S0 + 1.5
        want, ambiguous = 0.0, False
        for v in range(H - 1, v_top - 1, -4):
            u = _line(s, cf, hf, H, v) + 0.5
            ambiguous |= abs(u - round(u)) < 1e-2
            col = math.floor(u)
            if 0 <= col < W:
                want += float(z[v >> 2, col >> 2])
        if not ambiguous:
            assert abs(float(got[k]) - want) <= 1e-4 * (1 + abs(want)), k


def test_top_k_and_candidate_sets_hand_cases():
    assert list(P.top_k(np.array([1.0, 3.0, 3.0, 2.0], np.float32), 2)) == [1, 2]
    assert list(P.top_k(np.array([0.5, 0.5, 0.5], np.float32), 5)) == [0, 1, 2]
    cand, ev = P.candidate_sets(np.array([0, 2]), 11)
    assert list(np.nonzero(cand)[0]) == [0, 1, 2, 3, 8, 9, 10]
    assert list(np.nonzero(ev)[0]) == [0, 1, 2, 3, 4, 7, 8, 9, 10]


def _planted_energies(rng, ns):
    he = rng.integers(-50, 0, ns).astype(np.int64)
    for centre in rng.choice(np.arange(5, ns - 5), 6, replace=False):
        he[centre - 2:centre + 3] -= np.array([300, 600, 1000, 600, 300]) * int(rng.integers(1, 5))
    return he


def test_selection_over_every_start_equals_alg7():
    """With every start a candidate the proposal's selection is the exhaustive Alg. 7 (C oracle)."""
    p = oracle.default_params()
    rng = np.random.default_rng(11)
    for trial in range(30):
        ns = int(rng.integers(20, 400))
        S0 = ns // 4
        he = _planted_energies(rng, ns)
        if trial % 5 == 0:
            he[rng.integers(0, ns)] = he.min()          # equal energies
        cand = np.ones(ns, bool)
        got = P.select_on_set(he, cand, cand, S0, p.thr_num, p.thr_den, p.near_px, p.max_lanes)
        want = oracle.select(he, S0, p)
        assert got[0] == want["start_u"] and got[1] == want["energy"], trial


def test_selection_on_a_subset_only_tests_candidates():
    """Candidates 2 and 9 with their neighbours evaluated; start 6 (the deepest) is not, so it is missed.
    Minimum over the evaluated starts -9 gives t = -(9 // 4) = -2; both candidates are strict minima below t."""
    he = np.array([0, -5, -9, -5, 0, -1, -20, -1, 0, -3, -2, 0], np.int64)
    cand = np.zeros(12, bool)
    cand[[2, 9]] = True
    ev = cand.copy()
    ev[[1, 3, 8, 10]] = True
    assert P.select_on_set(he, cand, ev, 0, 1, 4, 1, 8) == ([2, 9], [-9, -3])
    assert P.select_on_set(he, cand, ev, 5, 1, 4, 7, 8) == ([-3], [-9])      # 9 suppressed (|9 - 2| <= 7)


def test_agreement_hand_cases():
    assert P.agreement([], []) == 1.0
    assert P.agreement([1, 2, 3], [1, 2, 3]) == 1.0
    assert P.agreement([1, 2], [2, 3]) == 0.5
    assert P.agreement([1], []) == 0.0
    assert math.isclose(P.agreement([1, 2, 3], [3]), 0.5)


def test_param_count_and_layout():
    assert P.param_count() == 160 + 4640 + 9248 + 4624 + 17 == 18689
    flat = np.arange(P.param_count(), dtype=np.float64)
    d = P.unpack(flat)
    assert d["W2"].shape == (32, 16, 3, 3) and d["W2"][0, 0, 0, 0] == 160
    assert np.array_equal(P.pack(d), flat)


def test_forward_on_a_real_frame_shapes():
    from paper_1807_02752_gb300 import scenes

    cfg = scenes.SMALL_320x120
    disp, img, _ = scenes.make_frame(cfg, 3)
    r = oracle.detect(disp, img, oracle.default_params(n_disp=cfg.n_disp))
    X = P.xmap_input(P.xmap_sums(r["Gw"]))
    assert X.shape == (30, 80) and X.max() > 0
    fw = P.forward(_random_params(12, 0.2), X)
    assert fw["z"].shape == (30, 80) and [a.shape[0] for a in fw["A"]] == [1, 16, 32, 32, 16]
