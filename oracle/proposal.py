"""CPU oracle of the learned lane-position proposal (the network-ranked form of the Alg. 7 search).

TEST INFRASTRUCTURE ONLY.  Like the rest of ``oracle/``, this module exists to check the CUDA library; the
library never imports it.  It is plain numpy, float64 wherever the network's precision rules below do not
fix a narrower type, with loops written the way the definitions read.  It shares no code with the CUDA path.

What it computes.  The exhaustive search of Eq. 24-25 evaluates the energy of the track started at every
bottom-row position; the proposal ranks those starts with a small convolutional network first and
evaluates exact energies only on the best-ranked ones.  The paper does not contain this form; the
configuration that asks for it fixes only its shape (a 4-layer BF16 network with 16-32-32-16 channels and
3x3 kernels, FP32 accumulation, on the 4x-downsampled weighted-gradient map, a per-row heatmap, top-k = 32).
The readings below fill in the rest; each is listed where it is used.

Readings
* N1 input map.  x(i, j) = sum of |G_x w_g| (the Q12 integer map of Eq. 23) over the 4x4 pixel block
  rows 4i..4i+3, columns 4j..4j+3 (clipped at the image edge); the map has ceil(H/4) x ceil(W/4) blocks.
  The network input is bf16(f32(x) * 2^-22).
* N2 network.  Four 3x3 convolutions, zero padding 1, stride 1, channels 1-16-32-32-16, each with bias and
  ReLU; then a 1x1 projection 16 -> 1 with bias gives the logit z(i, j).  The heatmap is sigmoid(z): the
  probability that a lane crosses block (i, j); row i of it is the per-row lane-position heatmap.
* N3 precision.  Weights enter each product rounded to bf16 (round to nearest even); activations are
  stored as bf16(relu(s)) with s accumulated in float (FP32 on the device, float64 rounded to float32
  here); biases are float32; logits float32.  Gradients entering a contraction (dS below) are rounded to
  bf16 the same way; weight gradients are float32 sums.
* N4 labels.  y(i, j) = 1 when the Eq. 25 track of a lane the plain method selected crosses block (i, j)
  on a road row (v_top <= v <= H-1, the column floor(u + 0.5) inside the image), else 0.
* N5 loss.  Mean over all blocks of pw * y * softplus(-z) + (1 - y) * softplus(z) with pw = 10 (lane
  blocks are about one in a hundred).  Optimiser: Adam (Kingma & Ba, Algorithm 1).
* N6 ranking.  Coarse start c covers the fine starts 4c..4c+3.  Its score sums the heatmap p =
  sigmoid(z) along the Eq. 25 track taken in steps of four rows: u starts at (4c - S0) + 1.5 on row H-1,
  each step adds p at block (v >> 2, floor(u + 0.5) >> 2) when that column is inside the image, then
  moves to row v - 4 with u += 4 (V_px(v) - u) / (v - V_py(v)) (the line toward the vanishing point, as in
  Eq. 25), until v < v_top.  Float32, one fixed expression order, no fused multiply-add.  The heatmap, not
  the logit, is summed: cells off the image add nothing, as they add nothing to an energy, and a sum of
  logits (negative almost everywhere) would rank tracks that leave the image early above lanes.
* N7 proposal.  The k best coarse starts (ties: smaller index first) give the candidate fine starts; each
  candidate and its two neighbours get exact Eq. 24 energies.  Local minima are tested only at candidates
  (both neighbours are then exact); the threshold, the ordering and the suppression are those of Alg. 7
  with the minimum taken over the evaluated starts.  When this selects no lane the frame falls back to
  the exhaustive search (and is flagged).
* N8 agreement.  2 |P & L| / (|P| + |L|) over the exact start positions (1 when both are empty).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 16, 32, 32, 16)      # N2
POS_WEIGHT = 10.0                   # N5
INPUT_SCALE_EXP = 22                # N1
F_FALLBACK = 64                     # N7: frame fell back to the exhaustive search


# ---------------------------------------------------------------------------------------------------
# parameter layout: per conv layer W [Cout][Cin][3][3] then b [Cout]; then the head w [16], b [1]
# ---------------------------------------------------------------------------------------------------
def param_shapes():
    shapes = []
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        shapes.append((f"W{l + 1}", (co, ci, 3, 3)))
        shapes.append((f"b{l + 1}", (co,)))
    shapes.append(("wh", (CHANNELS[4],)))
    shapes.append(("bh", (1,)))
    return shapes


def param_count() -> int:
    return int(sum(np.prod(s) for _, s in param_shapes()))


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in param_shapes():
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in param_shapes()])


# ---------------------------------------------------------------------------------------------------
# number formats
# ---------------------------------------------------------------------------------------------------
def f32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def bf16(x):
    """Round to bfloat16 (8 significand bits, round to nearest, ties to even), via float32; returns float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------------------------------
# N1 input map
# ---------------------------------------------------------------------------------------------------
def map_shape(H: int, W: int):
    return (H + 3) // 4, (W + 3) // 4


def xmap_sums(Gw: np.ndarray) -> np.ndarray:
    """Sum of |G_x w_g| over each 4x4 block (int64), block (i, j) = rows 4i.., columns 4j.."""
    H, W = Gw.shape
    h, w = map_shape(H, W)
    out = np.zeros((h, w), np.int64)
    a = np.abs(Gw.astype(np.int64))
    for i in range(h):
        for j in range(w):
            out[i, j] = a[4 * i:4 * i + 4, 4 * j:4 * j + 4].sum()
    return out


def xmap_input(sums: np.ndarray) -> np.ndarray:
    """bf16(f32(x) * 2^-22): the conversion to float32 rounds to nearest even, the scaling is exact."""
    return bf16(f32(sums.astype(np.float64)) * 2.0 ** -INPUT_SCALE_EXP)


# ---------------------------------------------------------------------------------------------------
# N2/N3 network
# ---------------------------------------------------------------------------------------------------
def conv3x3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """s[co, i, j] = sum_{ci, a, b} w[co, ci, a, b] x[ci, i + a - 1, j + b - 1], zero outside the map."""
    C, h, wd = x.shape
    xp = np.zeros((C, h + 2, wd + 2))
    xp[:, 1:h + 1, 1:wd + 1] = x
    out = np.zeros((w.shape[0], h, wd))
    for a in range(3):
        for b in range(3):
            patch = xp[:, a:a + h, b:b + wd]                      # [ci, h, w]
            out += np.einsum("oc,chw->ohw", w[:, :, a, b], patch)
    return out


def conv3x3_transpose(d: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in its input: g[ci, p] = sum_{co, a, b} w[co, ci, a, b] d[co, p - (a - 1, b - 1)]."""
    Co, h, wd = d.shape
    dp = np.zeros((Co, h + 2, wd + 2))
    dp[:, 1:h + 1, 1:wd + 1] = d
    out = np.zeros((w.shape[1], h, wd))
    for a in range(3):
        for b in range(3):
            patch = dp[:, 2 - a:2 - a + h, 2 - b:2 - b + wd]      # d at p - (a - 1, b - 1)
            out += np.einsum("oc,ohw->chw", w[:, :, a, b], patch)
    return out


def conv3x3_wgrad(d: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dW[co, ci, a, b] = sum_p d[co, p] x[ci, p + (a - 1, b - 1)]."""
    C, h, wd = x.shape
    xp = np.zeros((C, h + 2, wd + 2))
    xp[:, 1:h + 1, 1:wd + 1] = x
    out = np.zeros((d.shape[0], C, 3, 3))
    for a in range(3):
        for b in range(3):
            out[:, :, a, b] = np.einsum("ohw,chw->oc", d, xp[:, a:a + h, b:b + wd])
    return out


def _rnd(exact: bool):
    return (lambda t: t) if exact else bf16


def _acc(exact: bool):
    return (lambda t: t) if exact else f32


def forward(params: dict, X: np.ndarray, exact: bool = False) -> dict:
    """One frame: X [h][w] (already bf16 values).  Returns the activations A0..A4 ([C][h][w]) and z [h][w].

    exact=True drops every rounding (float64 throughout) and serves the finite-difference check."""
    q, acc = _rnd(exact), _acc(exact)
    A = [np.asarray(X, np.float64)[None]]
    for l in range(4):
        s = conv3x3(A[-1], q(params[f"W{l + 1}"])) + acc(params[f"b{l + 1}"])[:, None, None]
        A.append(q(acc(np.maximum(s, 0.0))))
    z = acc(np.einsum("c,chw->hw", q(params["wh"]), A[4]) + acc(params["bh"])[0])
    return {"A": A, "z": z}


def softplus(t):
    return np.logaddexp(0.0, t)


def sigmoid(t):
    return 0.5 * (1.0 + np.tanh(0.5 * t))


def loss_and_grad(params: dict, X: np.ndarray, Y: np.ndarray, exact: bool = False, pw: float = POS_WEIGHT):
    """Loss (N5) over a batch X [n][h][w], Y [n][h][w] and its gradient with respect to every parameter.

    Backward pass (N3 rounding points): dz = ((1 - y) sigmoid(z) - pw y sigmoid(-z)) / N;
    dA4 = w_h dz; dS_l = bf16(dA_l * [A_l > 0]); dW_l = sum_p dS_l (x) A_{l-1} (shifted), db_l = sum_p dS_l;
    dA_{l-1} = conv3x3_transpose(dS_l, bf16(W_l))."""
    q, acc = _rnd(exact), _acc(exact)
    n = X.shape[0]
    N = float(np.prod(X.shape))
    grads = {name: np.zeros(shape) for name, shape in param_shapes()}
    loss = 0.0
    for f in range(n):
        fw = forward(params, X[f], exact)
        A, z = fw["A"], fw["z"]
        y = Y[f].astype(np.float64)
        loss += float(np.sum(pw * y * softplus(-z) + (1.0 - y) * softplus(z)))
        dz = acc(((1.0 - y) * sigmoid(z) - pw * y * sigmoid(-z)) / N)
        grads["bh"][0] += dz.sum()
        grads["wh"] += np.einsum("hw,chw->c", dz, A[4])
        dA = q(params["wh"])[:, None, None] * dz[None]
        for l in range(4, 0, -1):
            dS = q(dA * (A[l] > 0))
            grads[f"W{l}"] += conv3x3_wgrad(dS, A[l - 1])
            grads[f"b{l}"] += dS.sum(axis=(1, 2))
            if l > 1:
                dA = conv3x3_transpose(dS, q(params[f"W{l}"]))
    return loss / N, grads


def adam(theta, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """Kingma & Ba, Algorithm 1 (bias-corrected moments), one step t >= 1; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------------------------------------------
# N4 labels and N6/N7 proposal (float32 track arithmetic, fixed order)
# ---------------------------------------------------------------------------------------------------
def _f(x):
    return np.float32(x)


def lane_labels(starts, Vpx, Vpy, v_top: int, H: int, W: int) -> np.ndarray:
    """N4: blocks crossed by the Eq. 25 tracks of the given bottom-row starts (u at v = H-1)."""
    h, w = map_shape(H, W)
    Y = np.zeros((h, w), np.uint8)
    for s in starts:
        u = _f(s)
        for v in range(H - 1, v_top - 1, -1):
            if v < H - 1:
                vx, vy = _f(Vpx[v + 1]), _f(Vpy[v + 1])
                num = _f(_f(vx + _f(_f(v) * u)) - _f(vy * u))
                den = _f(_f(v + 1) - vy)
                u = _f(num / den)
            col = np.floor(_f(u + _f(0.5)))
            if 0.0 <= col < W:
                Y[v >> 2, int(col) >> 2] = 1
    return Y


def heatmap(z: np.ndarray) -> np.ndarray:
    """N2/N6: the per-cell lane probability sigmoid(z) (float64)."""
    return sigmoid(np.asarray(z, np.float64))


def coarse_scores(hm: np.ndarray, Vpx, Vpy, v_top: int, H: int, W: int, S0: int, n_starts: int) -> np.ndarray:
    """N6: score of every coarse start c in [0, ceil(n_starts / 4)) from the float32 heatmap hm [h][w]."""
    nc = (n_starts + 3) // 4
    out = np.zeros(nc, np.float32)
    zz = np.asarray(hm, np.float32)
    for c in range(nc):
        u = _f(_f(4 * c - S0) + _f(1.5))
        acc = _f(0.0)
        v = H - 1
        while v >= v_top:
            col = np.floor(_f(u + _f(0.5)))
            if 0.0 <= col < W:
                acc = _f(acc + zz[v >> 2, int(col) >> 2])
            step = _f(_f(_f(4.0) * _f(_f(Vpx[v]) - u)) / _f(_f(v) - _f(Vpy[v])))
            u = _f(u + step)
            v -= 4
        out[c] = acc
    return out


def top_k(scores: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k largest scores, ties to the smaller index, in ranking order."""
    order = sorted(range(len(scores)), key=lambda c: (-float(scores[c]), c))
    return np.asarray(order[:k], np.int64)


def candidate_sets(top: np.ndarray, n_starts: int):
    """(candidates, evaluated): fine starts of the chosen coarse starts, and those plus their neighbours."""
    cand = np.zeros(n_starts, bool)
    for c in top:
        for r in range(4):
            if 4 * c + r < n_starts:
                cand[4 * c + r] = True
    ev = cand.copy()
    ev[1:] |= cand[:-1]
    ev[:-1] |= cand[1:]
    return cand, ev


def select_on_set(he: np.ndarray, cand: np.ndarray, ev: np.ndarray, S0: int, thr_num: int, thr_den: int,
                  near_px: int, max_lanes: int, thr_abs: int = 0):
    """N7: Alg. 7 selection restricted to the evaluated starts (thr_abs < 0: absolute threshold).
    Returns (start positions, energies)."""
    ns = len(he)
    idx = np.nonzero(ev)[0]
    if ns < 3 or len(idx) == 0:
        return [], []
    mn = int(min(int(he[i]) for i in idx))
    if mn >= 0:
        return [], []
    t = thr_abs if thr_abs != 0 else -(((-mn) * thr_num) // thr_den)
    minima = [i for i in range(1, ns - 1)
              if cand[i] and he[i] < he[i - 1] and he[i] < he[i + 1] and he[i] < t]
    minima.sort(key=lambda i: (int(he[i]), i))
    acc = []
    for i in minima:
        if len(acc) >= max_lanes:
            break
        if all(abs(i - a) > near_px for a in acc):
            acc.append(i)
    acc.sort()
    return [i - S0 for i in acc], [int(he[i]) for i in acc]


def agreement(P, L) -> float:
    """N8: 2 |P & L| / (|P| + |L|) over exact start positions; 1 when both are empty."""
    P, L = set(P), set(L)
    if not P and not L:
        return 1.0
    return 2.0 * len(P & L) / (len(P) + len(L))
