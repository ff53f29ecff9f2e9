"""Seeded synthetic stereo lane scenes with closed-form ground truth.

This module produces the inputs of the lane-detection path: a float32 disparity map and a uint8 left
image per frame, shaped like the KITTI raw frames the paper evaluates on (Sec. 3.2, 1242x375).  KITTI is
not available here, so every frame is synthetic and seeded.  The module holds none of the detector's
arithmetic; both the CUDA path and the CPU oracle consume what it renders.

Geometry (closed form, consistent with Eq. 14 and Eq. 25):

* road profile on the v-disparity map: d = f(v) = a (v - v_h)^2 + b (v - v_h), i.e. the parabola
  f(v) = beta0 + beta1 v + beta2 v^2 of Sec. 2.2, zero at the horizon row v_h;
* V_py(v) = v - f(v) / f'(v) (Eq. 14);
* lanes u_i(v) = A(v) + s_i f(v) with A(v) = alpha0 + alpha1 f + alpha2 f^2.  Every such curve is a
  field line of du/dv = (u - V_px(v)) / (v - V_py(v)), the relation Eq. 25 steps along, with
  V_px(v) = alpha0 - alpha2 f(v)^2, a quartic in v like the model of Eq. 19.

Lane spacing is 6.5 pixels per unit of road disparity (3.5 m lanes at a 0.54 m baseline).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1807027520


@dataclass(frozen=True)
class SceneConfig:
    """Shape and content recipe of one family of synthetic frames."""

    width: int = 1242
    height: int = 375
    n_disp: int = 128                 # disparity bins D of the v-disparity map
    lanes: tuple = (3, 3)             # inclusive range of lane-marking count
    stripe_px: tuple = (8.0, 15.0)    # marking width at the bottom row
    outlier_frac: float = 0.05        # pixels given a random disparity U(0, D-1)
    invalid_frac: float = 0.0         # pixels set to 0 (invalid after the LR check)
    max_curvature: float = 1.0 / 150  # image-plane curvature limit of a marking, 1/px
    dashed: bool = False
    shadow_frac: float = 0.0          # fraction of road rows darkened by shadow bands
    obstacles: tuple = (2, 4)
    b_range: tuple = (0.28, 0.38)     # road disparity slope per row near the horizon


# Named workloads.  The first is the single-frame case the oracle finishes in seconds, the second the
# 64-frame throughput workload, the third the high-resolution stress case.
SINGLE_1242x375 = SceneConfig()
BATCH64_1242x375 = SceneConfig(outlier_frac=0.10, invalid_frac=0.10)
HD_1920x1080 = SceneConfig(width=1920, height=1080, n_disp=256, lanes=(3, 6), stripe_px=(12.0, 22.0),
                           outlier_frac=0.30, max_curvature=1.0 / 80, dashed=True, shadow_frac=0.30,
                           b_range=(0.18, 0.24))
# Small frames for fast CPU tests of the oracle; same recipe, scaled.
SMALL_320x120 = SceneConfig(width=320, height=120, n_disp=48, lanes=(2, 3), stripe_px=(3.0, 6.0),
                            obstacles=(1, 2), b_range=(0.28, 0.38))

WORKLOADS = {
    "single_1242x375": (SINGLE_1242x375, 1),
    "batch64_1242x375": (BATCH64_1242x375, 64),
    "batch16_1920x1080": (HD_1920x1080, 16),
    "small_320x120": (SMALL_320x120, 4),
}


@dataclass
class Truth:
    """Planted parameters of one frame."""

    beta: np.ndarray                  # f(v) = beta0 + beta1 v + beta2 v^2 (float64)
    v_horizon: float
    vpy: np.ndarray                   # [H] float64, NaN above the horizon
    vpx: np.ndarray                   # [H] float64, NaN above the horizon
    lane_starts: np.ndarray           # u_i(v_max) of each planted marking (float64)
    lane_widths: np.ndarray           # marking width at v_max (px)
    lane_visible_rows: np.ndarray     # rows of each marking that are inside the image and unoccluded
    alpha: np.ndarray = field(default_factory=lambda: np.zeros(3))


def _rng(seed: int, frame: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([seed & 0xFFFFFFFF, frame, purpose]))


def _road(cfg: SceneConfig, r: np.random.Generator):
    H, D = cfg.height, cfg.n_disp
    vmax = H - 1
    a_max = 2e-4 * (375.0 / H) ** 1.3
    v = np.arange(H, dtype=np.float64)
    for _ in range(1000):
        vh = r.uniform(0.267 * H, 0.427 * H)
        b = r.uniform(*cfg.b_range)
        a = r.uniform(-a_max, a_max)
        road = v > vh
        fprime = 2.0 * a * (v[road] - vh) + b
        dmax = a * (vmax - vh) ** 2 + b * (vmax - vh)
        if fprime.min() >= 1.0 / 6.0 and dmax < D - 8:
            beta = np.array([a * vh * vh - b * vh, b - 2.0 * a * vh, a])
            return vh, a, b, beta
    raise RuntimeError("road sampling failed")


def _lanes(cfg: SceneConfig, r: np.random.Generator, f: np.ndarray, fp: np.ndarray, road_rows: np.ndarray):
    W, H = cfg.width, cfg.height
    vmax = H - 1
    fm = f[vmax]
    n = int(r.integers(cfg.lanes[0], cfg.lanes[1] + 1))
    fr = f[road_rows]
    fpr = fp[road_rows]
    fpp = np.gradient(fp)[road_rows]
    for _ in range(1000):
        a0 = W / 2 + r.uniform(-150, 150) * (W / 1242.0)
        a1 = r.uniform(-1.0, 1.0)
        a2 = r.uniform(-1.0, 1.0) * 0.25 * W / (fm * fm)
        s0 = (W / 2 - a0 - a2 * fm * fm) / fm - a1 - 3.25 * (n - 1)
        s = s0 + 6.5 * np.arange(n)
        vpx = a0 - a2 * fr * fr
        if vpx.min() < 20 or vpx.max() > W - 20:
            continue
        ok = True
        for si in s:
            k1 = a1 + si
            du = (k1 + 2 * a2 * fr) * fpr                       # du/dv
            d2u = (k1 + 2 * a2 * fr) * fpp + 2 * a2 * fpr * fpr  # d2u/dv2
            curv = np.abs(d2u) / (1.0 + du * du) ** 1.5
            u = a0 + k1 * fr + a2 * fr * fr
            vis = (u >= 0) & (u < W)
            if vis.any() and curv[vis].max() > cfg.max_curvature:
                ok = False
                break
        if ok:
            return np.array([a0, a1, a2]), s
    raise RuntimeError("lane sampling failed")


def make_frame(cfg: SceneConfig, frame: int, seed: int = BASE_SEED, with_clean: bool = False):
    """Render one frame.  Returns (disparity f32 [H,W], image u8 [H,W], Truth), and with with_clean also the
    disparity before the outlier and invalid pixels (the scene's own disparity)."""
    W, H, D = cfg.width, cfg.height, cfg.n_disp
    vmax = H - 1
    r_geo = _rng(seed, frame, 1)
    r_pix = _rng(seed, frame, 2)

    vh, a, b, beta = _road(cfg, r_geo)
    v = np.arange(H, dtype=np.float64)
    f = beta[0] + beta[1] * v + beta[2] * v * v
    fp = beta[1] + 2.0 * beta[2] * v
    road_rows = v > vh
    with np.errstate(divide="ignore", invalid="ignore"):
        vpy = np.where(road_rows, v - f / fp, np.nan)

    alpha, s = _lanes(cfg, r_geo, f, fp, road_rows)
    vpx = np.where(road_rows, alpha[0] - alpha[2] * f * f, np.nan)

    # ---- disparity -------------------------------------------------------------------------------
    disp = np.empty((H, W), dtype=np.float32)
    sky = ~road_rows
    n_sky = int(sky.sum())
    sky_d = r_pix.uniform(0.5, 3.0, size=(n_sky, W)).astype(np.float32)
    sky_d[r_pix.random((n_sky, W)) < 0.5] = 0.0
    disp[sky] = sky_d
    disp[road_rows] = f[road_rows].astype(np.float32)[:, None]

    # ---- image -----------------------------------------------------------------------------------
    img = np.empty((H, W), dtype=np.float64)
    img[sky] = r_geo.uniform(140, 190)
    img[road_rows] = r_geo.uniform(90, 120)

    if cfg.shadow_frac > 0:
        rows = np.nonzero(road_rows)[0]
        target = int(cfg.shadow_frac * rows.size)
        shade = np.zeros(H, dtype=bool)
        while shade[rows].sum() < target:
            h = int(r_geo.integers(5, 40))
            v0 = int(r_geo.integers(rows[0], rows[-1]))
            shade[v0:v0 + h] = True
        shade &= road_rows
        img[shade] *= r_geo.uniform(0.5, 0.7)

    uu = np.arange(W, dtype=np.float64)[None, :]
    fm = f[vmax]
    widths = r_geo.uniform(*cfg.stripe_px, size=len(s))
    lane_mask = np.zeros((H, W), dtype=bool)
    lane_rows_vis = []
    phase = r_geo.uniform(0, 1)
    sub = (np.arange(4) + 0.5) / 4.0 - 0.5          # 4 sub-rows per pixel row (vertical anti-aliasing)
    vs = v[:, None] + sub[None, :]                   # [H, 4]
    fs = beta[0] + beta[1] * vs + beta[2] * vs * vs
    fs = np.where(vs > vh, fs, np.nan)
    for i, si in enumerate(s):
        u_c = alpha[0] + (alpha[1] + si) * fs + alpha[2] * fs * fs              # [H, 4]
        half = np.maximum(1.0, widths[i] * fs / fm) / 2.0
        # exact horizontal overlap of pixel [u-0.5, u+0.5] with the stripe, averaged over sub-rows
        lo = np.maximum(uu[:, :, None] - 0.5, (u_c - half)[:, None, :])
        hi = np.minimum(uu[:, :, None] + 0.5, (u_c + half)[:, None, :])
        cov = np.nan_to_num(np.clip(hi - lo, 0.0, 1.0)).mean(axis=2)           # [H, W]
        if cfg.dashed:
            with np.errstate(divide="ignore", invalid="ignore"):
                on = np.mod(65.0 / f + phase, 1.0) < 0.5
            cov *= np.where(road_rows, on, False)[:, None]
        cov *= road_rows[:, None]
        lum = r_geo.uniform(200, 240)
        if cfg.shadow_frac > 0:
            lum_row = np.where(shade, lum * 0.6, lum)[:, None]
        else:
            lum_row = lum
        img = img + cov * (lum_row - img)
        m = cov > 0.5
        lane_mask |= m
        lane_rows_vis.append(m)

    # ---- obstacles (occlude road and lanes) ------------------------------------------------------
    n_obs = int(r_geo.integers(cfg.obstacles[0], cfg.obstacles[1] + 1))
    v_lo = int(np.ceil(vh)) + 20
    v_hi = vmax - 40
    occl = np.zeros((H, W), dtype=bool)
    for _ in range(n_obs):
        if v_hi <= v_lo:
            break
        vb = int(r_geo.integers(v_lo, v_hi + 1))
        hgt = int(r_geo.integers(40, 151) * H / 375.0)
        wid = int(r_geo.uniform(60, 250) * (W / 1242.0) * f[vb] / fm + 20)
        wid = min(wid, W - 1)
        u0 = int(r_geo.integers(0, W - wid + 1))
        v0 = max(0, vb - hgt + 1)
        disp[v0:vb + 1, u0:u0 + wid] = np.float32(f[vb])
        img[v0:vb + 1, u0:u0 + wid] = r_pix.uniform(30, 220, size=(vb + 1 - v0, wid))
        occl[v0:vb + 1, u0:u0 + wid] = True

    clean = disp.copy() if with_clean else None
    # ---- outliers and invalid pixels -------------------------------------------------------------
    if cfg.outlier_frac > 0:
        m = r_pix.random((H, W)) < cfg.outlier_frac
        disp[m] = r_pix.uniform(0.0, D - 1, size=int(m.sum())).astype(np.float32)
    if cfg.invalid_frac > 0:
        m = r_pix.random((H, W)) < cfg.invalid_frac
        disp[m] = 0.0

    img += r_pix.normal(0.0, 6.0, size=(H, W))
    img = np.clip(np.rint(img), 0, 255).astype(np.uint8)

    starts = alpha[0] + (alpha[1] + s) * fm + alpha[2] * fm * fm
    vis_rows = np.array([(m & ~occl).any(axis=1).sum() for m in lane_rows_vis])
    truth = Truth(beta=beta, v_horizon=vh, vpy=vpy, vpx=vpx, lane_starts=starts, lane_widths=widths,
                  lane_visible_rows=vis_rows, alpha=alpha)
    if with_clean:
        return disp, img, truth, clean
    return disp, img, truth


def make_stereo_frame(cfg: SceneConfig, frame: int, seed: int = BASE_SEED):
    """A rectified stereo pair of one frame: (left u8 [H,W], right u8 [H,W], clean disparity f32 [H,W], Truth).

    The left image is make_frame's image.  The right image sees the scene shifted by its disparity: the left
    pixel (u, v) lands on column round(u - d(u, v)), the nearest surface (largest d) winning where several
    land; columns nothing lands on (occlusions) take the nearest landed value to their right (the farther
    surface); then independent Gaussian noise of sigma 2 and rounding."""
    _, left, truth, clean = make_frame(cfg, frame, seed, with_clean=True)
    H, W = left.shape
    r = _rng(seed, frame, 3)
    right = np.zeros((H, W), dtype=np.float64)
    cols = np.arange(W)
    for v in range(H):
        order = np.argsort(clean[v], kind="stable")            # far first: the nearest surface lands last
        x = np.rint(cols[order] - clean[v][order].astype(np.float64)).astype(np.int64)
        ok = (x >= 0) & (x < W)
        row = np.full(W, -1.0)
        row[x[ok]] = left[v][order[ok]]
        filled = row >= 0
        if not filled.any():
            row[:] = left[v]
        else:
            # nearest landed value to the right (then to the left at the right edge)
            idx = np.where(filled, cols, W)
            nxt = np.minimum.accumulate(idx[::-1])[::-1]
            prv = np.maximum.accumulate(np.where(filled, cols, -1))
            take = np.where(nxt < W, nxt, prv)
            row = row[take]
        right[v] = row
    right += r.normal(0.0, 2.0, size=(H, W))
    right = np.clip(np.rint(right), 0, 255).astype(np.uint8)
    return left, right, clean, truth


def make_batch(cfg: SceneConfig, n_frames: int, seed: int = BASE_SEED, first_frame: int = 0):
    """Render n_frames frames with per-frame seeds.  Returns (disp [n,H,W] f32, img [n,H,W] u8, truths)."""
    disp = np.empty((n_frames, cfg.height, cfg.width), dtype=np.float32)
    img = np.empty((n_frames, cfg.height, cfg.width), dtype=np.uint8)
    truths = []
    for i in range(n_frames):
        d, im, t = make_frame(cfg, first_frame + i, seed)
        disp[i] = d
        img[i] = im
        truths.append(t)
    return disp, img, truths


def with_size(cfg: SceneConfig, **kw) -> SceneConfig:
    return dataclasses.replace(cfg, **kw)


def make_tiny_frame(w: int, h: int, n_disp: int, seed: int):
    """A small adversarial frame (seeded) for the smallest shapes the library accepts (16 x 16 and up), where
    the road scenes above do not fit: a disparity ramp from a random horizon row down to about n_disp - 1.5
    at the bottom row, with noise; one box of constant disparity; about 3 % NaN, 2 % +inf, 3 % zero, 2 %
    negative and 2 % at or above n_disp.  The image is grey noise with one to three bright stripes of random
    slope below the horizon.  Returns (disparity float32 [h][w], image uint8 [h][w])."""
    rng = np.random.default_rng(seed)
    v = np.arange(h, dtype=np.float64)[:, None] * np.ones((1, w))
    vh = int(rng.integers(h // 4, h // 2 + 1))
    disp = np.clip((v - vh) * (n_disp - 1.5) / max(1, h - 1 - vh), 0, None) + rng.normal(0, 0.3, (h, w))
    bw, bh = max(2, w // 5), max(2, h // 5)
    bx, by = int(rng.integers(0, w - bw)), int(rng.integers(0, h - bh))
    disp[by:by + bh, bx:bx + bw] = rng.uniform(1, n_disp - 1)
    r = rng.random((h, w))
    disp[r < 0.03] = np.nan
    disp[(r >= 0.03) & (r < 0.05)] = np.inf
    disp[(r >= 0.05) & (r < 0.08)] = 0.0
    disp[(r >= 0.08) & (r < 0.10)] = -rng.uniform(0, 5)
    disp[(r >= 0.10) & (r < 0.12)] = n_disp + rng.uniform(0, 40)
    img = 70 + rng.normal(0, 6, (h, w))
    for _ in range(int(rng.integers(1, 4))):
        c0, slope = rng.uniform(0, w), rng.uniform(-1.5, 1.5)
        for vv in range(vh, h):
            c = int(round(c0 + slope * (vv - vh)))
            img[vv, max(0, c - 1):max(0, c + 2)] = 200 + rng.normal(0, 10)
    return disp.astype(np.float32), np.clip(img, 0, 255).astype(np.uint8)
