"""GPU parity: the CUDA library against the oracle, element by element, on seeded synthetic frames.

Integer, index and set outputs (histograms, DP paths, inlier sets, edges, Sobel values, votes, m_x, the
bilateral output, M_1, energies, lanes) must be identical; fitted road and V_px parameters agree within
1e-4 relative.  Handles that record m_x and I^bf (ld_debug_capture) have them compared too; the 64-frame
workload runs without that capture, exactly as the benchmark launches it.
"""
import numpy as np
import pytest

from paper_1807_02752_gb300 import ld, scenes
from gpu_util import compare_frame, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build
    build.build()
    return torch


def _captured(W, H, n, p):
    det = ld.Detector(W, H, n, p)
    det.capture(True)
    return det


def _run(torch, det, disp, img):
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    out = det.detect(d, i)
    torch.cuda.synchronize()
    return det.lanes(out)


@pytest.mark.parametrize("name,n", [("small_320x120", 6), ("single_1242x375", 2)])
def test_every_stage_matches_oracle(torch_cuda, name, n):
    cfg, _ = scenes.WORKLOADS[name]
    disp, img, _ = scenes.make_batch(cfg, n)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = _captured(cfg.width, cfg.height, n, p)
    res = _run(torch_cuda, det, disp, img)
    for f in range(n):
        compare_frame(det, res[f], f, disp[f], img[f], p)


def test_batch64_sampled_frames_match_oracle(torch_cuda):
    """The 64-frame 1242x375 workload, launched as the benchmark launches it; sampled frames checked fully."""
    cfg, n = scenes.WORKLOADS["batch64_1242x375"]
    disp, img, _ = scenes.make_batch(cfg, n)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, n, p)
    res = _run(torch_cuda, det, disp, img)
    for f in (0, 17, 38, 63):
        compare_frame(det, res[f], f, disp[f], img[f], p)
    # every frame's lanes, without stage dumps
    for f in range(n):
        if f not in (0, 17, 38, 63) and f % 4 == 1:
            compare_frame(det, res[f], f, disp[f], img[f], p, stages=False)


def test_hd_frames_match_oracle(torch_cuda):
    cfg, _ = scenes.WORKLOADS["batch16_1920x1080"]
    disp, img, _ = scenes.make_batch(cfg, 2)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = _captured(cfg.width, cfg.height, 2, p)
    res = _run(torch_cuda, det, disp, img)
    for f in range(2):
        compare_frame(det, res[f], f, disp[f], img[f], p)


def test_ragged_and_tiny_sizes(torch_cuda):
    for (W, H, D) in [(333, 97, 40), (16, 16, 8), (1241, 376, 128), (17, 300, 32)]:
        cfg = scenes.with_size(scenes.SMALL_320x120, width=W, height=H, n_disp=D, obstacles=(0, 1) if W < 64 else (1, 2),
                               stripe_px=(2.0, 4.0) if W < 64 else (3.0, 6.0))
        try:
            disp, img, _ = scenes.make_batch(cfg, 2, first_frame=5)
        except RuntimeError:
            continue
        p = ld.default_params(n_disp=D)
        det = _captured(W + 7, H + 3, 4, p)  # handle larger than the frames
        res = _run(torch_cuda, det, disp, img)
        for f in range(2):
            compare_frame(det, res[f], f, disp[f], img[f], p)


def test_degenerate_frames(torch_cuda):
    """No valid disparity, no road, no edges: flags and results match the oracle, nothing faults."""
    cfg = scenes.SMALL_320x120
    d0, i0, _ = scenes.make_frame(cfg, 1)
    H, W = d0.shape
    frames = []
    frames.append((np.zeros((H, W), np.float32), i0))                          # all invalid
    frames.append((np.full((H, W), np.nan, np.float32), i0))                   # non-finite
    frames.append((d0, np.full((H, W), 120, np.uint8)))                        # no edges at all
    frames.append((np.full((H, W), 7.0, np.float32), i0))                      # constant disparity
    v = np.arange(H, dtype=np.float32)[:, None]
    frames.append(((-0.3 * (v - 40)).repeat(W, 1).astype(np.float32), i0))     # decreasing "road"
    frames.append((d0, i0))                                                    # a normal frame in the mix
    disp = np.stack([f[0] for f in frames])
    img = np.stack([f[1] for f in frames])
    p = ld.default_params(n_disp=cfg.n_disp)
    det = _captured(W, H, len(frames), p)
    res = _run(torch_cuda, det, disp, img)
    for f in range(len(frames)):
        compare_frame(det, res[f], f, disp[f], img[f], p)


def test_param_variants(torch_cuda):
    cfg = scenes.SMALL_320x120
    disp, img, _ = scenes.make_batch(cfg, 3, first_frame=11)
    for kw in ({"bilateral": 0}, {"bf_rho": 3, "sigma_r": 0.2}, {"ransac_hyps": 1}, {"ransac_hyps": 256, "seed": 7},
               {"chi": 5, "tau_x": 7, "lambda_x": 3}, {"thr_den": 4, "near_px": 5, "max_lanes": 2},
               {"ransac_rounds": 1}, {"box_nu": 0, "box_vs": 0}, {"box_nu": 3, "box_vs": 8},
               {"box_nu": 8, "box_vs": 1}, {"bilateral": 2}, {"bilateral": 2, "bf_rho": 2}, {"wg_gaussian": 1},
               {"thr_abs": -(1 << 22)}, {"thr_abs": -(1 << 22), "wg_gaussian": 1, "bilateral": 2},
               {"dp_literal": 1}, {"dp_literal": 1, "tau_y": 3, "lambda_y": 2}, {"band_literal_bottom": 1},
               {"band_literal_bottom": 1, "chi": 5}, {"band_literal_bottom": 1, "chi": 0}):
        p = ld.default_params(n_disp=cfg.n_disp, **kw)
        det = _captured(cfg.width, cfg.height, 3, p)
        res = _run(torch_cuda, det, disp, img)
        for f in range(3):
            compare_frame(det, res[f], f, disp[f], img[f], p)


def test_paper_literal_variants_full_size(torch_cuda):
    """The median pre-filter (ragged 8 x 32 tiles at 1242x375) and the Gaussian w_g at the full size."""
    cfg = scenes.SINGLE_1242x375
    disp, img, _ = scenes.make_batch(cfg, 2, first_frame=61)
    for kw in ({"bilateral": 2}, {"wg_gaussian": 1}, {"band_literal_bottom": 1}):
        p = ld.default_params(n_disp=cfg.n_disp, **kw)
        det = ld.Detector(cfg.width, cfg.height, 2, p)
        res = _run(torch_cuda, det, disp, img)
        for f in range(2):
            compare_frame(det, res[f], f, disp[f], img[f], p)


def test_wide_frames_chunked_m1(torch_cuda):
    """Frames too wide for one shared-memory chunk of the M_1 kernel (the column-chunked layout)."""
    cfg = scenes.with_size(scenes.SMALL_320x120, width=3000, height=96, n_disp=64)
    disp, img, _ = scenes.make_batch(cfg, 2, first_frame=3)
    for kw in ({}, {"box_nu": 2, "box_vs": 8}):
        p = ld.default_params(n_disp=cfg.n_disp, **kw)
        det = ld.Detector(cfg.width, cfg.height, 2, p)
        res = _run(torch_cuda, det, disp, img)
        for f in range(2):
            compare_frame(det, res[f], f, disp[f], img[f], p)


def test_maximum_frame_size(torch_cuda):
    """The largest frame a handle accepts (LD_MAX_W x LD_MAX_H = 4096 x 1088) at the most disparity bins
    (LD_MAX_D = 256): every stage, m_x and I^bf against the oracle."""
    cfg = scenes.with_size(scenes.HD_1920x1080, width=ld.MAX_W, height=ld.MAX_H, n_disp=ld.MAX_D)
    disp, img, _ = scenes.make_batch(cfg, 1, first_frame=11)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = _captured(cfg.width, cfg.height, 1, p)
    res = _run(torch_cuda, det, disp, img)
    compare_frame(det, res[0], 0, disp[0], img[0], p)
    det.close()


def test_graph_replay_and_host_path_agree(torch_cuda):
    torch = torch_cuda
    cfg = scenes.SINGLE_1242x375
    disp, img, _ = scenes.make_batch(cfg, 3, first_frame=20)
    p = ld.default_params()
    det = ld.Detector(cfg.width, cfg.height, 3, p)
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    out = det.alloc_lanes(3)
    first = None
    for _ in range(3):  # capture, then replay the captured graph
        det.detect(d, i, out)
        torch.cuda.synchronize()
        r = det.lanes(out).copy()
        if first is None:
            first = r
        assert r.tobytes() == first.tobytes()
    host = det.detect_host(disp, img)
    assert host.tobytes() == first.tobytes()
    # a frame alone gives the same result as in the batch
    det1 = ld.Detector(cfg.width, cfg.height, 1, p)
    alone = det1.detect_host(disp[1:2], img[1:2])
    assert alone.tobytes() == first[1:2].tobytes()


def test_argument_errors(torch_cuda):
    torch = torch_cuda
    import ctypes
    p = ld.default_params()
    det = ld.Detector(320, 120, 2, p)
    L = det.L
    d = torch.zeros((2, 120, 320), dtype=torch.float32, device="cuda")
    i = torch.zeros((2, 120, 320), dtype=torch.uint8, device="cuda")
    out = det.alloc_lanes(2)
    bad = [(None, i.data_ptr(), 320, 120, 2), (d.data_ptr(), i.data_ptr(), 321, 120, 2),
           (d.data_ptr(), i.data_ptr(), 320, 121, 2), (d.data_ptr(), i.data_ptr(), 320, 120, 3),
           (d.data_ptr(), i.data_ptr(), 15, 120, 1), (d.data_ptr(), i.data_ptr(), 320, 120, 0)]
    for a in bad:
        assert L.ld_detect(det.h, a[0], a[1], a[2], a[3], a[4], out.data_ptr()) == ld.E_ARG
        assert L.ld_last_error(det.h)
    buf = np.zeros(16, np.uint8)
    det2 = ld.Detector(320, 120, 2, p)
    assert L.ld_debug_get(det2.h, 0, ld.STAGE_HE, buf.ctypes.data, 16) == ld.E_STATE
    assert L.ld_detect(det.h, d.data_ptr(), i.data_ptr(), 320, 120, 2, out.data_ptr()) == ld.OK
    torch.cuda.synchronize()
    assert L.ld_debug_get(det.h, 5, ld.STAGE_HE, buf.ctypes.data, 16) == ld.E_ARG
    assert L.ld_debug_get(det.h, 0, 99, buf.ctypes.data, 16) == ld.E_ARG
    assert L.ld_debug_get(det.h, 0, ld.STAGE_HE, buf.ctypes.data, 16) == ld.E_ARG  # wrong size


def test_tuning_keeps_results(torch_cuda):
    """ld_tune only changes launch shapes: lanes and intermediate stages stay identical, before and after
    (the latter through a newly captured graph)."""
    torch = torch_cuda
    cfg, _ = scenes.WORKLOADS["single_1242x375"]
    disp, img, _ = scenes.make_batch(cfg, 3, first_frame=40)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, 3, p)
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    stages = (ld.STAGE_VDISP, ld.STAGE_ROWS, ld.STAGE_M1, ld.STAGE_HE)

    def run():
        out = det.detect(d, i)
        torch.cuda.synchronize()
        res = det.lanes(out).tobytes()
        dumps = [det.debug(f, st, cfg.width, cfg.height) for f in range(3) for st in stages]
        return res, dumps

    before = run()
    chosen = det.tune(d, i)
    assert chosen["vdisp_rows"] in (8, 16, 32) and chosen["grad_rows"] in (8, 12, 16, 24, 32)
    assert chosen["m1_rows"] in (8, 12, 14, 16)
    after = run()
    assert before[0] == after[0]
    for a, b in zip(before[1], after[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("name,n", [("single_1242x375", 2), ("batch64_1242x375", 64), ("batch16_1920x1080", 2)])
def test_lane_tracks_match_oracle(torch_cuda, name, n):
    """Alg. 7's drawing step (ld_lane_tracks): every selected lane's Eq. 25 track, bit-exact against the
    oracle's track on the oracle's V_p rows, NaN above v_top and in empty lane slots."""
    import oracle
    torch = torch_cuda
    cfg, _ = scenes.WORKLOADS[name]
    disp, img, _ = scenes.make_batch(cfg, n)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, n, p)
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    out = det.detect(d, i)
    tr = det.lane_tracks(out, n, cfg.height)
    torch.cuda.synchronize()
    tr = tr.cpu().numpy()
    for f in ((0, 1) if n <= 2 else (0, 9, 40, 63)):
        ref = oracle.detect(disp[f], img[f], oracle_params(p))
        for k in range(ld.MAX_LANES):
            if k < ref["n_lanes"]:
                want = oracle.track(ref["Vpx"], ref["Vpy"], ref["v_top"], ref["start_u"][k])
                assert np.array_equal(tr[f, k], want, equal_nan=True), f"frame {f} lane {k}"
            else:
                assert np.isnan(tr[f, k]).all()
    with pytest.raises(ld.LDError) as e:
        det.lane_tracks(out, n + 1, cfg.height)
    assert e.value.code == ld.E_ARG
    det.close()
