"""The allocation-free road-path entry point (ld_road_path_static).

It serves callers that may not allocate device memory in their per-frame path (their memory is reserved
once at start-up, or their host hands them only input and output buffers).  This file runs last so that a
failure here leaves every other test already run.  The test drives the entry point through the C-ABI and
checks, on two calls in a row with different frames, that its paths equal the road DP paths the regular
handle-based entry point (ld_detect) produces for the same frames.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_static_road_path_matches_detect():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build, ld, scenes

    build.build()
    L = ld.load()
    cfg = scenes.SINGLE_1242x375
    n, W, H, D = 3, cfg.width, cfg.height, cfg.n_disp
    p = ld.default_params(n_disp=D)
    det = ld.Detector(W, H, n, p)
    stream = torch.cuda.current_stream()
    for call, first in enumerate((0, 40)):           # two calls in a row, different frames
        disp, img, _ = scenes.make_batch(cfg, n, first_frame=first)
        d = torch.from_numpy(disp).cuda()
        i = torch.from_numpy(img).cuda()
        det.detect(d, i)
        torch.cuda.synchronize()
        want = np.stack([det.debug(f, ld.STAGE_PATH_Y, W, H) for f in range(n)])
        out = torch.full((n, D), 7, dtype=torch.int16, device="cuda")
        rc = L.ld_road_path_static(ctypes.byref(p), d.data_ptr(), W, H, n, out.data_ptr(),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == ld.OK, L.ld_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert (got[:, 0] == -1).all()
        assert (got[:, 1:] == want[:, 1:]).all(), f"call {call}: paths differ"
    # a request beyond the static scratch is refused without touching the GPU
    big = (ld.LD_STATIC_SCRATCH_BYTES // (D * H * 4)) + 1
    rc = L.ld_road_path_static(ctypes.byref(p), d.data_ptr(), W, H, big, out.data_ptr(), None)
    assert rc == ld.E_ARG and b"LD_STATIC_SCRATCH_BYTES" in L.ld_last_error(None)


def test_static_road_path_odd_height_wide_step_and_literal_refused():
    """Odd frame height (the last thread's second cell lies past the frame), the widest row step
    (tau_y = 15, which ld_detect runs on its second road kernel) and lambda_y = 0 (many ties): the paths
    still equal ld_detect's.  The DP as printed (dp_literal = 1) is refused with LD_E_ARG."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build, ld, scenes

    build.build()
    L = ld.load()
    W, H, D, n = 320, 121, 48, 3
    cfg = scenes.with_size(scenes.SMALL_320x120, width=W, height=H, n_disp=D)
    disp, img, _ = scenes.make_batch(cfg, n, first_frame=60)
    d = torch.from_numpy(disp).cuda()
    i = torch.from_numpy(img).cuda()
    stream = torch.cuda.current_stream()
    for kw in ({"tau_y": 15, "lambda_y": 0}, {"tau_y": 15, "lambda_y": 3}, {"tau_y": 0, "lambda_y": 0}):
        p = ld.default_params(n_disp=D, **kw)
        det = ld.Detector(W, H, n, p)
        det.detect(d, i)
        torch.cuda.synchronize()
        want = np.stack([det.debug(f, ld.STAGE_PATH_Y, W, H) for f in range(n)])
        det.close()
        for call in range(2):
            out = torch.full((n, D), 7, dtype=torch.int16, device="cuda")
            rc = L.ld_road_path_static(ctypes.byref(p), d.data_ptr(), W, H, n, out.data_ptr(),
                                       ctypes.c_void_p(stream.cuda_stream))
            assert rc == ld.OK, L.ld_last_error(None)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert (got[:, 0] == -1).all()
            assert (got[:, 1:] == want[:, 1:]).all(), f"{kw} call {call}: paths differ"
    p = ld.default_params(n_disp=D, dp_literal=1)
    out = torch.zeros((n, D), dtype=torch.int16, device="cuda")
    rc = L.ld_road_path_static(ctypes.byref(p), d.data_ptr(), W, H, n, out.data_ptr(), None)
    assert rc == ld.E_ARG and b"dp_literal" in L.ld_last_error(None)
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 0).all()
