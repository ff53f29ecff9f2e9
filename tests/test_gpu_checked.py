"""The bounds-checked build (LD_CHECKED, lib/libld_checked.so).

Its kernels test every data-derived index, every append to a fixed-capacity list and each tile against its
frame before the access, and count a failure instead of trapping (include/ld.h, ld_check_status).  These
tests run the whole path through that library on the smallest shapes it accepts, with adversarial
disparities (NaN, +inf, zero, negative, beyond D), and on the camera sizes.  They require a clean status
and, for every frame, every stage dump equal to the oracle's.  The recorder itself is checked with
ld_check_selftest, which evaluates one failing test and accesses nothing.
"""
import numpy as np
import pytest

from paper_1807_02752_gb300 import ld, scenes
from gpu_util import compare_frame

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build
    build.build(checked=True)
    L = ld.load(checked=True)
    assert L.ld_checked_build() == 1
    return torch, L


def _clean(L):
    st = ld.check_status(L)
    assert st["failures"] == 0, f"bounds-check failures: {st}"


def test_selftest_records_and_resets(checked):
    torch, L = checked
    assert L.ld_check_reset() == ld.OK
    _clean(L)
    assert L.ld_check_selftest() == ld.OK
    assert ld.check_status(L) == {"failures": 1, "site": "selftest", "index": 7, "bound": 7}
    assert L.ld_check_reset() == ld.OK
    _clean(L)
    R = ld.load()                      # the regular library: no checks, a clean status, no self-test
    assert R.ld_checked_build() == 0
    assert ld.check_status(R)["failures"] == 0
    assert R.ld_check_selftest() == ld.E_STATE


def _run(torch, L, frames, p, capture=True):
    disp = np.stack([f[0] for f in frames])
    img = np.stack([f[1] for f in frames])
    n, H, W = disp.shape
    det = ld.Detector(W, H, n, p, lib=L)
    try:
        if capture:
            det.capture(True)
        assert L.ld_check_reset() == ld.OK
        out = det.detect(torch.from_numpy(disp).cuda(), torch.from_numpy(img).cuda())
        torch.cuda.synchronize()
        _clean(L)
        rows = ld.Detector.lanes(out)
        for k in range(n):
            compare_frame(det, rows[k], k, disp[k], img[k], p)
    finally:
        det.close()


@pytest.mark.parametrize("shape", [(16, 16, 4), (17, 16, 4), (24, 18, 8), (70, 33, 16), (130, 50, 24),
                                   (257, 67, 32)])
def test_tiny_shapes(checked, shape):
    torch, L = checked
    w, h, D = shape
    frames = [scenes.make_tiny_frame(w, h, D, 900 + k) for k in range(4)]
    _run(torch, L, frames, ld.default_params(n_disp=D))


@pytest.mark.parametrize("kw", [{"bilateral": 0}, {"bilateral": 2}, {"dp_literal": 1}, {"tau_y": 15},
                                {"tau_x": 7, "chi": 5}, {"lambda_g": 0}])
def test_tiny_shapes_param_variants(checked, kw):
    torch, L = checked
    frames = [scenes.make_tiny_frame(70, 33, 16, 950 + k) for k in range(3)]
    _run(torch, L, frames, ld.default_params(n_disp=16, **kw))


def test_camera_size_and_groups(checked):
    """Four 1242x375 frames at D = 256 through the checked library, then a mixed-size call (one launch per
    stage over three tiny sizes): a clean status, and every frame the oracle's."""
    torch, L = checked
    cfg = scenes.with_size(scenes.BATCH64_1242x375, n_disp=256)
    frames = [scenes.make_frame(cfg, 1200 + k)[:2] for k in range(4)]
    _run(torch, L, frames, ld.default_params(n_disp=256), capture=False)
    p = ld.default_params(n_disp=16)
    groups = []
    for g, (w, h) in enumerate(((70, 33), (40, 20), (130, 50))):
        fr = [scenes.make_tiny_frame(w, h, 16, 1300 + 10 * g + k) for k in range(2)]
        groups.append((torch.from_numpy(np.stack([f[0] for f in fr])).cuda(),
                       torch.from_numpy(np.stack([f[1] for f in fr])).cuda()))
    stream = torch.cuda.Stream()
    det = ld.Detector(130, 50, 6, p, stream=stream, lib=L)
    try:
        assert L.ld_check_reset() == ld.OK
        with torch.cuda.stream(stream):
            for mixed in (False, True):
                outs = det.detect_groups(groups, mixed=mixed)
                torch.cuda.synchronize()
                _clean(L)
                for (d, i), o in zip(groups, outs):
                    res = ld.Detector.lanes(o)
                    dn, im = d.cpu().numpy(), i.cpu().numpy()
                    for k in range(dn.shape[0]):
                        compare_frame(None, res[k], k, dn[k], im[k], p, stages=False)
    finally:
        det.close()


def test_maximum_frame_size_checked(checked):
    """One 4096 x 1088 frame at D = 256 (the handle limits) through the checked library: a clean status and
    every stage the oracle's."""
    torch, L = checked
    cfg = scenes.with_size(scenes.HD_1920x1080, width=ld.MAX_W, height=ld.MAX_H, n_disp=ld.MAX_D)
    frames = [scenes.make_frame(cfg, 1400)[:2]]
    _run(torch, L, frames, ld.default_params(n_disp=cfg.n_disp))


def test_serving_checked(checked):
    """The serving runtime through the checked library: frames of two sizes from three streams, pinned and
    batched submits with slots added under a budget; a clean status and every result the frame's result
    alone (regular library)."""
    torch, L = checked
    sizes = [(70, 33), (130, 50)]
    p = ld.default_params(n_disp=16)
    frames = []
    for k in range(8):
        for sid in range(3):
            wh = sizes[(sid + k) % 2]
            frames.append((sid, wh) + scenes.make_tiny_frame(wh[0], wh[1], 16, 1500 + 10 * sid + k))
    alone = []
    dets = {wh: ld.Detector(wh[0], wh[1], 1, p) for wh in sizes}
    for sid, wh, d, i in frames:
        alone.append(dets[wh].detect_host(d[None], i[None])[0].tobytes())
    for det in dets.values():
        det.close()
    assert L.ld_check_reset() == ld.OK
    srv = ld.Server(sizes, p, n_streams=3, slots_per_size=1, max_batch=2, max_wait_us=200,
                    hbm_budget_bytes=1 << 30, lib=L)
    got = []
    keep = []
    try:
        for wh in sizes:   # runs of one size, pinned, several slots' worth per call
            run = [t for t, f in enumerate(frames) if f[1] == wh]
            d = torch.from_numpy(np.stack([frames[t][2] for t in run])).pin_memory()
            i = torch.from_numpy(np.stack([frames[t][3] for t in run])).pin_memory()
            keep.append((d, i))
            tags = np.array(run, np.uint64)
            sids = np.array([frames[t][0] for t in run], np.int32)
            at = 0
            while at < len(run):
                at += srv.submit_batch(sids[at:], d[at:], i[at:], tags[at:], pinned=True)
                if at < len(run):
                    got.extend(srv.poll(timeout_ms=50))
        srv.drain()
        while len(r := srv.poll()):
            got.extend(r)
        torch.cuda.synchronize()
        _clean(L)
        assert sorted(int(r["tag"]) for r in got) == list(range(len(frames)))
        for r in got:
            assert r["lanes"].tobytes() == alone[int(r["tag"])], f"frame {int(r['tag'])}"
    finally:
        srv.close()
