"""Frames of several sizes in one call: ld_detect_groups (one launch sequence per group, the groups on two
forked streams) and ld_detect_mixed (one launch per stage over every frame, each CTA on its frame's
descriptor).  Every group's results must be the ones ld_detect gives its frames, byte for byte, on a
stream of the handle's own (one captured graph, then replays) and on the legacy default stream (groups one
after another); and every frame's lanes, flags and fitted rows must be the oracle's."""
import numpy as np
import pytest

from paper_1807_02752_gb300 import ld, scenes
from gpu_util import compare_frame

pytestmark = pytest.mark.gpu

SIZES = [((320, 120), 3), ((256, 96), 2), ((400, 150), 1), ((320, 120), 2)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build
    build.build()
    return torch


def _groups(torch, sizes, n_disp, first=300):
    out = []
    for g, ((w, h), n) in enumerate(sizes):
        cfg = scenes.with_size(scenes.SMALL_320x120, width=w, height=h, n_disp=n_disp)
        fr = [scenes.make_frame(cfg, first + 10 * g + k)[:2] for k in range(n)]
        d = torch.from_numpy(np.stack([f[0] for f in fr])).cuda()
        i = torch.from_numpy(np.stack([f[1] for f in fr])).cuda()
        out.append((d, i))
    return out


def _check_oracle(groups, outs, p):
    """Every frame of every group against the oracle (lanes, flags, energies, f and V_px rows)."""
    for g, ((d, i), o) in enumerate(zip(groups, outs)):
        res = ld.Detector.lanes(o)
        dn, im = d.cpu().numpy(), i.cpu().numpy()
        for k in range(dn.shape[0]):
            compare_frame(None, res[k], k, dn[k], im[k], p, stages=False)


def _alone(torch, groups, p):
    res = []
    for d, i in groups:
        n, H, W = d.shape
        det = ld.Detector(W, H, n, p)
        out = det.detect(d, i)
        torch.cuda.synchronize()
        res.append(ld.Detector.lanes(out).tobytes())
        det.close()
    return res


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("own_stream", [True, False])
def test_groups_match_ld_detect(torch_cuda, own_stream, mixed):
    torch = torch_cuda
    p = ld.default_params(n_disp=48)
    groups = _groups(torch, SIZES, 48)
    want = _alone(torch, groups, p)
    stream = torch.cuda.Stream() if own_stream else None
    det = ld.Detector(400, 150, sum(n for _, n in SIZES), p, stream=stream)
    try:
        with torch.cuda.stream(stream or torch.cuda.current_stream()):
            outs = [det.alloc_lanes(d.shape[0]) for d, _ in groups]
            for rep in range(3):            # capture, then replays of the same list
                for o in outs:
                    o.zero_()
                det.detect_groups(groups, outs, mixed=mixed)
                torch.cuda.synchronize()
                got = [ld.Detector.lanes(o).tobytes() for o in outs]
                assert got == want, f"call {rep}"
                if rep == 0:
                    _check_oracle(groups, outs, p)
            # another list (reversed order, so other workspace offsets and stream choices): a new graph
            rev, routs = groups[::-1], outs[::-1]
            for o in routs:
                o.zero_()
            det.detect_groups(rev, routs, mixed=mixed)
            torch.cuda.synchronize()
            assert [ld.Detector.lanes(o).tobytes() for o in outs] == want
            # the workspace held several sizes: ld_debug_get refuses until the next single-size call
            with pytest.raises(ld.LDError) as e:
                det.debug(0, ld.STAGE_VDISP, 320, 120)
            assert e.value.code == ld.E_STATE
            # a plain single-size call on the same handle afterwards is unaffected
            d, i = groups[0]
            o = det.detect(d, i)
            torch.cuda.synchronize()
            assert ld.Detector.lanes(o).tobytes() == want[0]
    finally:
        det.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_groups_full_sizes(torch_cuda, mixed):
    """Three camera sizes at D = 256 (1242x375, 1280x720, 1920x1080) in one captured call."""
    torch = torch_cuda
    p = ld.default_params(n_disp=256)
    groups = []
    for g, (cfg, n) in enumerate(((scenes.with_size(scenes.BATCH64_1242x375, n_disp=256), 4),
                                  (scenes.with_size(scenes.HD_1920x1080, width=1280, height=720, n_disp=256), 2),
                                  (scenes.with_size(scenes.HD_1920x1080, n_disp=256), 2))):
        fr = [scenes.make_frame(cfg, 700 + 10 * g + k)[:2] for k in range(n)]
        groups.append((torch.from_numpy(np.stack([f[0] for f in fr])).cuda(),
                       torch.from_numpy(np.stack([f[1] for f in fr])).cuda()))
    want = _alone(torch, groups, p)
    stream = torch.cuda.Stream()
    det = ld.Detector(1920, 1080, 8, p, stream=stream)
    try:
        with torch.cuda.stream(stream):
            outs = det.detect_groups(groups, mixed=mixed)
            outs = det.detect_groups(groups, outs, mixed=mixed)
            torch.cuda.synchronize()
            assert [ld.Detector.lanes(o).tobytes() for o in outs] == want
        _check_oracle(groups, outs, p)
    finally:
        det.close()


def test_group_argument_errors(torch_cuda):
    torch = torch_cuda
    p = ld.default_params(n_disp=48)
    det = ld.Detector(320, 120, 4, p)
    try:
        d = torch.zeros((3, 120, 320), dtype=torch.float32, device="cuda")
        i = torch.zeros((3, 120, 320), dtype=torch.uint8, device="cuda")
        d2 = torch.zeros((2, 96, 256), dtype=torch.float32, device="cuda")
        i2 = torch.zeros((2, 96, 256), dtype=torch.uint8, device="cuda")
        big = torch.zeros((1, 150, 400), dtype=torch.float32, device="cuda")
        bigi = torch.zeros((1, 150, 400), dtype=torch.uint8, device="cuda")
        for groups in ([(d, i), (d2, i2)],          # 5 frames > max_batch 4
                       [(big, bigi)],               # larger than the handle's frames
                       []):                         # no group
            with pytest.raises(ld.LDError) as e:
                det.detect_groups(groups)
            assert e.value.code == ld.E_ARG
        outs = det.detect_groups([(d[:2], i[:2]), (d2, i2)])   # exactly max_batch: accepted
        torch.cuda.synchronize()
        assert len(outs) == 2
    finally:
        det.close()


@pytest.mark.parametrize("kw", [{"bilateral": 2}, {"dp_literal": 1}, {"tau_y": 15}, {"bilateral": 0, "chi": 5}])
def test_mixed_param_variants(torch_cuda, kw):
    """ld_detect_mixed with the median pre-filter, the literal Eq. 12, the wide road step and the raw image:
    every group's results are the ones ld_detect gives it."""
    torch = torch_cuda
    p = ld.default_params(n_disp=48, **kw)
    groups = _groups(torch, SIZES, 48, first=500)
    want = _alone(torch, groups, p)
    stream = torch.cuda.Stream()
    det = ld.Detector(400, 150, sum(n for _, n in SIZES), p, stream=stream)
    try:
        with torch.cuda.stream(stream):
            outs = det.detect_groups(groups, mixed=True)
            torch.cuda.synchronize()
            assert [ld.Detector.lanes(o).tobytes() for o in outs] == want
    finally:
        det.close()
