"""GPU parity of the stereo stage (ld_stereo_*): both search-range-propagation maps and the checked
disparity bit-exact against the oracle (integer decisions throughout), parameter variants and ragged
sizes, and the whole path from stereo pairs equal to the oracle's detection on the oracle's disparity."""
import numpy as np
import pytest

import oracle
from paper_1807_02752_gb300 import ld, scenes
from gpu_util import oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02752_gb300 import build
    build.build()
    return torch


def _pairs(cfg, n, first):
    fr = [scenes.make_stereo_frame(cfg, first + k) for k in range(n)]
    return np.stack([f[0] for f in fr]), np.stack([f[1] for f in fr])


def _check_maps(torch, cfg, n, first, pairs=None, **kw):
    left, right = pairs if pairs is not None else _pairs(cfg, n, first)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, n, p)
    sp = ld.stereo_params(**kw)
    st = ld.Stereo(det, sp)
    disp = st.run(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()).cpu().numpy()
    dmax = sp.d_max if sp.d_max >= 0 else cfg.n_disp - 1
    for f in range(n):
        lf, rt, d = oracle.stereo(left[f], right[f], sp.rho, dmax, sp.tau, sp.tr_lrc)
        glf, grt, _ = st.maps(f, cfg.width, cfg.height)
        assert np.array_equal(glf, lf), (f, kw, "left map")
        assert np.array_equal(grt, rt), (f, kw, "right map")
        assert np.array_equal(disp[f], d.astype(np.float32)), (f, kw, "checked disparity")
    st.close()
    det.close()


@pytest.mark.parametrize("name,n", [("small_320x120", 3), ("single_1242x375", 2)])
def test_stereo_maps_match_oracle(torch_cuda, name, n):
    cfg, _ = scenes.WORKLOADS[name]
    _check_maps(torch_cuda, cfg, n, first=7)


@pytest.mark.parametrize("kw", [{"rho": 1}, {"rho": 2, "tau": 0}, {"tau": 3, "d_max": 20}, {"tr_lrc": 0},
                                {"d_max": 5}])
def test_stereo_parameter_variants(torch_cuda, kw):
    _check_maps(torch_cuda, scenes.with_size(scenes.SMALL_320x120, n_disp=48), 2, first=17, **kw)


def test_stereo_ragged_sizes(torch_cuda):
    """Random textured pairs (a right image shifted by a row-dependent disparity, plus noise) at ragged sizes."""
    rng = np.random.default_rng(3)
    for w, h in ((333, 97), (17, 16), (1241, 60), (16, 300)):
        left = rng.integers(0, 256, (2, h, w), dtype=np.uint8)
        right = np.empty_like(left)
        for v in range(h):
            s = v * 20 // h
            right[:, v] = np.roll(left[:, v], -s, axis=1)
        right = np.clip(right.astype(int) + rng.integers(-3, 4, right.shape), 0, 255).astype(np.uint8)
        cfg = scenes.with_size(scenes.SMALL_320x120, width=w, height=h, n_disp=32)
        _check_maps(torch_cuda, cfg, 2, first=0, pairs=(left, right))


def test_detect_from_stereo_pairs_matches_oracle(torch_cuda):
    torch = torch_cuda
    cfg = scenes.with_size(scenes.SMALL_320x120, n_disp=48)
    n = 3
    left, right = _pairs(cfg, n, 27)
    p = ld.default_params(n_disp=cfg.n_disp)
    det = ld.Detector(cfg.width, cfg.height, n, p)
    st = ld.Stereo(det)
    out = st.detect(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
    torch.cuda.synchronize()
    got = ld.lanes_to_dicts(ld.Detector.lanes(out))
    op = oracle_params(p)
    for f in range(n):
        _, _, d = oracle.stereo(left[f], right[f], 3, cfg.n_disp - 1, 1, 3)
        ref = oracle.detect(d.astype(np.float32), left[f], op)
        for k in ("flags", "v_top", "n_lanes", "start_u", "energy"):
            assert got[f][k] == ref[k], (f, k, got[f][k], ref[k])
    st.close()
    det.close()


def test_stereo_argument_errors(torch_cuda):
    torch = torch_cuda
    cfg = scenes.SMALL_320x120
    det = ld.Detector(cfg.width, cfg.height, 2, ld.default_params(n_disp=cfg.n_disp))
    for kw in ({"rho": 4}, {"rho": 0}, {"tau": -1}, {"d_max": -2}, {"tr_lrc": -1}):
        with pytest.raises(ld.LDError) as e:
            ld.Stereo(det, ld.stereo_params(**kw))
        assert e.value.code == ld.E_ARG
    st = ld.Stereo(det)
    with pytest.raises(ld.LDError) as e:
        st.maps(0, cfg.width, cfg.height)             # no call yet
    assert e.value.code == ld.E_STATE
    big = torch.zeros((3, cfg.height, cfg.width), dtype=torch.uint8, device="cuda")
    with pytest.raises(ld.LDError) as e:
        st.run(big, big)                                # more frames than the handle's batch
    assert e.value.code == ld.E_ARG
    wide = torch.zeros((1, cfg.height, cfg.width + 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(ld.LDError) as e:
        st.run(wide, wide)
    assert e.value.code == ld.E_ARG
    st.close()
    det.close()
