"""Helpers shared by the GPU parity tests: run the CUDA library and the oracle on the same frames and
compare every stage."""
import numpy as np

import oracle
from paper_1807_02752_gb300 import ld


def oracle_params(lp: "ld.Params"):
    return oracle.default_params(**lp.as_dict())


def fvals(beta_or_gamma, H, centre, e, rows):
    tau = (rows - centre) / 2.0 ** e
    return np.polyval(np.asarray(beta_or_gamma)[::-1], tau)


def compare_frame(det: "ld.Detector", res_row, fidx: int, disp, img, p: "ld.Params", stages=True):
    """Compare frame fidx of the last detect call with the oracle.  Returns the oracle result."""
    H, W = disp.shape
    ref = oracle.detect(disp, img, oracle_params(p), dumps=True)
    got = ld.lanes_to_dicts(np.array([res_row]))[0]
    ctx = f"frame {fidx}"
    # lanes, flags, integers: bit-exact
    for k in ("flags", "v_top", "n_lanes", "start_u", "energy", "rounds_y", "rounds_x", "centre", "scale_exp"):
        assert got[k] == ref[k], f"{ctx}: {k} gpu={got[k]} oracle={ref[k]}"
    # fitted parameters: within 1e-4 relative, compared as f(v) and V_px(v) on the road rows
    rows = np.arange(max(ref["v_top"], 0), H)
    if rows.size and not ref["flags"] & (oracle.F_DEGEN_Y | oracle.F_NO_ROAD):
        a = fvals(got["beta"], H, got["centre"], got["scale_exp"], rows)
        b = fvals(ref["beta"], H, ref["centre"], ref["scale_exp"], rows)
        assert np.allclose(a, b, rtol=1e-4, atol=1e-4 * np.abs(b).max()), ctx
    if rows.size and not ref["flags"] & (oracle.F_DEGEN_Y | oracle.F_NO_ROAD | oracle.F_DEGEN_X):
        a = fvals(got["gamma"], H, got["centre"], got["scale_exp"], rows)
        b = fvals(ref["gamma"], H, ref["centre"], ref["scale_exp"], rows)
        assert np.allclose(a, b, rtol=1e-4, atol=1e-4 * np.abs(b).max()), ctx
    if not stages:
        return ref
    assert (det.debug(fidx, ld.STAGE_VDISP, W, H) == ref["m_y"]).all(), f"{ctx}: v-disparity"
    assert (det.debug(fidx, ld.STAGE_PATH_Y, W, H)[1:] == ref["path_y"][1:]).all(), f"{ctx}: road DP path"
    assert (det.debug(fidx, ld.STAGE_INL_Y, W, H) == ref["inl_y"]).all(), f"{ctx}: road inlier set"
    rws = det.debug(fidx, ld.STAGE_ROWS, W, H)
    for i, k in enumerate(("F", "Vpy", "Vpx")):
        assert np.allclose(rws[i], ref[k], rtol=1e-4, atol=1e-4), f"{ctx}: {k}"
    cnt, ent = det.debug(fidx, ld.STAGE_EDGES, W, H)
    edge = np.zeros((H, W), np.uint8)
    gx = np.zeros((H, W), np.int16)
    gy = np.zeros((H, W), np.int16)
    votes = np.zeros((H, W), np.int32)
    for v in np.nonzero(cnt)[0]:
        e = ent[v, :cnt[v]]
        u = e[:, 0].astype(np.int64)
        assert len(np.unique(u)) == len(u), f"{ctx}: duplicate edge entries on row {v}"
        edge[v, u] = 1
        gx[v, u] = e[:, 2]
        gy[v, u] = e[:, 3]
        b = e[:, 1]
        np.add.at(votes[v], b[b >= 0].astype(np.int64), 1)
    assert (edge == ref["edge"]).all(), f"{ctx}: edge map ({int(edge.sum())} vs {int(ref['edge'].sum())})"
    assert (gx == ref["Gx"]).all() and (gy == ref["Gy"]).all(), f"{ctx}: Sobel values"
    assert (votes == ref["votes"]).all(), f"{ctx}: sparse V_px votes"
    if not ref["flags"] & (oracle.F_DEGEN_Y | oracle.F_NO_ROAD):
        vt = ref["v_top"]
        assert (det.debug(fidx, ld.STAGE_PATH_X, W, H)[vt:] == ref["path_x"][vt:]).all(), f"{ctx}: V_px DP path"
        assert (det.debug(fidx, ld.STAGE_INL_X, W, H) == ref["inl_x"]).all(), f"{ctx}: V_px inlier set"
    vt = min(ref["v_top"], H)
    assert (det.debug(fidx, ld.STAGE_M1, W, H)[vt:] == ref["M1"][vt:]).all(), f"{ctx}: M_1"
    assert (det.debug(fidx, ld.STAGE_HE, W, H) == ref["HE"]).all(), f"{ctx}: energy histogram"
    if getattr(det, "capturing", False):
        compare_captured(det, fidx, disp, ref, p, ctx)
    return ref


def compare_captured(det, fidx, disp, ref, p, ctx):
    """The two intermediates the kernels keep on chip (ld_debug_capture): m_x of Alg. 5, bit-exact on every
    row, and I^bf of Eq. 15-16, bit-exact at every pixel the gradient kernel filtered, which must include the
    3x3 neighbourhood of every edge pixel."""
    H, W = disp.shape
    mx = det.debug(fidx, ld.STAGE_MX, W, H)
    assert (mx == ref["m_x"]).all(), f"{ctx}: m_x ({int((mx != ref['m_x']).sum())} cells differ)"
    ibf = det.debug(fidx, ld.STAGE_IBF, W, H)
    done = ibf >= 0
    bad = done & (ibf != ref["Ibf"].astype(np.int16))
    assert not bad.any(), f"{ctx}: I^bf differs at {int(bad.sum())} pixels, first {np.argwhere(bad)[:3].tolist()}"
    # edges are never pruned, so the gradient kernel must have filtered every pixel their Sobel reads
    edge = ref["edge"].astype(bool)
    need = edge.copy()
    for dv in (-1, 0, 1):
        for du in (-1, 0, 1):
            need |= np.roll(np.roll(edge, dv, 0), du, 1)
    missing = need & ~done
    assert not missing.any(), f"{ctx}: I^bf not computed at {int(missing.sum())} pixels the Sobel of an edge reads"
