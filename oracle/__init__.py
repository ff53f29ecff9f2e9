"""CPU oracle of the stereo lane-detection path (ctypes binding of ``oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain single-threaded restatement of the paper's steps
(Fan & Dahnoun, arXiv 1807.02752, Sec. 2.2-2.4) that the tests, the smoke check and the benchmark's
CPU-baseline leg compare the CUDA library against.  The library itself never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_LANES = 8
F_NO_ROAD, F_CAP_Y, F_DEGEN_Y, F_CAP_X, F_DEGEN_X, F_NO_LANES = 1, 2, 4, 8, 16, 32


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no FMA contraction)."""
    stale = force or not os.path.exists(_LIB) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB)
    if stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("n_disp", C.c_int32), ("tau_y", C.c_int32), ("lambda_y", C.c_int32), ("tr_y", C.c_float),
        ("eps_num", C.c_int32), ("eps_den", C.c_int32), ("varpi", C.c_float), ("bilateral", C.c_int32),
        ("bf_rho", C.c_int32), ("sigma_s", C.c_double), ("sigma_r", C.c_double), ("edge_thresh", C.c_int32),
        ("vote_rho", C.c_int32), ("chi", C.c_int32), ("tau_x", C.c_int32), ("lambda_x", C.c_int32),
        ("tr_x", C.c_float), ("sigma_g", C.c_double), ("box_nu", C.c_int32), ("box_vs", C.c_int32),
        ("lambda_g", C.c_int32), ("xi_num", C.c_int32), ("xi_den", C.c_int32), ("thr_num", C.c_int32),
        ("thr_den", C.c_int32), ("near_px", C.c_int32), ("max_lanes", C.c_int32), ("ransac_hyps", C.c_int32),
        ("ransac_rounds", C.c_int32), ("seed", C.c_uint64), ("wg_gaussian", C.c_int32), ("pad0", C.c_int32),
        ("thr_abs", C.c_int64), ("dp_literal", C.c_int32), ("band_literal_bottom", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Lanes(C.Structure):
    _fields_ = [
        ("n_lanes", C.c_int32), ("flags", C.c_int32), ("start_u", C.c_int32 * MAX_LANES),
        ("energy", C.c_int64 * MAX_LANES), ("v_top", C.c_int32), ("centre", C.c_int32),
        ("scale_exp", C.c_int32), ("beta", C.c_double * 3), ("gamma", C.c_double * 5),
        ("rounds_y", C.c_int32), ("rounds_x", C.c_int32),
    ]


_P = C.c_void_p


class Dumps(C.Structure):
    _fields_ = [(n, _P) for n in ("m_y", "path_y", "inl_y", "F", "Vpy", "Ibf", "edge", "Gx", "Gy", "votes",
                                  "m_x", "path_x", "inl_x", "Vpx", "Gw", "M1", "HE")]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        i32, p = C.c_int32, C.c_void_p
        L.or_default_params.argtypes = [C.POINTER(Params)]
        L.or_n_starts.argtypes = [i32, C.POINTER(Params)]
        L.or_n_starts.restype = i32
        L.or_tables.argtypes = [C.POINTER(Params), p, p, p]
        L.or_philox4x32_10.argtypes = [p, p, p]
        L.or_vdisparity.argtypes = [p, i32, i32, i32, p]
        L.or_dp_vdisp.argtypes = [p, i32, i32, i32, i32, p]
        L.or_dp_vdisp.restype = C.c_int64
        L.or_dp_vdisp_literal.argtypes = [p, i32, i32, i32, i32, p]
        L.or_dp_vdisp_literal.restype = C.c_int64
        L.or_lsf.argtypes = [p, p, p, i32, i32, i32, i32, p]
        L.or_lsf.restype = i32
        L.or_hypothesis.argtypes = [p, p, p, i32, i32, C.c_float, i32, i32, i32, C.POINTER(Params), i32, i32, p, p]
        L.or_hypothesis.restype = i32
        L.or_ransac.argtypes = [p, p, i32, i32, C.c_float, i32, C.POINTER(Params), i32, i32, p, p, p]
        L.or_ransac.restype = i32
        L.or_bilateral.argtypes = [p, i32, i32, C.POINTER(Params), p]
        L.or_median.argtypes = [p, i32, i32, i32, p]
        L.or_integral.argtypes = [p, i32, i32, i32, p]
        L.or_block_stats.argtypes = [p, i32, i32, i32, p, p]
        L.or_ncc_cmp.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64]
        L.or_ncc_cmp.restype = i32
        L.or_srp.argtypes = [p, p, i32, i32, i32, i32, i32, i32, p]
        L.or_lrc.argtypes = [p, p, i32, i32, i32, p]
        L.or_stereo.argtypes = [p, p, i32, i32, i32, i32, i32, i32, p, p, p]
        L.or_sobel.argtypes = [p, i32, i32, p, p]
        L.or_band.argtypes = [p, i32, i32, i32, i32, i32, i32, p]
        L.or_dp_vpx.argtypes = [p, i32, i32, i32, i32, i32, p]
        L.or_dp_vpx.restype = C.c_int64
        L.or_box_sobel.argtypes = [p, i32, i32, i32, i32, p, p]
        L.or_energy.argtypes = [p, i32, i32, i32, p, p, i32, i32, i32, p]
        L.or_select.argtypes = [p, i32, i32, C.POINTER(Params), C.POINTER(Lanes)]
        L.or_track.argtypes = [p, p, i32, i32, i32, p]
        L.or_detect.argtypes = [p, p, i32, i32, C.POINTER(Params), C.POINTER(Lanes), C.POINTER(Dumps)]
        L.or_detect.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    lib().or_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def basis(H: int):
    """(centre, e) of the polynomial basis tau = (v - centre) / 2^e used for every fit."""
    centre = (H - 1) // 2
    e = 0
    while (1 << e) < max(centre, H - 1 - centre):
        e += 1
    return centre, e


def n_starts(W: int, p: Params | None = None) -> int:
    p = p or default_params()
    return int(lib().or_n_starts(W, C.byref(p)))


def tables(p: Params | None = None):
    p = p or default_params()
    n = 2 * p.bf_rho + 1
    ws = np.zeros(n * n, np.int32)
    wr = np.zeros(256, np.int32)
    wg = np.zeros(16385, np.int32)
    lib().or_tables(C.byref(p), _ptr(ws), _ptr(wr), _ptr(wg))
    return ws.reshape(n, n), wr, wg


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def vdisparity(disp: np.ndarray, D: int) -> np.ndarray:
    d = np.ascontiguousarray(disp, np.float32)
    H, W = d.shape
    m = np.zeros((H, D), np.int32)
    lib().or_vdisparity(_ptr(d), W, H, D, _ptr(m))
    return m


def dp_vdisp(m_y: np.ndarray, tau: int = 6, lam: int = 1):
    m = np.ascontiguousarray(m_y, np.int32)
    H, D = m.shape
    path = np.zeros(D, np.int16)
    e = lib().or_dp_vdisp(_ptr(m), H, D, tau, lam, _ptr(path))
    return int(e), path


def dp_vdisp_literal(m_y: np.ndarray, tau: int = 6, lam: int = 1):
    m = np.ascontiguousarray(m_y, np.int32)
    H, D = m.shape
    path = np.zeros(D, np.int16)
    e = lib().or_dp_vdisp_literal(_ptr(m), H, D, tau, lam, _ptr(path))
    return int(e), path


def lsf(x, y, m: int, centre: int, e: int, use=None):
    x = np.ascontiguousarray(x, np.int32)
    y = np.ascontiguousarray(y, np.int32)
    u = None if use is None else np.ascontiguousarray(use, np.uint8)
    coef = np.zeros(5, np.float64)
    rc = lib().or_lsf(_ptr(x), _ptr(y), None if u is None else _ptr(u), len(x), m, centre, e, _ptr(coef))
    return rc, coef[:m]


def hypothesis(x, y, member, m, tr, stage, rnd, hyp, p: Params, centre, e):
    x = np.ascontiguousarray(x, np.int32)
    y = np.ascontiguousarray(y, np.int32)
    mem = np.ascontiguousarray(member, np.uint8)
    chosen = np.zeros(5, np.int32)
    inl = np.zeros(len(x), np.uint8)
    c = lib().or_hypothesis(_ptr(x), _ptr(y), _ptr(mem), len(x), m, tr, stage, rnd, hyp, C.byref(p), centre, e,
                            _ptr(chosen), _ptr(inl))
    return int(c), chosen[:m], inl


def ransac(x, y, m, tr, stage, p: Params, centre, e):
    x = np.ascontiguousarray(x, np.int32)
    y = np.ascontiguousarray(y, np.int32)
    mem = np.zeros(len(x), np.uint8)
    coef = np.zeros(5, np.float64)
    rounds = np.zeros(1, np.int32)
    fl = lib().or_ransac(_ptr(x), _ptr(y), len(x), m, tr, stage, C.byref(p), centre, e, _ptr(mem), _ptr(coef),
                         _ptr(rounds))
    return int(fl), mem, coef[:m], int(rounds[0])


def bilateral(img: np.ndarray, p: Params | None = None) -> np.ndarray:
    p = p or default_params()
    im = np.ascontiguousarray(img, np.uint8)
    H, W = im.shape
    out = np.zeros_like(im)
    lib().or_bilateral(_ptr(im), W, H, C.byref(p), _ptr(out))
    return out


def median(img: np.ndarray, rho: int = 5) -> np.ndarray:
    im = np.ascontiguousarray(img, np.uint8)
    H, W = im.shape
    out = np.zeros_like(im)
    lib().or_median(_ptr(im), W, H, rho, _ptr(out))
    return out


def integral(img: np.ndarray, square: bool = False) -> np.ndarray:
    im = np.ascontiguousarray(img, np.uint8)
    H, W = im.shape
    out = np.zeros((H + 1, W + 1), np.int64)
    lib().or_integral(_ptr(im), W, H, 1 if square else 0, _ptr(out))
    return out


def block_stats(img: np.ndarray, rho: int = 3):
    im = np.ascontiguousarray(img, np.uint8)
    H, W = im.shape
    s = np.zeros((H, W), np.int32)
    D = np.zeros((H, W), np.int64)
    lib().or_block_stats(_ptr(im), W, H, rho, _ptr(s), _ptr(D))
    return s, D


def ncc_cmp(N1: int, D1: int, N2: int, D2: int) -> int:
    return int(lib().or_ncc_cmp(N1, D1, N2, D2))


def srp(a: np.ndarray, b: np.ndarray, rho: int = 3, dmax: int = 127, tau: int = 1, direction: int = 0):
    aa, bb = np.ascontiguousarray(a, np.uint8), np.ascontiguousarray(b, np.uint8)
    H, W = aa.shape
    out = np.zeros((H, W), np.int16)
    lib().or_srp(_ptr(aa), _ptr(bb), W, H, rho, dmax, tau, direction, _ptr(out))
    return out


def lrc(lf: np.ndarray, rt: np.ndarray, tr: int = 3):
    a, b = np.ascontiguousarray(lf, np.int16), np.ascontiguousarray(rt, np.int16)
    H, W = a.shape
    out = np.zeros((H, W), np.int16)
    lib().or_lrc(_ptr(a), _ptr(b), W, H, tr, _ptr(out))
    return out


def stereo(left: np.ndarray, right: np.ndarray, rho: int = 3, dmax: int = 127, tau: int = 1, tr: int = 3):
    """(left map, right map, checked disparity) of a rectified pair, int16 [H][W]."""
    L_, R_ = np.ascontiguousarray(left, np.uint8), np.ascontiguousarray(right, np.uint8)
    H, W = L_.shape
    lf, rt, d = (np.zeros((H, W), np.int16) for _ in range(3))
    lib().or_stereo(_ptr(L_), _ptr(R_), W, H, rho, dmax, tau, tr, _ptr(lf), _ptr(rt), _ptr(d))
    return lf, rt, d


def sobel(I: np.ndarray):
    im = np.ascontiguousarray(I, np.uint8)
    H, W = im.shape
    gx = np.zeros((H, W), np.int16)
    gy = np.zeros((H, W), np.int16)
    lib().or_sobel(_ptr(im), W, H, _ptr(gx), _ptr(gy))
    return gx, gy


def band(votes: np.ndarray, v_top: int, chi: int = 25, rho: int = 1, literal_bottom: bool = False) -> np.ndarray:
    c = np.ascontiguousarray(votes, np.int32)
    H, W = c.shape
    m = np.zeros((H, W), np.int32)
    lib().or_band(_ptr(c), W, H, v_top, chi, rho, 1 if literal_bottom else 0, _ptr(m))
    return m


def dp_vpx(m_x: np.ndarray, v_top: int, tau: int = 5, lam: int = 1):
    m = np.ascontiguousarray(m_x, np.int32)
    H, W = m.shape
    path = np.zeros(H, np.int16)
    e = lib().or_dp_vpx(_ptr(m), W, H, v_top, tau, lam, _ptr(path))
    return int(e), path


def box_sobel(gw: np.ndarray, nu: int = 1, vs: int = 3):
    g = np.ascontiguousarray(gw, np.int32)
    H, W = g.shape
    m0 = np.zeros((H, W), np.int32)
    m1 = np.zeros((H, W), np.int32)
    lib().or_box_sobel(_ptr(g), W, H, nu, vs, _ptr(m0), _ptr(m1))
    return m0, m1


def energy(m1: np.ndarray, v_top: int, vpx, vpy, S0: int, ns: int, lambda_g: int = 1) -> np.ndarray:
    m = np.ascontiguousarray(m1, np.int32)
    H, W = m.shape
    vx = np.ascontiguousarray(vpx, np.float32)
    vy = np.ascontiguousarray(vpy, np.float32)
    he = np.zeros(ns, np.int64)
    lib().or_energy(_ptr(m), W, H, v_top, _ptr(vx), _ptr(vy), S0, ns, lambda_g, _ptr(he))
    return he


def select(he: np.ndarray, S0: int, p: Params | None = None):
    p = p or default_params()
    h = np.ascontiguousarray(he, np.int64)
    out = Lanes()
    lib().or_select(_ptr(h), len(h), S0, C.byref(p), C.byref(out))
    return lanes_dict(out)


def track(vpx, vpy, v_top: int, start_u: int) -> np.ndarray:
    """Alg. 7's drawing step: the Eq. 25 track of a lane started at (start_u, H-1), float32 [H], NaN above v_top."""
    vx = np.ascontiguousarray(vpx, np.float32)
    vy = np.ascontiguousarray(vpy, np.float32)
    out = np.zeros(len(vx), np.float32)
    lib().or_track(_ptr(vx), _ptr(vy), len(vx), v_top, start_u, _ptr(out))
    return out


def lanes_dict(out: Lanes) -> dict:
    n = out.n_lanes
    return {
        "n_lanes": n, "flags": out.flags, "start_u": list(out.start_u)[:n], "energy": list(out.energy)[:n],
        "v_top": out.v_top, "centre": out.centre, "scale_exp": out.scale_exp, "beta": list(out.beta),
        "gamma": list(out.gamma), "rounds_y": out.rounds_y, "rounds_x": out.rounds_x,
    }


def detect(disp: np.ndarray, img: np.ndarray, p: Params | None = None, dumps: bool = True) -> dict:
    """Run the whole path on one frame.  Returns the lanes and, with dumps=True, every intermediate."""
    p = p or default_params()
    d = np.ascontiguousarray(disp, np.float32)
    im = np.ascontiguousarray(img, np.uint8)
    H, W = d.shape
    D = p.n_disp
    ns = n_starts(W, p)
    arrays = {}
    du = Dumps()
    if dumps:
        spec = {
            "m_y": ((H, D), np.int32), "path_y": ((D,), np.int16), "inl_y": ((D,), np.uint8),
            "F": ((H,), np.float32), "Vpy": ((H,), np.float32), "Ibf": ((H, W), np.uint8),
            "edge": ((H, W), np.uint8), "Gx": ((H, W), np.int16), "Gy": ((H, W), np.int16),
            "votes": ((H, W), np.int32), "m_x": ((H, W), np.int32), "path_x": ((H,), np.int16),
            "inl_x": ((H,), np.uint8), "Vpx": ((H,), np.float32), "Gw": ((H, W), np.int32),
            "M1": ((H, W), np.int32), "HE": ((ns,), np.int64),
        }
        for k, (shape, dt) in spec.items():
            arrays[k] = np.zeros(shape, dt)
            setattr(du, k, arrays[k].ctypes.data)
    out = Lanes()
    rc = lib().or_detect(_ptr(d), _ptr(im), W, H, C.byref(p), C.byref(out), C.byref(du))
    if rc != 0:
        raise ValueError("oracle rejected the frame")
    res = lanes_dict(out)
    res.update(arrays)
    return res
