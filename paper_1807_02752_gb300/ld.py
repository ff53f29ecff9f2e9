"""Python binding of the CUDA lane-detection library (include/ld.h), argument marshalling only.

Every step of the path runs in the library's kernels.  PyTorch is used for device memory and streams.
If lib/libld.so has not been built, load() raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libld.so")
LIB_CHECKED_PATH = os.path.join(HERE, "lib", "libld_checked.so")   # build.build(checked=True)

MAX_LANES = 8
MAX_W, MAX_H, MAX_D = 4096, 1088, 256   # LD_MAX_W, LD_MAX_H, LD_MAX_D: the largest frame a handle takes
LD_STATIC_SCRATCH_BYTES = 8 << 20
OK, E_ARG, E_CUDA, E_NOMEM, E_STATE = 0, -1, -2, -3, -4
F_NO_ROAD, F_CAP_Y, F_DEGEN_Y, F_CAP_X, F_DEGEN_X, F_NO_LANES, F_FALLBACK = 1, 2, 4, 8, 16, 32, 64
NET_PARAMS, NET_TOPK_MAX = 18689, 256
NET_STAGE_XSUM, NET_STAGE_HEATMAP, NET_STAGE_SCORES, NET_STAGE_CFLAG = 1, 2, 3, 4
STAGE_VDISP, STAGE_PATH_Y, STAGE_INL_Y, STAGE_ROWS, STAGE_EDGES, STAGE_PATH_X, STAGE_INL_X, STAGE_M1, STAGE_HE = range(1, 10)
STAGE_MX, STAGE_IBF = 10, 11


class Params(C.Structure):
    """ld_params."""

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


LANES_DTYPE = np.dtype([
    ("n_lanes", "<i4"), ("flags", "<i4"), ("start_u", "<i4", (MAX_LANES,)), ("energy", "<i8", (MAX_LANES,)),
    ("v_top", "<i4"), ("centre", "<i4"), ("scale_exp", "<i4"), ("rounds_y", "<i4"), ("rounds_x", "<i4"),
    ("reserved", "<i4"), ("beta", "<f8", (3,)), ("gamma", "<f8", (5,)),
])
assert LANES_DTYPE.itemsize == 192

MAX_SIZE_CLASSES = 8
E_BUSY = -5


class StereoParams(C.Structure):
    """ld_stereo_params."""

    _fields_ = [("rho", C.c_int32), ("tau", C.c_int32), ("d_max", C.c_int32), ("tr_lrc", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("n_sizes", C.c_int32), ("sizes", (C.c_int32 * 2) * MAX_SIZE_CLASSES), ("slots_per_size", C.c_int32),
                ("max_batch", C.c_int32), ("max_wait_us", C.c_int32), ("n_streams", C.c_int32),
                ("reserved", C.c_int32), ("hbm_budget_bytes", C.c_int64)]


class Group(C.Structure):
    _fields_ = [("disp", C.c_void_p), ("img", C.c_void_p), ("out_lanes", C.c_void_p), ("w", C.c_int32),
                ("h", C.c_int32), ("n_frames", C.c_int32), ("pad", C.c_int32)]


assert C.sizeof(Group) == 40


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64), ("batches", C.c_int64),
                ("mean_batch", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("slots", C.c_int64),
                ("device_bytes", C.c_int64)]


RESULT_DTYPE = np.dtype([("tag", "<u8"), ("stream_id", "<i4"), ("w", "<i4"), ("h", "<i4"), ("pad", "<i4"),
                         ("seq", "<i8"), ("latency_ms", "<f8"), ("lanes", LANES_DTYPE)])
assert RESULT_DTYPE.itemsize == 232

_libs = {}


def load(checked: bool = False):
    """Load lib/libld.so (built by build.py / __graft_entry__.build()), or with checked=True the
    bounds-checked build lib/libld_checked.so (build.build(checked=True))."""
    path = LIB_CHECKED_PATH if checked else LIB_PATH
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_1807_02752_gb300/build.py)")
    L = C.CDLL(path)
    p, i32, P = C.c_void_p, C.c_int32, C.POINTER(Params)
    L.ld_params_default.argtypes = [P]
    L.ld_params_default.restype = None
    L.ld_n_starts.argtypes = [P, i32]
    L.ld_n_starts.restype = i32
    L.ld_create.argtypes = [P, i32, i32, i32, p, C.POINTER(p)]
    L.ld_create.restype = C.c_int
    L.ld_detect.argtypes = [p, p, p, i32, i32, i32, p]
    L.ld_detect.restype = C.c_int
    L.ld_detect_host.argtypes = [p, p, p, i32, i32, i32, p]
    L.ld_detect_host.restype = C.c_int
    L.ld_debug_get.argtypes = [p, i32, i32, p, C.c_size_t]
    L.ld_debug_get.restype = C.c_int
    L.ld_debug_size.argtypes = [p, i32]
    L.ld_debug_size.restype = C.c_size_t
    L.ld_lane_tracks.argtypes = [p, p, i32, p]
    L.ld_lane_tracks.restype = C.c_int
    L.ld_debug_capture.argtypes = [p, i32]
    L.ld_debug_capture.restype = C.c_int
    L.ld_tables.argtypes = [P, p, p, p]
    L.ld_tables.restype = C.c_int
    L.ld_flat_range.argtypes = [P]
    L.ld_flat_range.restype = i32
    L.ld_launches_per_detect.argtypes = []
    L.ld_launches_per_detect.restype = i32
    L.ld_launch_name.argtypes = [i32]
    L.ld_launch_name.restype = C.c_char_p
    L.ld_detect_timed.argtypes = [p, p, p, i32, i32, i32, p, p]
    L.ld_detect_timed.restype = C.c_int
    L.ld_last_error.argtypes = [p]
    L.ld_last_error.restype = C.c_char_p
    L.ld_destroy.argtypes = [p]
    L.ld_destroy.restype = None
    L.ld_road_path_static.argtypes = [P, p, i32, i32, i32, p, p]
    L.ld_road_path_static.restype = C.c_int
    L.ld_detect_groups.argtypes = [p, p, i32]
    L.ld_detect_groups.restype = C.c_int
    L.ld_detect_mixed.argtypes = [p, p, i32]
    L.ld_detect_mixed.restype = C.c_int
    L.ld_tune.argtypes = [p, p, p, i32, i32, i32, p, p]
    L.ld_tune.restype = C.c_int
    L.ld_server_create.argtypes = [P, C.POINTER(ServerConfig), C.POINTER(p)]
    L.ld_server_create.restype = C.c_int
    L.ld_server_submit.argtypes = [p, i32, p, p, i32, i32, C.c_uint64]
    L.ld_server_submit.restype = C.c_int
    L.ld_server_submit_pinned.argtypes = [p, i32, p, p, i32, i32, C.c_uint64]
    L.ld_server_submit_pinned.restype = C.c_int
    L.ld_server_submit_batch.argtypes = [p, i32, p, p, p, i32, i32, p, i32]
    L.ld_server_submit_batch.restype = C.c_int
    L.ld_server_poll.argtypes = [p, p, i32, i32]
    L.ld_server_poll.restype = C.c_int
    L.ld_server_drain.argtypes = [p]
    L.ld_server_drain.restype = C.c_int
    L.ld_server_stream_state.argtypes = [p, i32, p]
    L.ld_server_stream_state.restype = C.c_int
    L.ld_server_stats_get.argtypes = [p, C.POINTER(ServerStats)]
    L.ld_server_stats_get.restype = C.c_int
    L.ld_server_last_error.argtypes = [p]
    L.ld_server_last_error.restype = C.c_char_p
    L.ld_server_destroy.argtypes = [p]
    L.ld_server_destroy.restype = None
    L.ld_server_set_learned.argtypes = [p, p, i32]
    L.ld_server_set_learned.restype = C.c_int
    L.ld_net_param_count.argtypes = []
    L.ld_net_param_count.restype = i32
    L.ld_net_create.argtypes = [p, i32, C.POINTER(p)]
    L.ld_net_set_params.argtypes = [p, p]
    L.ld_net_get_params.argtypes = [p, p]
    L.ld_net_forward.argtypes = [p, p, i32, i32, i32, p]
    L.ld_net_grad.argtypes = [p, p, p, i32, i32, i32, p, p]
    L.ld_net_apply_grad.argtypes = [p, p, C.c_float]
    L.ld_net_train_step.argtypes = [p, p, p, i32, i32, i32, C.c_float, p]
    L.ld_make_training_pairs.argtypes = [p, p, p, i32, i32, i32, p, p, p]
    L.ld_detect_learned.argtypes = [p, p, p, p, i32, i32, i32, i32, p]
    L.ld_net_debug_get.argtypes = [p, i32, i32, p, C.c_size_t]
    L.ld_net_debug_size.argtypes = [p, i32]
    L.ld_net_debug_size.restype = C.c_size_t
    L.ld_net_status.argtypes = [p]
    L.ld_net_status.restype = C.c_int
    L.ld_net_last_error.argtypes = [p]
    L.ld_net_last_error.restype = C.c_char_p
    L.ld_net_destroy.argtypes = [p]
    L.ld_net_destroy.restype = None
    L.ld_stereo_params_default.argtypes = [C.POINTER(StereoParams)]
    L.ld_stereo_params_default.restype = None
    L.ld_stereo_create.argtypes = [p, C.POINTER(StereoParams), C.POINTER(p)]
    L.ld_stereo_run.argtypes = [p, p, p, i32, i32, i32, p]
    L.ld_stereo_run_timed.argtypes = [p, p, p, i32, i32, i32, p, p]
    L.ld_detect_stereo.argtypes = [p, p, p, i32, i32, i32, p]
    L.ld_stereo_maps.argtypes = [p, i32, p, p, p]
    L.ld_stereo_last_error.argtypes = [p]
    L.ld_stereo_last_error.restype = C.c_char_p
    L.ld_stereo_destroy.argtypes = [p]
    L.ld_stereo_destroy.restype = None
    for name in ("ld_stereo_create", "ld_stereo_run", "ld_stereo_run_timed", "ld_detect_stereo", "ld_stereo_maps"):
        getattr(L, name).restype = C.c_int
    for name in ("ld_net_create", "ld_net_set_params", "ld_net_get_params", "ld_net_forward", "ld_net_grad",
                 "ld_net_apply_grad", "ld_net_train_step", "ld_make_training_pairs", "ld_detect_learned",
                 "ld_net_debug_get"):
        getattr(L, name).restype = C.c_int
    L.ld_net_set_fused.argtypes = [p, i32]
    L.ld_net_set_fused.restype = C.c_int
    L.ld_checked_build.argtypes = []
    L.ld_checked_build.restype = i32
    L.ld_check_status.argtypes = [p]
    L.ld_check_status.restype = C.c_int
    L.ld_check_reset.argtypes = []
    L.ld_check_reset.restype = C.c_int
    L.ld_check_site_name.argtypes = [i32]
    L.ld_check_site_name.restype = C.c_char_p
    L.ld_check_selftest.argtypes = []
    L.ld_check_selftest.restype = C.c_int
    _libs[path] = L
    return L


def check_status(L) -> dict:
    """Bounds-check failures recorded by the kernels of library L (ld_check_status): the count and the
    first failure's site, index and bound."""
    out = (C.c_int64 * 4)()
    rc = L.ld_check_status(out)
    if rc != OK:
        raise LDError(rc, L.ld_last_error(None).decode())
    return {"failures": int(out[0]), "site": L.ld_check_site_name(int(out[1])).decode(), "index": int(out[2]),
            "bound": int(out[3])}


EXPORTED = ["ld_params_default", "ld_n_starts", "ld_create", "ld_detect", "ld_detect_host", "ld_detect_timed",
            "ld_debug_get", "ld_debug_size", "ld_debug_capture", "ld_lane_tracks", "ld_tables", "ld_flat_range", "ld_launches_per_detect", "ld_launch_name", "ld_last_error",
            "ld_destroy", "ld_road_path_static", "ld_tune", "ld_detect_groups", "ld_detect_mixed", "ld_server_create", "ld_server_submit",
            "ld_server_submit_pinned", "ld_server_submit_batch", "ld_server_poll",
            "ld_server_drain", "ld_server_stream_state", "ld_server_stats_get", "ld_server_last_error",
            "ld_server_destroy", "ld_server_set_learned", "ld_net_param_count", "ld_net_create", "ld_net_set_params", "ld_net_get_params",
            "ld_net_set_fused",
            "ld_net_forward", "ld_net_grad", "ld_net_apply_grad", "ld_net_train_step", "ld_make_training_pairs",
            "ld_detect_learned", "ld_net_debug_size", "ld_net_debug_get", "ld_net_status", "ld_net_last_error", "ld_net_destroy",
            "ld_stereo_params_default", "ld_stereo_create", "ld_stereo_run", "ld_stereo_run_timed", "ld_detect_stereo",
            "ld_stereo_maps", "ld_stereo_last_error", "ld_stereo_destroy", "ld_checked_build", "ld_check_status",
            "ld_check_reset", "ld_check_site_name", "ld_check_selftest"]


def launch_names():
    L = load()
    return [L.ld_launch_name(k).decode() for k in range(L.ld_launches_per_detect())]


def default_params(**kw) -> Params:
    p = Params()
    load().ld_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def tables(p: Params | None = None):
    p = p or default_params()
    n = 2 * p.bf_rho + 1
    ws = np.zeros(n * n, np.int32)
    wr = np.zeros(256, np.int32)
    wg = np.zeros(16385, np.int32)
    rc = load().ld_tables(C.byref(p), ws.ctypes.data, wr.ctypes.data, wg.ctypes.data)
    if rc != OK:
        raise ValueError("invalid parameters")
    return ws.reshape(n, n), wr, wg


class LDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ld error {code}: {msg}")
        self.code = code


def lanes_to_dicts(arr: np.ndarray):
    out = []
    for r in arr:
        n = int(r["n_lanes"])
        out.append({"n_lanes": n, "flags": int(r["flags"]), "start_u": r["start_u"][:n].tolist(),
                    "energy": r["energy"][:n].tolist(), "v_top": int(r["v_top"]), "centre": int(r["centre"]),
                    "scale_exp": int(r["scale_exp"]), "rounds_y": int(r["rounds_y"]), "rounds_x": int(r["rounds_x"]),
                    "beta": r["beta"].tolist(), "gamma": r["gamma"].tolist()})
    return out


class Detector:
    """A library handle: workspace for frames up to max_w x max_h and batches up to max_batch."""

    def __init__(self, max_w: int, max_h: int, max_batch: int, params: Params | None = None, stream=None,
                 lib=None):
        import torch

        self.L = lib if lib is not None else load()
        self.params = params if params is not None else default_params()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        rc = self.L.ld_create(C.byref(self.params), max_w, max_h, max_batch, C.c_void_p(stream.cuda_stream), C.byref(h))
        if rc != OK:
            raise LDError(rc, self.L.ld_last_error(None).decode())
        self.h = h
        self.max_w, self.max_h, self.max_batch = max_w, max_h, max_batch
        self.capturing = False

    def _check(self, rc):
        if rc != OK:
            raise LDError(rc, self.L.ld_last_error(self.h).decode())

    def n_starts(self, w: int) -> int:
        return int(self.L.ld_n_starts(C.byref(self.params), w))

    def alloc_lanes(self, n: int):
        import torch

        return torch.empty(n * LANES_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

    def detect(self, disp, img, out=None):
        """Enqueue the path on device tensors disp [n,H,W] float32 and img [n,H,W] uint8.

        Returns the device result buffer (uint8, n * 192 bytes); read it with lanes() after syncing.
        """
        assert disp.is_cuda and img.is_cuda and disp.dtype.itemsize == 4 and img.dtype.itemsize == 1
        assert disp.is_contiguous() and img.is_contiguous() and disp.shape == img.shape
        n, H, W = disp.shape
        if out is None:
            out = self.alloc_lanes(n)
        self._check(self.L.ld_detect(self.h, disp.data_ptr(), img.data_ptr(), W, H, n, out.data_ptr()))
        return out

    @staticmethod
    def lanes(out) -> np.ndarray:
        return np.frombuffer(out.cpu().numpy().tobytes(), dtype=LANES_DTYPE)

    def detect_groups(self, groups, outs=None, mixed=False):
        """Frames of several sizes in one call: groups is a list of (disp, img) device tensors [n,H,W], one
        size per group.  Returns the device result buffers, one per group (see lanes()).  mixed=True runs
        ld_detect_mixed (one launch per stage over all frames) instead of ld_detect_groups."""
        arr = (Group * max(1, len(groups)))()
        outs = [self.alloc_lanes(d.shape[0]) for d, _ in groups] if outs is None else outs
        for k, ((d, i), o) in enumerate(zip(groups, outs)):
            assert d.is_cuda and i.is_cuda and d.dtype.itemsize == 4 and i.dtype.itemsize == 1
            assert d.is_contiguous() and i.is_contiguous() and d.shape == i.shape
            n, H, W = d.shape
            arr[k] = Group(d.data_ptr(), i.data_ptr(), o.data_ptr(), W, H, n, 0)
        self._check((self.L.ld_detect_mixed if mixed else self.L.ld_detect_groups)(self.h, arr, len(groups)))
        return outs

    def detect_host(self, disp: np.ndarray, img: np.ndarray) -> np.ndarray:
        """Host buffers in, host results out (copies and kernels on the handle's stream, synchronous)."""
        disp = np.ascontiguousarray(disp, np.float32)
        img = np.ascontiguousarray(img, np.uint8)
        n, H, W = disp.shape
        res = np.zeros(n, LANES_DTYPE)
        self._check(self.L.ld_detect_host(self.h, disp.ctypes.data, img.ctypes.data, W, H, n, res.ctypes.data))
        return res

    def detect_timed(self, disp, img, out):
        """Eager launch with an event around every kernel; returns the per-kernel milliseconds."""
        n, H, W = disp.shape
        ms = np.zeros(self.L.ld_launches_per_detect(), np.float32)
        self._check(self.L.ld_detect_timed(self.h, disp.data_ptr(), img.data_ptr(), W, H, n, out.data_ptr(),
                                           ms.ctypes.data))
        return ms

    def tune(self, disp, img, out=None):
        """Time candidate tile shapes on these frames (device tensors) and keep the fastest for their size.
        Returns the chosen rows per CTA of the v-disparity, gradient and M_1 kernels."""
        n, H, W = disp.shape
        out = self.alloc_lanes(n) if out is None else out
        chosen = np.zeros(3, np.int32)
        self._check(self.L.ld_tune(self.h, disp.data_ptr(), img.data_ptr(), W, H, n, out.data_ptr(),
                                   chosen.ctypes.data))
        return {"vdisp_rows": int(chosen[0]), "grad_rows": int(chosen[1]), "m1_rows": int(chosen[2])}

    def detect_host_ptr(self, disp_ptr: int, img_ptr: int, W: int, H: int, n: int, res: np.ndarray):
        self._check(self.L.ld_detect_host(self.h, disp_ptr, img_ptr, W, H, n, res.ctypes.data))

    def debug(self, frame: int, stage: int, W: int, H: int):
        size = int(self.L.ld_debug_size(self.h, stage))
        buf = np.zeros(size, np.uint8)
        self._check(self.L.ld_debug_get(self.h, frame, stage, buf.ctypes.data, size))
        D = self.params.n_disp
        if stage == STAGE_VDISP:
            return buf.view(np.int32).reshape(H, D)
        if stage == STAGE_PATH_Y:
            return buf.view(np.int16)
        if stage in (STAGE_INL_Y, STAGE_INL_X):
            return buf
        if stage == STAGE_ROWS:
            return buf.view(np.float32).reshape(3, H)
        if stage == STAGE_EDGES:
            cnt = buf[:4 * H].view(np.int32)
            ent = buf[4 * H:].view(np.int16).reshape(H, W, 4)
            return cnt, ent
        if stage == STAGE_PATH_X:
            return buf.view(np.int16)
        if stage == STAGE_M1:
            return buf.view(np.int32).reshape(H, W)
        if stage == STAGE_HE:
            return buf.view(np.int64)
        if stage == STAGE_MX:
            return buf.view(np.int32).reshape(H, W)
        if stage == STAGE_IBF:
            return buf.view(np.int16).reshape(H, W)
        return buf

    def lane_tracks(self, out, n: int, H: int):
        """Eq. 25 tracks of the selected lanes of the last call's first n frames (out: that call's device
        result buffer).  Returns a device float32 tensor [n][LD_MAX_LANES][H], NaN where no lane is."""
        import torch

        tr = torch.empty((n, MAX_LANES, H), dtype=torch.float32, device="cuda")
        self._check(self.L.ld_lane_tracks(self.h, out.data_ptr(), n, tr.data_ptr()))
        return tr

    def capture(self, on: bool = True):
        """Record m_x and I^bf on later calls (LD_STAGE_MX / LD_STAGE_IBF); allocates a capture buffer."""
        self._check(self.L.ld_debug_capture(self.h, 1 if on else 0))
        self.capturing = bool(on)

    def close(self):
        if getattr(self, "h", None):
            self.L.ld_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of frames of several sizes from several camera streams (ld_server_* of ld.h)."""

    def __init__(self, sizes, params: Params | None = None, slots_per_size: int = 2, max_batch: int = 16,
                 max_wait_us: int = 500, n_streams: int = 8, hbm_budget_bytes: int = 0, lib=None):
        self.L = lib if lib is not None else load()
        self.params = params or default_params()
        cfg = ServerConfig()
        cfg.n_sizes = len(sizes)
        for k, (w, h) in enumerate(sizes):
            cfg.sizes[k][0] = w
            cfg.sizes[k][1] = h
        cfg.slots_per_size, cfg.max_batch, cfg.max_wait_us, cfg.n_streams = slots_per_size, max_batch, max_wait_us, n_streams
        cfg.hbm_budget_bytes = hbm_budget_bytes
        self.cfg = cfg
        s = C.c_void_p()
        rc = self.L.ld_server_create(C.byref(self.params), C.byref(cfg), C.byref(s))
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(None).decode())
        self.s = s

    def submit(self, stream_id: int, disp: np.ndarray, img: np.ndarray, tag: int = 0) -> bool:
        """Copy one frame in; False when every slot of its size class is busy (poll and retry)."""
        d = np.ascontiguousarray(disp, np.float32)
        i = np.ascontiguousarray(img, np.uint8)
        H, W = d.shape
        rc = self.L.ld_server_submit(self.s, stream_id, d.ctypes.data, i.ctypes.data, W, H, tag)
        if rc == E_BUSY:
            return False
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())
        return True

    def submit_pinned(self, stream_id: int, disp, img, tag: int = 0) -> bool:
        """Submit one frame held in page-locked host memory (pinned torch tensors [h][w]): read by the device
        directly, so both must stay unchanged until the frame's result has been polled."""
        H, W = disp.shape
        assert disp.is_contiguous() and img.is_contiguous() and disp.dtype.itemsize == 4 and img.dtype.itemsize == 1
        rc = self.L.ld_server_submit_pinned(self.s, stream_id, disp.data_ptr(), img.data_ptr(), W, H, tag)
        if rc == E_BUSY:
            return False
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())
        return True

    def submit_batch(self, stream_ids, disp, img, tags, pinned: bool = False) -> int:
        """Submit frames [n][h][w] of one size (numpy arrays, or pinned torch tensors with pinned=True: then
        they must stay unchanged until their results have been polled).  Returns how many were accepted (the
        first ones)."""
        sid = np.ascontiguousarray(stream_ids, np.int32)
        tg = np.ascontiguousarray(tags, np.uint64)
        if pinned:
            assert disp.is_contiguous() and img.is_contiguous() and disp.dtype.itemsize == 4 and img.dtype.itemsize == 1
            n, H, W = disp.shape
            dp, ip = disp.data_ptr(), img.data_ptr()
        else:
            disp = np.ascontiguousarray(disp, np.float32)
            img = np.ascontiguousarray(img, np.uint8)
            n, H, W = disp.shape
            dp, ip = disp.ctypes.data, img.ctypes.data
        assert sid.shape == (n,) and tg.shape == (n,)
        rc = self.L.ld_server_submit_batch(self.s, n, sid.ctypes.data, dp, ip, W, H, tg.ctypes.data, 1 if pinned else 0)
        if rc == E_BUSY:
            return 0
        if rc < 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())
        return rc

    def set_learned(self, theta=None, top_k: int = 0):
        """Run the batches in the learned form (theta: float32 device tensor of NET_PARAMS values, copied in)
        or, with top_k = 0, in the plain form.  Only while no frame is in the server."""
        if top_k > 0:
            assert theta is not None and theta.is_cuda and theta.numel() == NET_PARAMS
            assert theta.dtype.itemsize == 4 and theta.is_contiguous()
        ptr = None if theta is None else theta.data_ptr()
        rc = self.L.ld_server_set_learned(self.s, ptr, top_k)
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())

    def poll(self, max_out: int = 256, timeout_ms: int = 0) -> np.ndarray:
        out = np.zeros(max_out, RESULT_DTYPE)
        k = self.L.ld_server_poll(self.s, out.ctypes.data, max_out, timeout_ms)
        if k < 0:
            raise LDError(k, self.L.ld_server_last_error(self.s).decode())
        return out[:k]

    def drain(self):
        rc = self.L.ld_server_drain(self.s)
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())

    def stream_state(self, stream_id: int) -> np.ndarray:
        out = np.zeros(1, LANES_DTYPE)
        rc = self.L.ld_server_stream_state(self.s, stream_id, out.ctypes.data)
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())
        return out[0]

    def stats(self) -> dict:
        st = ServerStats()
        rc = self.L.ld_server_stats_get(self.s, C.byref(st))
        if rc != 0:
            raise LDError(rc, self.L.ld_server_last_error(self.s).decode())
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            self.L.ld_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The learned lane-position proposal of a Detector (ld_net_*): device tensors in, device tensors out."""

    def __init__(self, det: "Detector", training: bool = False):
        self.L = load()
        self.det = det
        h = C.c_void_p()
        rc = self.L.ld_net_create(det.h, 1 if training else 0, C.byref(h))
        if rc != OK:
            raise LDError(rc, self.L.ld_net_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LDError(rc, self.L.ld_net_last_error(self.h).decode())

    @staticmethod
    def map_shape(W: int, H: int):
        return (H + 3) // 4, (W + 3) // 4

    def set_params(self, theta):
        """theta: float32 device tensor of NET_PARAMS values (resets the optimiser state)."""
        assert theta.is_cuda and theta.numel() == NET_PARAMS and theta.dtype.itemsize == 4 and theta.is_contiguous()
        self._check(self.L.ld_net_set_params(self.h, theta.data_ptr()))

    def set_fused(self, on: bool = True):
        """Inference forward as one fused kernel (the default) or one kernel per layer (ld_net_set_fused)."""
        self._check(self.L.ld_net_set_fused(self.h, 1 if on else 0))

    def get_params(self):
        import torch

        out = torch.empty(NET_PARAMS, dtype=torch.float32, device="cuda")
        self._check(self.L.ld_net_get_params(self.h, out.data_ptr()))
        return out

    def forward(self, xsum, W: int, H: int):
        import torch

        n = xsum.shape[0]
        mh, mw = self.map_shape(W, H)
        z = torch.empty((n, mh, mw), dtype=torch.float32, device="cuda")
        self._check(self.L.ld_net_forward(self.h, xsum.data_ptr(), W, H, n, z.data_ptr()))
        return z

    def grad(self, xsum, labels, W: int, H: int):
        import torch

        n = xsum.shape[0]
        g = torch.empty(NET_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self.L.ld_net_grad(self.h, xsum.data_ptr(), labels.data_ptr(), W, H, n, g.data_ptr(),
                                       loss.data_ptr()))
        return g, loss

    def apply_grad(self, g, lr: float):
        self._check(self.L.ld_net_apply_grad(self.h, g.data_ptr(), lr))

    def train_step(self, xsum, labels, W: int, H: int, lr: float, loss=None):
        n = xsum.shape[0]
        self._check(self.L.ld_net_train_step(self.h, xsum.data_ptr(), labels.data_ptr(), W, H, n, lr,
                                             None if loss is None else loss.data_ptr()))

    def training_pairs(self, disp, img, xsum_out=None, labels_out=None, lanes_out=None):
        """The plain method's lanes, block sums and labels of frames disp/img [n][H][W] (device tensors)."""
        import torch

        n, H, W = disp.shape
        mh, mw = self.map_shape(W, H)
        xs = xsum_out if xsum_out is not None else torch.empty((n, mh, mw), dtype=torch.int32, device="cuda")
        lb = labels_out if labels_out is not None else torch.empty((n, mh, mw), dtype=torch.uint8, device="cuda")
        ln = lanes_out if lanes_out is not None else self.det.alloc_lanes(n)
        self._check(self.L.ld_make_training_pairs(self.h, disp.data_ptr(), img.data_ptr(), W, H, n, xs.data_ptr(),
                                                  lb.data_ptr(), ln.data_ptr()))
        return xs, lb, ln

    def detect(self, disp, img, top_k: int = 32, heatmap=None, out=None):
        """Learned form of Detector.detect (device tensors); heatmap [n][mh][mw] replaces the network's."""
        n, H, W = disp.shape
        out = self.det.alloc_lanes(n) if out is None else out
        self._check(self.L.ld_detect_learned(self.h, None if heatmap is None else heatmap.data_ptr(),
                                             disp.data_ptr(), img.data_ptr(), W, H, n, top_k, out.data_ptr()))
        return out

    def status(self):
        """Raise if a tensor-core wait of the network kernels ran out (synchronises the device)."""
        self._check(self.L.ld_net_status(self.h))

    def debug(self, frame: int, stage: int):
        size = int(self.L.ld_net_debug_size(self.h, stage))
        buf = np.zeros(size, np.uint8)
        self._check(self.L.ld_net_debug_get(self.h, frame, stage, buf.ctypes.data, size))
        if stage in (NET_STAGE_XSUM,):
            return buf.view(np.int32)
        if stage in (NET_STAGE_HEATMAP, NET_STAGE_SCORES):
            return buf.view(np.float32)
        return buf

    def close(self):
        if getattr(self, "h", None):
            self.L.ld_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stereo_params(**kw) -> StereoParams:
    sp = StereoParams()
    load().ld_stereo_params_default(C.byref(sp))
    for k, v in kw.items():
        setattr(sp, k, v)
    return sp


class Stereo:
    """Stereo matching of a Detector's frames (ld_stereo_*): device uint8 pairs in, device float disparity out."""

    def __init__(self, det: "Detector", sp: StereoParams | None = None):
        self.L = load()
        self.det = det
        self.sp = sp if sp is not None else stereo_params()
        h = C.c_void_p()
        rc = self.L.ld_stereo_create(det.h, C.byref(self.sp), C.byref(h))
        if rc != OK:
            raise LDError(rc, self.L.ld_stereo_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LDError(rc, self.L.ld_stereo_last_error(self.h).decode())

    def run(self, left, right, out=None):
        import torch

        n, H, W = left.shape
        out = torch.empty((n, H, W), dtype=torch.float32, device="cuda") if out is None else out
        self._check(self.L.ld_stereo_run(self.h, left.data_ptr(), right.data_ptr(), W, H, n, out.data_ptr()))
        return out

    def run_timed(self, left, right, out):
        n, H, W = left.shape
        ms = np.zeros(2, np.float32)
        self._check(self.L.ld_stereo_run_timed(self.h, left.data_ptr(), right.data_ptr(), W, H, n, out.data_ptr(),
                                               ms.ctypes.data))
        return ms

    def detect(self, left, right, out=None):
        n, H, W = left.shape
        out = self.det.alloc_lanes(n) if out is None else out
        self._check(self.L.ld_detect_stereo(self.h, left.data_ptr(), right.data_ptr(), W, H, n, out.data_ptr()))
        return out

    def maps(self, frame: int, W: int, H: int):
        lf = np.zeros((H, W), np.int16)
        rt = np.zeros((H, W), np.int16)
        d = np.zeros((H, W), np.float32)
        self._check(self.L.ld_stereo_maps(self.h, frame, lf.ctypes.data, rt.ctypes.data, d.ctypes.data))
        return lf, rt, d

    def close(self):
        if getattr(self, "h", None):
            self.L.ld_stereo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
