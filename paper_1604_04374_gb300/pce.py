"""ctypes binding of include/pce.h (argument marshalling only).

The functions named pce_* take and return the same things as their C
counterparts, with device pointers and streams passed as Python integers.
``Plan`` wraps a plan handle around torch CUDA tensors.  Every failing call
raises PceError carrying the status and pce_last_error_string().
"""
from __future__ import annotations

import ctypes
import math
import os

from . import build as _build

PCE_OK, PCE_ERR_INVALID, PCE_ERR_UNSUPPORTED, PCE_ERR_OOM, PCE_ERR_CUDA, PCE_ERR_TIMEOUT = range(6)
PCE_FLAG_NONE = 0
PCE_FLAG_UNFUSED = 1
PCE_FLAG_LOWP_STORAGE = 2
PCE_FLAG_PRODUCT_CONVOLUTION = 4
PCE_FLAG_SECTIONED = 8
STATUS_NAMES = {0: "PCE_OK", 1: "PCE_ERR_INVALID", 2: "PCE_ERR_UNSUPPORTED", 3: "PCE_ERR_OOM",
                4: "PCE_ERR_CUDA", 5: "PCE_ERR_TIMEOUT"}

_lib = None


class PceTask(ctypes.Structure):
    """struct pce_task of include/pce.h."""
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("batch", ctypes.c_int64), ("adjoint", ctypes.c_int), ("reserved", ctypes.c_int)]


def _task_array(tasks):
    """tasks: iterable of (plan handle, in ptr, out ptr, batch, adjoint)."""
    tasks = list(tasks)
    arr = (PceTask * max(1, len(tasks)))()
    for i, (plan, ip, op, b, adj) in enumerate(tasks):
        arr[i] = PceTask(plan, ip, op, b, 1 if adj else 0, 0)
    return arr, len(tasks)


class PceError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libpce.so (built in-tree by paper_1604_04374_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1604_04374_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.pce_plan_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int,
                                    P, P, ctypes.c_uint32, P]
    lib.pce_plan_create_from_spectra.argtypes = lib.pce_plan_create.argtypes
    lib.pce_plan_create_separable.argtypes = [ctypes.POINTER(P), ctypes.POINTER(i64), ctypes.c_int, P, P, P,
                                              ctypes.c_uint32, P]
    lib.pce_plan_create_separable_from_spectra.argtypes = lib.pce_plan_create_separable.argtypes
    lib.pce_plan_slots.argtypes = [P]
    lib.pce_plan_slots.restype = ctypes.c_int
    lib.pce_apply.argtypes = [P, P, P, i64, P]
    lib.pce_apply_adjoint.argtypes = [P, P, P, i64, P]
    lib.pce_plan_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(i64)]
    lib.pce_plan_hhat.argtypes = [P, P, P]
    lib.pce_plan_destroy.argtypes = [P]
    lib.pce_last_error_string.restype = ctypes.c_char_p
    lib.pce_last_error_string.argtypes = []
    lib.pce_launch_count.argtypes = [P, ctypes.c_int, i64]
    lib.pce_launch_count.restype = i64
    lib.pce_backward_workspace_bytes.argtypes = [P, i64]
    lib.pce_backward_workspace_bytes.restype = i64
    lib.pce_backward.argtypes = [P, P, P, P, P, P, i64, P, i64, P]
    lib.pce_backward.restype = ctypes.c_int
    lib.pce_plan_status.argtypes = [P, P]
    lib.pce_plan_status.restype = ctypes.c_int
    lib.pce_plan_inject_wait_timeout.argtypes = [P, i64]
    lib.pce_plan_inject_wait_timeout.restype = ctypes.c_int
    lib.pce_apply_noalloc.argtypes = [P, P, P, i64, P]
    lib.pce_apply_noalloc.restype = ctypes.c_int
    lib.pce_plan_set_timing.argtypes = [P, ctypes.c_int]
    lib.pce_plan_timing.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(i64)]
    TP = ctypes.POINTER(PceTask)
    lib.pce_apply_batch.argtypes = [TP, ctypes.c_int, P]
    lib.pce_batch_create.argtypes = [ctypes.POINTER(P), TP, ctypes.c_int, ctypes.c_int]
    lib.pce_batch_run.argtypes = [P, P]
    lib.pce_batch_launch.argtypes = [P, P]
    lib.pce_batch_info.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.pce_batch_destroy.argtypes = [P]
    lib.pce_batch_autotune.argtypes = [P, P]
    lib.pce_construct_projection_1d.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
    lib.pce_construct_projection_1d.restype = ctypes.c_int
    lib.pce_construct_projection_bspline_1d.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
    lib.pce_construct_projection_bspline_1d.restype = ctypes.c_int
    I = ctypes.c_int
    lib.pce_construct_projection_2d.argtypes = [P, I, I, I, I, I, I, P, P, P, P]
    lib.pce_construct_projection_2d.restype = ctypes.c_int
    lib.pce_construct_svd_1d.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_ulonglong, P, P, P, P]
    lib.pce_construct_svd_1d.restype = ctypes.c_int
    lib.pce_batch_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.pce_batch_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.pce_batch_set_tuning.restype = ctypes.c_int
    lib.pce_batch_tuning_log.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.pce_batch_tuning_log.restype = ctypes.c_int
    lib.pce_schedule_lpt.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.pce_plan_autotune.argtypes = [P, i64, ctypes.c_char_p, P]
    IP = ctypes.POINTER(ctypes.c_int)
    lib.pce_plan_tuning.argtypes = [P, IP, IP, IP, ctypes.POINTER(ctypes.c_double)]
    lib.pce_plan_tuning_log.argtypes = [P, ctypes.c_int, IP, IP, IP, ctypes.POINTER(ctypes.c_double)]
    lib.pce_plan_tuning_log.restype = ctypes.c_int
    lib.pce_plan_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.pce_plan_set_tuning.restype = ctypes.c_int
    for name in ("pce_plan_create", "pce_plan_create_from_spectra", "pce_apply", "pce_apply_adjoint",
                 "pce_plan_info", "pce_plan_hhat", "pce_plan_destroy", "pce_plan_set_timing",
                 "pce_plan_timing", "pce_plan_create_separable", "pce_plan_create_separable_from_spectra",
                 "pce_apply_batch", "pce_batch_create", "pce_batch_run",
                 "pce_batch_launch", "pce_batch_info", "pce_batch_destroy", "pce_schedule_lpt",
                 "pce_plan_autotune", "pce_plan_tuning", "pce_batch_autotune", "pce_batch_tuning"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != PCE_OK:
        raise PceError(status, pce_last_error_string())


def pce_last_error_string() -> str:
    return load_library().pce_last_error_string().decode()


def pce_plan_create(ndims: int, shape, m: int, w_ptr: int, h_ptr: int, flags: int = 0,
                    stream: int = 0) -> int:
    handle = ctypes.c_void_p()
    shp = (ctypes.c_int64 * len(shape))(*shape)
    _check(load_library().pce_plan_create(ctypes.byref(handle), ndims, shp, m, w_ptr, h_ptr,
                                          flags, stream))
    return handle.value


def pce_plan_create_separable(shape, m: int, wy_ptr: int, wx_ptr: int, h_ptr: int, flags: int = 0,
                              stream: int = 0, spectra: bool = False) -> int:
    handle = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 2)(*shape)
    lib = load_library()
    fn = lib.pce_plan_create_separable_from_spectra if spectra else lib.pce_plan_create_separable
    _check(fn(ctypes.byref(handle), shp, m, wy_ptr, wx_ptr, h_ptr, flags, stream))
    return handle.value


def pce_plan_slots(plan: int) -> int:
    return int(load_library().pce_plan_slots(plan))


def pce_plan_create_from_spectra(ndims: int, shape, m: int, w_ptr: int, hhat_ptr: int,
                                 flags: int = 0, stream: int = 0) -> int:
    handle = ctypes.c_void_p()
    shp = (ctypes.c_int64 * len(shape))(*shape)
    _check(load_library().pce_plan_create_from_spectra(ctypes.byref(handle), ndims, shp, m, w_ptr,
                                                       hhat_ptr, flags, stream))
    return handle.value


def pce_apply(plan: int, u_ptr: int, y_ptr: int, batch: int, stream: int = 0) -> None:
    _check(load_library().pce_apply(plan, u_ptr, y_ptr, batch, stream))


def pce_apply_adjoint(plan: int, v_ptr: int, x_ptr: int, batch: int, stream: int = 0) -> None:
    _check(load_library().pce_apply_adjoint(plan, v_ptr, x_ptr, batch, stream))


def pce_apply_noalloc(plan: int, u_ptr: int, y_ptr: int, batch: int, stream: int = 0) -> None:
    """y = H_m u on a 2D plan with the intermediates in the library's static device scratch."""
    _check(load_library().pce_apply_noalloc(plan, u_ptr, y_ptr, batch, stream))


def pce_plan_status(plan: int, stream: int = 0) -> None:
    """Raise PceError(PCE_ERR_TIMEOUT) if a kernel gave up a bounded wait since the last check."""
    _check(load_library().pce_plan_status(plan, stream))


def pce_plan_inject_wait_timeout(plan: int, wait_cycles: int) -> None:
    _check(load_library().pce_plan_inject_wait_timeout(plan, wait_cycles))


def pce_backward_workspace_bytes(plan: int, batch: int) -> int:
    return int(load_library().pce_backward_workspace_bytes(plan, batch))


def pce_backward(plan: int, u_ptr: int, r_ptr: int, du_ptr: int, dw_ptr: int, dhhat_ptr: int,
                 batch: int, workspace_ptr: int, workspace_bytes: int, stream: int = 0) -> None:
    """Gradients of L(y), y = H_m u, given r = dL/dy (any output pointer may be 0 to skip it)."""
    _check(load_library().pce_backward(plan, u_ptr, r_ptr, du_ptr or None, dw_ptr or None,
                                       dhhat_ptr or None, batch, workspace_ptr or None,
                                       workspace_bytes, stream))


def pce_plan_info(plan: int, m: int):
    mm = ctypes.c_int()
    boxes = (ctypes.c_int * (4 * m))()
    scratch = ctypes.c_int64()
    _check(load_library().pce_plan_info(plan, ctypes.byref(mm), boxes, ctypes.byref(scratch)))
    return mm.value, [tuple(boxes[4 * k:4 * k + 4]) for k in range(m)], scratch.value


def pce_plan_hhat(plan: int, hhat_ptr: int, stream: int = 0) -> None:
    _check(load_library().pce_plan_hhat(plan, hhat_ptr, stream))


def pce_plan_destroy(plan: int) -> None:
    _check(load_library().pce_plan_destroy(plan))


def pce_launch_count(plan: int, adjoint: bool, batch: int) -> int:
    return int(load_library().pce_launch_count(plan, 1 if adjoint else 0, batch))


def pce_apply_batch(tasks, stream: int = 0) -> None:
    arr, n = _task_array(tasks)
    _check(load_library().pce_apply_batch(arr, n, stream))


def pce_batch_create(tasks, lanes: int) -> int:
    arr, n = _task_array(tasks)
    handle = ctypes.c_void_p()
    _check(load_library().pce_batch_create(ctypes.byref(handle), arr, n, lanes))
    return handle.value


def pce_batch_run(batch: int, stream: int = 0) -> None:
    _check(load_library().pce_batch_run(batch, stream))


def pce_batch_launch(batch: int, stream: int = 0) -> None:
    _check(load_library().pce_batch_launch(batch, stream))


def pce_batch_info(batch: int, n: int):
    """(lanes, scratch bytes, launches per run, modelled makespan ms, [lane of each task])."""
    lanes = ctypes.c_int()
    scratch = ctypes.c_int64()
    launches = ctypes.c_int64()
    ms = ctypes.c_double()
    lane_of = (ctypes.c_int * max(1, n))()
    _check(load_library().pce_batch_info(batch, ctypes.byref(lanes), ctypes.byref(scratch),
                                         ctypes.byref(launches), ctypes.byref(ms), lane_of))
    return lanes.value, scratch.value, launches.value, ms.value, list(lane_of)[:n]


def pce_batch_destroy(batch: int) -> None:
    _check(load_library().pce_batch_destroy(batch))


def pce_batch_autotune(batch: int, stream: int = 0) -> None:
    _check(load_library().pce_batch_autotune(batch, stream))


def pce_batch_tuning(batch: int):
    """(column-variant policy, row-variant policy); -1 = every plan's own choice."""
    c = ctypes.c_int()
    r = ctypes.c_int()
    _check(load_library().pce_batch_tuning(batch, ctypes.byref(c), ctypes.byref(r)))
    return c.value, r.value


def pce_batch_tuning_log(batch: int):
    """[(column policy, row policy, ms per run)] of every policy the last batch autotune timed."""
    lib = load_library()
    n = lib.pce_batch_tuning_log(batch, 0, None, None, None)
    c = (ctypes.c_int * max(1, n))()
    r = (ctypes.c_int * max(1, n))()
    ms = (ctypes.c_double * max(1, n))()
    lib.pce_batch_tuning_log(batch, n, c, r, ms)
    return [(c[i], r[i], ms[i]) for i in range(n)]


def pce_construct_projection_1d(T_ptr: int, n: int, m: int, h_ptr: int, w_ptr: int, stream: int = 0) -> None:
    _check(load_library().pce_construct_projection_1d(T_ptr, n, m, h_ptr, w_ptr, stream))


def pce_construct_projection_bspline_1d(T_ptr: int, n: int, m: int, alpha: int, h_ptr: int, w_ptr: int,
                                        stream: int = 0) -> None:
    _check(load_library().pce_construct_projection_bspline_1d(T_ptr, n, m, alpha, h_ptr, w_ptr, stream))


def pce_construct_projection_2d(T_ptr: int, ny: int, nx: int, sy: int, sx: int, gy: int, gx: int, h_ptr: int,
                                wy_ptr: int, wx_ptr: int, stream: int = 0) -> None:
    _check(load_library().pce_construct_projection_2d(T_ptr, ny, nx, sy, sx, gy, gx, h_ptr, wy_ptr, wx_ptr, stream))


def construct_projection_2d(T, gy: int, gx: int, stream=None):
    """(h [m, ny, nx], wy [m, ny], wx [m, nx]) of the L2 projection of the windowed 2D TVIR
    T [ny, nx, sy, sx] (impulse response at every input position over a centred shift
    window) onto the tensor-product hats of a gy x gx node grid (pce_construct_projection_2d);
    Plan(wy=wy, wx=wx, h=h) applies the projected operator."""
    import torch
    _need_cuda_f32(T, "T")
    if T.dim() != 4:
        raise ValueError("T must be [ny, nx, sy, sx]")
    ny, nx, sy, sx = (int(v) for v in T.shape)
    m = gy * gx
    h = torch.empty((m, ny, nx), dtype=torch.float32, device=T.device)
    wy = torch.empty((m, ny), dtype=torch.float32, device=T.device)
    wx = torch.empty((m, nx), dtype=torch.float32, device=T.device)
    pce_construct_projection_2d(T.data_ptr(), ny, nx, sy, sx, gy, gx, h.data_ptr(), wy.data_ptr(), wx.data_ptr(),
                                _stream_handle(stream))
    return h, wy, wx


def pce_construct_svd_1d(T_ptr: int, n: int, m: int, oversample: int, power_iters: int, seed: int,
                         h_ptr: int, w_ptr: int, sigma_ptr: int = 0, stream: int = 0) -> None:
    _check(load_library().pce_construct_svd_1d(T_ptr, n, m, oversample, power_iters, seed, h_ptr, w_ptr,
                                               sigma_ptr or None, stream))


def construct_svd_1d(T, m: int, oversample: int = 10, power_iters: int = 2, seed: int = 0, stream=None):
    """(h [m, n], w [m, n], sigma [m]) of the truncated SVD of the TVIR T [n, n]
    (T[d, j]: shift d, input position j): h_k = sigma_k f_k, w_k = e_k
    (pce_construct_svd_1d, randomised range finder)."""
    import torch
    _need_cuda_f32(T, "T")
    n = int(T.shape[0])
    if T.dim() != 2 or T.shape[1] != n:
        raise ValueError("T must be [n, n]")
    h = torch.empty((m, n), dtype=torch.float32, device=T.device)
    w = torch.empty((m, n), dtype=torch.float32, device=T.device)
    sig = torch.empty((m,), dtype=torch.float32, device=T.device)
    pce_construct_svd_1d(T.data_ptr(), n, m, oversample, power_iters, seed, h.data_ptr(), w.data_ptr(),
                         sig.data_ptr(), _stream_handle(stream))
    return h, w, sig


def construct_projection_1d(T, m: int, alpha: int = 1, stream=None):
    """(h [m, n], w [m, n]) of the L2 projection of the TVIR T [n, n] (T[d, j]: shift d,
    input position j) onto m periodic B-splines of order alpha (1: hats,
    pce_construct_projection_1d; 2, 3: pce_construct_projection_bspline_1d)."""
    import torch
    _need_cuda_f32(T, "T")
    n = int(T.shape[0])
    if T.dim() != 2 or T.shape[1] != n:
        raise ValueError("T must be [n, n]")
    h = torch.empty((m, n), dtype=torch.float32, device=T.device)
    w = torch.empty((m, n), dtype=torch.float32, device=T.device)
    if alpha == 1:
        pce_construct_projection_1d(T.data_ptr(), n, m, h.data_ptr(), w.data_ptr(), _stream_handle(stream))
    else:
        pce_construct_projection_bspline_1d(T.data_ptr(), n, m, alpha, h.data_ptr(), w.data_ptr(),
                                            _stream_handle(stream))
    return h, w


def pce_schedule_lpt(cost, lanes: int):
    """(lane of every task, makespan) under the longest-processing-time-first rule."""
    n = len(cost)
    c = (ctypes.c_double * max(1, n))(*cost)
    out = (ctypes.c_int * max(1, n))()
    ms = ctypes.c_double()
    _check(load_library().pce_schedule_lpt(c, n, lanes, out, ctypes.byref(ms)))
    return list(out)[:n], ms.value


def pce_plan_autotune(plan: int, batch: int, cache_path: str | None = None, stream: int = 0) -> None:
    path = cache_path.encode() if cache_path else None
    _check(load_library().pce_plan_autotune(plan, batch, path, stream))


def pce_plan_tuning(plan: int):
    """(right-hand sides per launch, column variant, row variant, measured ms per apply)."""
    c = ctypes.c_int()
    v = ctypes.c_int()
    r = ctypes.c_int()
    ms = ctypes.c_double()
    _check(load_library().pce_plan_tuning(plan, ctypes.byref(c), ctypes.byref(v), ctypes.byref(r),
                                          ctypes.byref(ms)))
    return c.value, v.value, r.value, ms.value


def pce_plan_set_tuning(plan: int, chunk: int, col_variant: int, row_variant: int) -> None:
    _check(load_library().pce_plan_set_tuning(plan, chunk, col_variant, row_variant))


def pce_plan_tuning_log(plan: int):
    """[(chunk, column variant, row variant, ms per apply)] of every candidate the last autotune timed."""
    lib = load_library()
    n = lib.pce_plan_tuning_log(plan, 0, None, None, None, None)
    c = (ctypes.c_int * max(1, n))()
    v = (ctypes.c_int * max(1, n))()
    r = (ctypes.c_int * max(1, n))()
    ms = (ctypes.c_double * max(1, n))()
    lib.pce_plan_tuning_log(plan, n, c, v, r, ms)
    return [(c[i], v[i], r[i], ms[i]) for i in range(n)]


KERNEL_KINDS = ("rows_r2c_window", "cols_fwd", "rows_c2r", "rows_r2c", "cols_adj", "rows_adj",
                "fwd_1d", "adj_1d", "plain")


def pce_plan_set_timing(plan: int, enable: bool) -> None:
    _check(load_library().pce_plan_set_timing(plan, 1 if enable else 0))


def pce_plan_timing(plan: int, kind: int):
    """(summed device milliseconds, launches) of kernel kind ``kind`` since timing was enabled."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load_library().pce_plan_timing(plan, kind, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


# ----------------------------------------------------------------- torch side

def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _need_cuda_f32(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """A convolution-product operator H_m on one CUDA device.

    ``w``: float32 CUDA tensor [m, *shape]; exactly one of ``h`` (float32
    [m, *shape], origin at index 0) or ``hhat`` (complex64 [m, Ny, Nx/2+1] or
    [m, N/2+1]).  ``shape`` is (N,) or (Ny, Nx).
    """

    def __init__(self, w=None, h=None, hhat=None, stream=None, flags: int = 0, wy=None, wx=None):
        import torch
        if w is None:
            # separable windows w_k = wy_k (x) wx_k
            _need_cuda_f32(wy, "wy")
            _need_cuda_f32(wx, "wx")
            if wy.dim() != 2 or wx.dim() != 2 or wy.shape[0] != wx.shape[0]:
                raise ValueError("wy must be [m, Ny] and wx [m, Nx]")
            self.m = int(wy.shape[0])
            self.shape = (int(wy.shape[1]), int(wx.shape[1]))
            self.ndims = 2
            self.device = wy.device
            if (h is None) == (hhat is None):
                raise ValueError("give exactly one of h and hhat")
            src = h if h is not None else hhat
            if h is not None:
                _need_cuda_f32(h, "h")
                if tuple(h.shape) != (self.m,) + self.shape:
                    raise ValueError("h must be [m, Ny, Nx]")
            else:
                want = (self.m, self.shape[0], self.shape[1] // 2 + 1)
                if hhat.dtype != torch.complex64 or tuple(hhat.shape) != want or not hhat.is_contiguous():
                    raise ValueError(f"hhat must be a contiguous complex64 tensor of shape {want}")
            with torch.cuda.device(self.device):
                self.handle = pce_plan_create_separable(self.shape, self.m, wy.data_ptr(), wx.data_ptr(),
                                                        src.data_ptr(), flags, _stream_handle(stream),
                                                        spectra=hhat is not None)
            return
        _need_cuda_f32(w, "w")
        self.m = int(w.shape[0])
        self.shape = tuple(int(s) for s in w.shape[1:])
        self.ndims = len(self.shape)
        self.device = w.device
        sh = _stream_handle(stream)
        with torch.cuda.device(self.device):
            if (h is None) == (hhat is None):
                raise ValueError("give exactly one of h and hhat")
            if h is not None:
                _need_cuda_f32(h, "h")
                if tuple(h.shape) != tuple(w.shape):
                    raise ValueError("h and w must have the same shape")
                self.handle = pce_plan_create(self.ndims, self.shape, self.m, w.data_ptr(), h.data_ptr(),
                                              flags, sh)
            else:
                if hhat.dtype != torch.complex64 or not hhat.is_cuda or not hhat.is_contiguous():
                    raise ValueError("hhat must be a contiguous complex64 CUDA tensor")
                want = (self.m,) + self.shape[:-1] + (self.shape[-1] // 2 + 1,)
                if tuple(hhat.shape) != want:
                    raise ValueError(f"hhat must have shape {want}")
                self.handle = pce_plan_create_from_spectra(self.ndims, self.shape, self.m, w.data_ptr(),
                                                           hhat.data_ptr(), flags, sh)

    def _io(self, x, out, name):
        import torch
        _need_cuda_f32(x, name)
        if tuple(x.shape[-self.ndims:]) != self.shape:
            raise ValueError(f"{name} must end with shape {self.shape}")
        batch = x.numel() // max(1, math.prod(self.shape))
        if out is None:
            out = torch.empty_like(x)
        else:
            _need_cuda_f32(out, "out")
            if out.shape != x.shape:
                raise ValueError("out must have the input's shape")
        return batch, out

    def apply(self, u, out=None, stream=None):
        """y = H_m u for u of shape [..., *shape]."""
        batch, out = self._io(u, out, "u")
        pce_apply(self.handle, u.data_ptr(), out.data_ptr(), batch, _stream_handle(stream))
        return out

    def apply_adjoint(self, v, out=None, stream=None):
        """x = H_m^* v for v of shape [..., *shape]."""
        batch, out = self._io(v, out, "v")
        pce_apply_adjoint(self.handle, v.data_ptr(), out.data_ptr(), batch, _stream_handle(stream))
        return out

    def info(self):
        """(m, support boxes [(r0, nr, c0, nc)], scratch bytes)."""
        return pce_plan_info(self.handle, self.m)

    def slots(self) -> int:
        """Distinct column factors when the separable fast path is on, else 0."""
        return pce_plan_slots(self.handle)

    def hhat(self, stream=None):
        import torch
        out = torch.empty((self.m,) + self.shape[:-1] + (self.shape[-1] // 2 + 1,),
                          dtype=torch.complex64, device=self.device)
        pce_plan_hhat(self.handle, out.data_ptr(), _stream_handle(stream))
        return out

    def launch_count(self, adjoint: bool, batch: int) -> int:
        return pce_launch_count(self.handle, adjoint, batch)

    def backward(self, u, r, need_u=True, need_w=True, need_hhat=True, stream=None):
        """(du, dw, dhhat) of L(y), y = H_m u, given r = dL/dy; skipped ones are None."""
        import torch
        batch, _ = self._io(u, u, "u")
        _need_cuda_f32(r, "r")
        if r.shape != u.shape:
            raise ValueError("r must have the shape of u")
        du = torch.empty_like(u) if need_u else None
        dw = torch.empty((self.m,) + self.shape, dtype=torch.float32, device=self.device) if need_w else None
        dh = (torch.empty((self.m,) + self.shape[:-1] + (self.shape[-1] // 2 + 1,), dtype=torch.complex64,
                          device=self.device) if need_hhat else None)
        nbytes = pce_backward_workspace_bytes(self.handle, batch)
        ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.device)
        pce_backward(self.handle, u.data_ptr(), r.data_ptr(), du.data_ptr() if du is not None else 0,
                     dw.data_ptr() if dw is not None else 0, dh.data_ptr() if dh is not None else 0,
                     batch, ws.data_ptr(), nbytes, _stream_handle(stream))
        return du, dw, dh

    def autotune(self, batch: int, cache: str | None = None, stream=None):
        """Pick the column variant and right-hand sides per launch by timing; returns tuning()."""
        pce_plan_autotune(self.handle, batch, cache, _stream_handle(stream))
        return self.tuning()

    def tuning(self):
        """(right-hand sides per launch, column variant, row variant, measured ms per apply)."""
        return pce_plan_tuning(self.handle)

    def tuning_log(self):
        """[(chunk, column variant, row variant, ms per apply)] of every candidate the last autotune timed."""
        return pce_plan_tuning_log(self.handle)

    def set_tuning(self, chunk: int = 0, col_variant: int = 0, row_variant: int = 0) -> None:
        """Set the autotuner's choices by hand (chunk 0: the plan's scratch chunk)."""
        pce_plan_set_tuning(self.handle, chunk, col_variant, row_variant)

    def set_timing(self, enable: bool) -> None:
        pce_plan_set_timing(self.handle, enable)

    def timing(self) -> dict:
        """{kernel kind: (device ms, launches)} recorded since set_timing(True)."""
        out = {}
        for kind, name in enumerate(KERNEL_KINDS):
            ms, n = pce_plan_timing(self.handle, kind)
            if n:
                out[name] = (ms, n)
        return out

    def close(self):
        if getattr(self, "handle", None):
            pce_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A reusable batch of independent applies (pce_batch_*).

    ``tasks``: list of (Plan, input tensor, output tensor, adjoint flag); the
    tensors are held so that their memory stays valid while the batch lives.
    """

    def __init__(self, tasks, lanes: int = 16):
        self._keep = []
        raw = []
        for plan, x, y, adj in tasks:
            batch, y = plan._io(x, y, "in")
            self._keep.append((plan, x, y))
            raw.append((plan.handle, x.data_ptr(), y.data_ptr(), batch, adj))
        self.n = len(raw)
        self.handle = pce_batch_create(raw, lanes)

    def run(self, stream=None):
        pce_batch_run(self.handle, _stream_handle(stream))

    def launch(self, stream=None):
        """Replay the batch as one CUDA graph launch (captured at the first call)."""
        pce_batch_launch(self.handle, _stream_handle(stream))

    def info(self):
        return pce_batch_info(self.handle, self.n)

    def autotune(self, stream=None):
        """Pick the variant policies by timing the whole batch; returns (policies, log)."""
        pce_batch_autotune(self.handle, _stream_handle(stream))
        return pce_batch_tuning(self.handle), pce_batch_tuning_log(self.handle)

    def set_tuning(self, col_policy: int, row_policy: int) -> None:
        """Set the variant policies by hand (-1: every plan's own choice)."""
        _check(load_library().pce_batch_set_tuning(self.handle, col_policy, row_policy))

    def close(self):
        if getattr(self, "handle", None):
            pce_batch_destroy(self.handle)
            self.handle = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_batch(tasks, stream=None) -> None:
    """One-shot batch: tasks = [(Plan, input, output, adjoint flag)] (pce_apply_batch)."""
    raw = []
    for plan, x, y, adj in tasks:
        batch, y = plan._io(x, y, "in")
        raw.append((plan.handle, x.data_ptr(), y.data_ptr(), batch, adj))
    pce_apply_batch(raw, _stream_handle(stream))
