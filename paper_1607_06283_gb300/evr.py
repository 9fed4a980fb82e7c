"""Thin ctypes binding of libevr (include/evr.h), names as in the C ABI.

Argument marshalling only: numpy arrays and torch CUDA tensors are turned into
pointers and sizes, and return codes into exceptions.  Every step of the
reconstruction runs in the library's CUDA kernels.  Importing this module loads
paper_1607_06283_gb300/_build/libevr.so and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libevr.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "evr.h")

EVR_OK = 0
EVR_ERR_INVALID_ARG = -1
EVR_ERR_OUT_OF_RANGE = -2
EVR_ERR_BAD_POLARITY = -3
EVR_ERR_NONMONOTONIC = -4
EVR_ERR_OOM = -5
EVR_ERR_CUDA = -6
EVR_ERR_TIMEOUT = -7
EVR_ERR_NOT_SUPPORTED = -8
EVR_T_INIT_FIRST = -(2 ** 63)
EVR_SOLVER_AUTO, EVR_SOLVER_UNFUSED, EVR_SOLVER_TILED = 0, 1, 2
EVR_BATCH_SCHEDULE_AUTO, EVR_BATCH_SCHEDULE_GRAPH, EVR_BATCH_SCHEDULE_PERSISTENT = -1, 0, 1
(EVR_STATE_U, EVR_STATE_P1, EVR_STATE_P2, EVR_STATE_P3, EVR_STATE_F, EVR_STATE_TLAST,
 EVR_STATE_NPOS, EVR_STATE_NNEG, EVR_STATE_CLOCK, EVR_STATE_TINIT, EVR_STATE_SQRTG,
 EVR_STATE_TX, EVR_STATE_TY) = range(13)


class EvrError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {evr_strerror(code)} ({code})")
        self.code = code


class evr_params(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_float),
        ("delta_pos", ctypes.c_float),
        ("delta_neg", ctypes.c_float),
        ("u_min", ctypes.c_float),
        ("u_max", ctypes.c_float),
        ("u_init", ctypes.c_float),
        ("tau", ctypes.c_float),
        ("sigma", ctypes.c_float),
        ("time_scale", ctypes.c_float),
        ("t_max_us", ctypes.c_int64),
        ("t_init_us", ctypes.c_int64),
        ("data_mode", ctypes.c_int),
        ("manifold", ctypes.c_int),
        ("solver", ctypes.c_int),
        ("tile_config", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("data_term", ctypes.c_int),
        ("tvl1_iters", ctypes.c_int),
        ("tvl1_lambda", ctypes.c_float),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libevr.so is not built ({LIB_PATH}); run paper_1607_06283_gb300.build.build() "
            "(nvcc, sm_103a).  There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    sig = {
        "evr_default_params": ([vp], i),
        "evr_create": ([i, i, vp, vp], i),
        "evr_destroy": ([vp], None),
        "evr_set_cuda_stream": ([vp, vp], i),
        "evr_push_events": ([vp, vp, vp, vp, vp, sz], i),
        "evr_push_events_device": ([vp, vp, vp, vp, vp, sz], i),
        "evr_solve": ([vp, i], i),
        "evr_step_device": ([vp, vp, vp, vp, vp, sz, i], i),
        "evr_step": ([vp, vp, vp, vp, vp, sz, i], i),
        "evr_get_image": ([vp, vp, sz], i),
        "evr_get_image_device": ([vp, vp, sz], i),
        "evr_get_image_async": ([vp, vp, sz, ctypes.POINTER(ctypes.c_uint64)], i),
        "evr_wait_image": ([vp, ctypes.c_uint64], i),
        "evr_get_state": ([vp, i, vp, sz], i),
        "evr_set_state": ([vp, i, vp, sz], i),
        "evr_gap": ([vp, vp, vp], i),
        "evr_synchronize": ([vp], i),
        "evr_enable_kernel_timing": ([vp, i], i),
        "evr_kernel_time": ([vp, vp, vp, vp], i),
        "evr_solver_name": ([vp], ctypes.c_char_p),
        "evr_solver_settled": ([vp], i),
        "evr_selftest_wait_timeout": ([vp], i),
        "evr_selftest_cluster_wait_timeout": ([vp], i),
        "evr_selftest_resident_wait_timeout": ([vp], i),
        "evr_strerror": ([i], ctypes.c_char_p),
        "evr_test_fail_alloc_after": ([i], i),
        "evr_measure_peak": ([i, vp, vp], i),
        "evr_gap_static": ([vp] * 7 + [i, i, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       i, vp, vp], i),
        "evr_unrolled_workspace_bytes": ([i, i, i, i, i, i], sz),
        "evr_unrolled_forward": ([vp] * 5 + [i, i, i, i] + [ctypes.c_float] * 5 + [i, i] +
                                 [vp] * 4, i),
        "evr_unrolled_backward": ([vp] * 3 + [i, i, i, i] + [ctypes.c_float] * 5 + [i, i] +
                                  [vp] * 8, i),
        "evr_data_image": ([vp] * 3 + [i, i, i, ctypes.c_float, ctypes.c_float, vp, vp], i),
        "evr_unrolled_timing_start": ([], i),
        "evr_unrolled_timing_stop": ([vp] * 5, i),
        "evr_batch_create": ([i, vp, vp, vp, vp], i),
        "evr_batch_get_images_async": ([vp, vp, sz, ctypes.POINTER(ctypes.c_uint64)], i),
        "evr_batch_wait_images": ([vp, ctypes.c_uint64], i),
        "evr_batch_destroy": ([vp], None),
        "evr_batch_set_cuda_stream": ([vp, vp], i),
        "evr_batch_set_grouping": ([vp, ctypes.c_longlong, i], i),
        "evr_batch_set_schedule": ([vp, i], i),
        "evr_batch_get_schedule": ([vp, vp], i),
        "evr_batch_selftest_persist_timeout": ([vp], i),
        "evr_batch_step_device": ([vp] * 6 + [i], i),
        "evr_batch_step": ([vp] * 6 + [i], i),
        "evr_batch_get_image": ([vp, i, vp, sz], i),
        "evr_batch_get_state": ([vp, i, i, vp, sz], i),
        "evr_batch_get_images": ([vp, vp, sz], i),
        "evr_batch_synchronize": ([vp, vp], i),
        "evr_batch_enable_kernel_timing": ([vp, i], i),
        "evr_batch_kernel_time": ([vp, vp, vp, vp], i),
        "evr_batch_solver_name": ([vp], ctypes.c_char_p),
        "evr_data_image_backward": ([vp] * 4 + [i, i, i, ctypes.c_float, ctypes.c_float] +
                                    [vp] * 5, i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def header_functions() -> list:
    """Names of the functions include/evr.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(evr_[a-z_]+)\s*\(", text)))


def _check(rc: int, what: str) -> None:
    if rc != EVR_OK:
        raise EvrError(rc, what)


def evr_strerror(code: int) -> str:
    return _lib.evr_strerror(int(code)).decode()


def evr_default_params() -> evr_params:
    p = evr_params()
    _check(_lib.evr_default_params(ctypes.byref(p)), "evr_default_params")
    return p


def evr_create(W: int, H: int, params: evr_params | None = None):
    params = params or evr_default_params()
    h = ctypes.c_void_p()
    _check(_lib.evr_create(int(W), int(H), ctypes.byref(params), ctypes.byref(h)), "evr_create")
    return h


def evr_destroy(h) -> None:
    _lib.evr_destroy(h)


EVR_OWN_STREAM = ctypes.c_void_p(-1 & 0xFFFFFFFFFFFFFFFF)


def evr_set_cuda_stream(h, stream_handle) -> None:
    """stream_handle: a cudaStream_t as an int (torch's ``Stream.cuda_stream``; 0 is the
    legacy default stream) or EVR_OWN_STREAM."""
    arg = stream_handle if isinstance(stream_handle, ctypes.c_void_p) else ctypes.c_void_p(
        int(stream_handle))
    _check(_lib.evr_set_cuda_stream(h, arg), "evr_set_cuda_stream")


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def evr_push_events(h, x, y, t_us, pol) -> int:
    """Host arrays; returns the library's code (0 or a negative EVR_ERR_*)."""
    x, px = _host(x, np.uint16)
    y, py = _host(y, np.uint16)
    t, pt = _host(t_us, np.int64)
    p, pp = _host(pol, np.int8)
    n = len(x)
    if not (len(y) == len(t) == len(p) == n):
        raise ValueError("event arrays differ in length")
    return _lib.evr_push_events(h, px, py, pt, pp, n)


def evr_push_events_device(h, x, y, t_us, pol) -> int:
    """torch CUDA tensors (uint16/int32 x,y are accepted as uint16 views), int64 t, int8 pol."""
    n = int(x.numel())
    for a in (x, y, t_us, pol):
        if not a.is_cuda or not a.is_contiguous() or int(a.numel()) != n:
            raise ValueError("device events must be contiguous CUDA tensors of equal length")
    return _lib.evr_push_events_device(h, x.data_ptr(), y.data_ptr(), t_us.data_ptr(),
                                       pol.data_ptr(), n)


def evr_step_device(h, x, y, t_us, pol, iters: int) -> int:
    """Push (device tensors) and solve in one call; returns 0 or the immediate error."""
    rc = _lib.evr_step_device(h, x.data_ptr(), y.data_ptr(), t_us.data_ptr(), pol.data_ptr(),
                              int(x.numel()), int(iters))
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA, EVR_ERR_OOM):
        _check(rc, "evr_step_device")
    return rc


def evr_step(h, x, y, t_us, pol, iters: int) -> int:
    """Push (host arrays) and solve in one call; returns 0 or the immediate error code of
    the host-side checks (as evr_push_events)."""
    x, px = _host(x, np.uint16)
    y, py = _host(y, np.uint16)
    t, pt = _host(t_us, np.int64)
    p, pp = _host(pol, np.int8)
    if not (len(y) == len(t) == len(p) == len(x)):
        raise ValueError("event arrays differ in length")
    rc = _lib.evr_step(h, px, py, pt, pp, len(x), int(iters))
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA, EVR_ERR_OOM):
        _check(rc, "evr_step")
    return rc


def evr_solve(h, iters: int) -> None:
    _check(_lib.evr_solve(h, int(iters)), "evr_solve")


def evr_get_image(h, out: np.ndarray) -> int:
    """Fills a float32 host array of W*H elements; returns the pending device status."""
    assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    rc = _lib.evr_get_image(h, out.ctypes.data, out.size)
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA):
        _check(rc, "evr_get_image")
    return rc


def evr_get_image_async(h, out: np.ndarray) -> int:
    """Queues the copy of the image into a float32 host array of W*H elements (pinned
    memory keeps it asynchronous); returns the ticket for evr_wait_image.  The array
    must stay alive and unread until then."""
    assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
    t = ctypes.c_uint64(0)
    _check(_lib.evr_get_image_async(h, out.ctypes.data, out.size, ctypes.byref(t)),
           "evr_get_image_async")
    return int(t.value)


def evr_wait_image(h, ticket: int) -> int:
    """Waits for a readback; returns the pending device status (0 = none)."""
    rc = _lib.evr_wait_image(h, ctypes.c_uint64(ticket))
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA):
        _check(rc, "evr_wait_image")
    return rc


def evr_get_image_device(h, out) -> None:
    _check(_lib.evr_get_image_device(h, out.data_ptr(), int(out.numel())), "evr_get_image_device")


_STATE_DT = {EVR_STATE_U: np.float32, EVR_STATE_P1: np.float32, EVR_STATE_P2: np.float32,
             EVR_STATE_P3: np.float32, EVR_STATE_F: np.float32, EVR_STATE_SQRTG: np.float32,
             EVR_STATE_TX: np.float32, EVR_STATE_TY: np.float32,
             EVR_STATE_TLAST: np.int64, EVR_STATE_NPOS: np.int32, EVR_STATE_NNEG: np.int32}


def evr_get_state(h, which: int, W: int, H: int):
    if which in (EVR_STATE_CLOCK, EVR_STATE_TINIT):
        out = np.zeros(1, np.int64)
    else:
        out = np.empty((H, W), _STATE_DT[which])
    rc = _lib.evr_get_state(h, int(which), out.ctypes.data, out.nbytes)
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA):
        _check(rc, "evr_get_state")
    return (out[0] if out.size == 1 and which in (EVR_STATE_CLOCK, EVR_STATE_TINIT) else out), rc


def evr_set_state(h, which: int, arr) -> None:
    if which in (EVR_STATE_CLOCK, EVR_STATE_TINIT):
        a = np.array([int(arr)], dtype=np.int64)
    else:
        a = np.ascontiguousarray(arr, dtype=_STATE_DT[which])
    _check(_lib.evr_set_state(h, int(which), a.ctypes.data, a.nbytes), "evr_set_state")


CHECKPOINT_PLANES = (EVR_STATE_U, EVR_STATE_P1, EVR_STATE_P2, EVR_STATE_P3, EVR_STATE_F,
                     EVR_STATE_TLAST, EVR_STATE_NPOS, EVR_STATE_NNEG, EVR_STATE_CLOCK,
                     EVR_STATE_TINIT)


def evr_gap(h):
    pr, du = ctypes.c_double(), ctypes.c_double()
    rc = _lib.evr_gap(h, ctypes.byref(pr), ctypes.byref(du))
    if rc in (EVR_ERR_INVALID_ARG, EVR_ERR_CUDA):
        _check(rc, "evr_gap")
    return pr.value, du.value


EVR_GAP_STATIC_MAX_PIXELS = 4194304


def evr_gap_static(u, p1, p2, p3, f, tx, ty, W: int, H: int, pitch: int, lam: float,
                   u_min: float, u_max: float, out, stream_handle: int = 0,
                   data_term: int = 0) -> int:
    """Gap of caller-provided device planes (torch CUDA tensors) into `out`
    (a CUDA float64 tensor of 2 elements); allocates no device memory.  Returns the
    library's code.  Raises ValueError before calling the library when a plane is not
    a contiguous CUDA float32 tensor of at least pitch*H elements on out's device, or
    `out` is not a contiguous CUDA float64 tensor of at least 2 elements."""
    import torch
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.numel() >= 2):
        raise ValueError("out must be a contiguous CUDA float64 tensor of >= 2 elements")
    need = int(pitch) * int(H)
    for a in (u, p1, p2, p3, f, tx, ty):
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32
                and a.is_contiguous() and a.device == out.device and a.numel() >= need):
            raise ValueError(f"each plane must be a contiguous CUDA float32 tensor of >= "
                             f"pitch*H = {need} elements on {out.device}")
    ptrs = [a.data_ptr() for a in (u, p1, p2, p3, f, tx, ty)]
    return _lib.evr_gap_static(*ptrs, int(W), int(H), int(pitch), float(lam), float(u_min),
                               float(u_max), int(data_term), out.data_ptr(),
                               ctypes.c_void_p(int(stream_handle)))


def evr_measure_peak(level: int, stream_handle: int = 0) -> float:
    """Measured GB/s of memory level `level` (0 L2, 1 shared memory, all SMs)."""
    g = ctypes.c_double()
    _check(_lib.evr_measure_peak(int(level), ctypes.byref(g), ctypes.c_void_p(int(stream_handle))),
           "evr_measure_peak")
    return g.value


def evr_synchronize(h) -> int:
    rc = _lib.evr_synchronize(h)
    if rc == EVR_ERR_CUDA:
        _check(rc, "evr_synchronize")
    return rc


def evr_enable_kernel_timing(h, enable: bool) -> None:
    _check(_lib.evr_enable_kernel_timing(h, 1 if enable else 0), "evr_enable_kernel_timing")


def evr_kernel_time(h):
    ms, la, pi = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.evr_kernel_time(h, ctypes.byref(ms), ctypes.byref(la), ctypes.byref(pi)),
           "evr_kernel_time")
    return ms.value, la.value, pi.value


def evr_solver_name(h) -> str:
    return _lib.evr_solver_name(h).decode()


def evr_solver_settled(h) -> bool:
    rc = _lib.evr_solver_settled(h)
    if rc < 0:
        _check(rc, "evr_solver_settled")
    return rc == 1


def evr_unrolled_timing_start() -> None:
    _check(_lib.evr_unrolled_timing_start(), "evr_unrolled_timing_start")


def evr_unrolled_timing_stop():
    """(reverse-pass ms, reverse-pass launches, their pixel-iterations, their pixels x
    launches, all launches of the differentiation calls) since the start."""
    ms = ctypes.c_double()
    n, pi, pl, la = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.evr_unrolled_timing_stop(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(pi),
                                         ctypes.byref(pl), ctypes.byref(la)),
           "evr_unrolled_timing_stop")
    return ms.value, n.value, pi.value, pl.value, la.value


class Stream:
    """Owning wrapper of one evr_stream handle for a W x H sensor."""

    def __init__(self, W: int, H: int, params: evr_params | None = None, **overrides):
        p = params or evr_default_params()
        for k, v in overrides.items():
            setattr(p, "lambda_" if k == "lam" else k, v)
        self.W, self.H, self.params = int(W), int(H), p
        self.h = evr_create(W, H, p)

    def close(self):
        if getattr(self, "h", None):
            evr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, x, y, t, pol) -> int:
        return evr_push_events(self.h, x, y, t, pol)

    def push_device(self, x, y, t, pol) -> int:
        return evr_push_events_device(self.h, x, y, t, pol)

    def solve(self, iters: int) -> None:
        evr_solve(self.h, iters)

    def image(self) -> np.ndarray:
        out = np.empty((self.H, self.W), np.float32)
        rc = evr_get_image(self.h, out)
        if rc:
            raise EvrError(rc, "pending device-side rejection")
        return out

    def state(self, which: int):
        v, rc = evr_get_state(self.h, which, self.W, self.H)
        return v

    def p(self) -> np.ndarray:
        return np.stack([self.state(EVR_STATE_P1), self.state(EVR_STATE_P2),
                         self.state(EVR_STATE_P3)])

    def gap(self):
        return evr_gap(self.h)

    def save(self) -> dict:
        """Checkpoint: every plane needed to resume the stream."""
        return {w: np.copy(self.state(w)) for w in CHECKPOINT_PLANES}

    def load(self, ckpt: dict) -> None:
        """Restore a checkpoint taken with save() from a stream of the same size."""
        for w in CHECKPOINT_PLANES:
            evr_set_state(self.h, w, ckpt[w])

    def synchronize(self) -> int:
        return evr_synchronize(self.h)

    @property
    def solver_name(self) -> str:
        return evr_solver_name(self.h)


class Batch:
    """Owning wrapper of an evr_batch handle: n streams of sizes (W[s], H[s])."""

    def __init__(self, sizes, params: evr_params | None = None, **overrides):
        p = params or evr_default_params()
        for k, v in overrides.items():
            setattr(p, "lambda_" if k == "lam" else k, v)
        self.sizes = [(int(w), int(h)) for w, h in sizes]
        self.n = len(self.sizes)
        self.params = p
        W = (ctypes.c_int * self.n)(*[w for w, _ in self.sizes])
        H = (ctypes.c_int * self.n)(*[h for _, h in self.sizes])
        h = ctypes.c_void_p()
        _check(_lib.evr_batch_create(self.n, W, H, ctypes.byref(p), ctypes.byref(h)),
               "evr_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.evr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_cuda_stream(self, handle) -> None:
        arg = handle if isinstance(handle, ctypes.c_void_p) else ctypes.c_void_p(int(handle))
        _check(_lib.evr_batch_set_cuda_stream(self.h, arg), "evr_batch_set_cuda_stream")

    def set_grouping(self, budget_bytes: int, branches: int = 1) -> None:
        """L2 grouping of a step's work: budget_bytes of pass working set per group
        (0: one group, < 0: autotuned), one to four graph branches."""
        _check(_lib.evr_batch_set_grouping(self.h, int(budget_bytes), int(branches)),
               "evr_batch_set_grouping")

    def set_schedule(self, schedule: int) -> None:
        """EVR_BATCH_SCHEDULE_GRAPH (a graph of launches per step),
        EVR_BATCH_SCHEDULE_PERSISTENT (one persistent launch per step) or
        EVR_BATCH_SCHEDULE_AUTO (the faster, chosen at the next tuning)."""
        _check(_lib.evr_batch_set_schedule(self.h, int(schedule)), "evr_batch_set_schedule")

    @property
    def schedule(self) -> int:
        v = ctypes.c_int()
        _check(_lib.evr_batch_get_schedule(self.h, ctypes.byref(v)), "evr_batch_get_schedule")
        return v.value

    def selftest_persist_timeout(self) -> int:
        """Status of a persistent timing run whose first item waits for a count that is
        never reached (EVR_ERR_TIMEOUT when the bounded waits work)."""
        return _lib.evr_batch_selftest_persist_timeout(self.h)

    def step(self, x, y, t, pol, offsets, iters: int) -> None:
        """Host arrays: all streams' events concatenated; offsets (n+1) int64."""
        x, px = _host(x, np.uint16)
        y, py = _host(y, np.uint16)
        t, pt = _host(t, np.int64)
        p, pp = _host(pol, np.int8)
        o, po = _host(offsets, np.int64)
        if len(o) != self.n + 1:
            raise ValueError("offsets must have n + 1 entries")
        _check(_lib.evr_batch_step(self.h, px, py, pt, pp, po, int(iters)), "evr_batch_step")

    def step_device(self, x, y, t, pol, offsets, iters: int) -> None:
        """torch CUDA tensors; offsets int64 of n + 1 entries on the device."""
        _check(_lib.evr_batch_step_device(self.h, x.data_ptr(), y.data_ptr(), t.data_ptr(),
                                          pol.data_ptr(), offsets.data_ptr(), int(iters)),
               "evr_batch_step_device")

    def image(self, s: int) -> np.ndarray:
        W, H = self.sizes[s]
        out = np.empty((H, W), np.float32)
        _check(_lib.evr_batch_get_image(self.h, int(s), out.ctypes.data, out.size),
               "evr_batch_get_image")
        return out

    def images(self, out: np.ndarray | None = None) -> np.ndarray:
        """All images concatenated (float32, sum of W*H)."""
        n = sum(w * h for w, h in self.sizes)
        if out is None:
            out = np.empty(n, np.float32)
        _check(_lib.evr_batch_get_images(self.h, out.ctypes.data, out.size),
               "evr_batch_get_images")
        return out

    def images_async(self, out: np.ndarray) -> int:
        """Queues the readback of all images into `out` (pinned for an asynchronous
        copy); returns the ticket for wait_images."""
        assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
        t = ctypes.c_uint64(0)
        _check(_lib.evr_batch_get_images_async(self.h, out.ctypes.data, out.size,
                                               ctypes.byref(t)), "evr_batch_get_images_async")
        return int(t.value)

    def wait_images(self, ticket: int) -> None:
        _check(_lib.evr_batch_wait_images(self.h, ctypes.c_uint64(ticket)),
               "evr_batch_wait_images")

    def state(self, s: int, which: int):
        W, H = self.sizes[s]
        if which in (EVR_STATE_CLOCK, EVR_STATE_TINIT):
            out = np.zeros(1, np.int64)
        else:
            out = np.empty((H, W), _STATE_DT[which])
        _check(_lib.evr_batch_get_state(self.h, int(s), int(which), out.ctypes.data, out.nbytes),
               "evr_batch_get_state")
        return out[0] if which in (EVR_STATE_CLOCK, EVR_STATE_TINIT) else out

    def synchronize(self):
        s = ctypes.c_int(-1)
        rc = _lib.evr_batch_synchronize(self.h, ctypes.byref(s))
        if rc == EVR_ERR_CUDA:
            _check(rc, "evr_batch_synchronize")
        return rc, s.value

    def enable_kernel_timing(self, on: bool) -> None:
        _check(_lib.evr_batch_enable_kernel_timing(self.h, 1 if on else 0),
               "evr_batch_enable_kernel_timing")

    def kernel_time(self):
        ms, la, pi = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.evr_batch_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(la),
                                          ctypes.byref(pi)), "evr_batch_kernel_time")
        return ms.value, la.value, pi.value

    @property
    def solver_name(self) -> str:
        return _lib.evr_batch_solver_name(self.h).decode()
