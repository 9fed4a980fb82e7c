"""Python access to the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is plain C (``evr_oracle.c``), compiled with ``gcc -O2
-ffp-contract=off`` into ``oracle/_build/liborc.so`` and loaded with ctypes.
Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
it; the CUDA library never does, and the two share no code.

Every function mirrors one C entry point; see ``evr_oracle.h`` for the passage
of the paper (Reinbacher, Graber, Pock, BMVC 2016) each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evr_oracle.c")
_HDR = os.path.join(_HERE, "evr_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_OMP_PATH = os.path.join(_OUT_DIR, "liborc_omp.so")  # same source, OpenMP over pixels
_lock = threading.Lock()
_lib = None
_lib_omp = None

ORC_OK = 0
ORC_ERR_INVALID_ARG = -1
ORC_ERR_OUT_OF_RANGE = -2
ORC_ERR_BAD_POLARITY = -3
ORC_ERR_NONMONOTONIC = -4
ORC_ERR_OOM = -5

U, P1, P2, P3, F, TAU, G, TLAST, NPOS, NNEG, TREF, TINIT, TX, TY = range(14)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (gcc, no FMA contraction), or with
    omp=True into liborc_omp.so: the same source with its per-pixel loops spread over the
    host's cores by OpenMP (bit-identical results; used to time the CPU baseline)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    path = _OMP_PATH if omp else _LIB_PATH
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest:
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", "-Wall", "-Wno-unknown-pragmas", *(["-fopenmp"] if omp else []),
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


class _Params(ctypes.Structure):
    _fields_ = [
        ("lambda_", ctypes.c_double),
        ("delta_pos", ctypes.c_double),
        ("delta_neg", ctypes.c_double),
        ("u_min", ctypes.c_double),
        ("u_max", ctypes.c_double),
        ("u_init", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("time_scale", ctypes.c_double),
        ("t_max_us", ctypes.c_int64),
        ("t_init_us", ctypes.c_int64),
        ("t_init_first", ctypes.c_int),
        ("data_mode", ctypes.c_int),
        ("manifold", ctypes.c_int),
        ("data_term", ctypes.c_int),
        ("tvl1_iters", ctypes.c_int),
        ("tvl1_lambda", ctypes.c_double),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _lib_handle(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            lib = ctypes.CDLL(build(omp=omp))
            vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.orc_grad.argtypes = [i, i, _D, _D, _D]
            lib.orc_metric.argtypes = [i, i, _D, _D, _D, _D]
            lib.orc_Lg.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_divg.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_prox_kl.argtypes = [d, d, d, d, d]
            lib.orc_prox_kl.restype = d
            lib.orc_project.argtypes = [d, d, d, d, _D]
            lib.orc_pd_iterations.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D, _D,
                                              i, d, d, d, d, d]
            lib.orc_pd_grad.argtypes = [i, i, _D, _D, _D, _D, _D, _D, i, d, d, d, d, d, _D,
                                        _D, _D, _D, _D]
            lib.orc_energy.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D, _D, d, d, d, _D, _D]
            lib.orc_energy_l2.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D, _D, d, _D, _D]
            lib.orc_prox_l2.argtypes = [d, d, d]
            lib.orc_prox_l2.restype = d
            lib.orc_tvl1.argtypes = [i, i, _D, i, d, _D]
            lib.orc_pd_iterations_dt.argtypes = [i, i, _D, _D, _D, _D, _D, _D, _D, _D,
                                                 i, d, d, d, d, d, i]
            lib.orc_create.argtypes = [i, i, ctypes.POINTER(_Params)]
            lib.orc_create.restype = vp
            lib.orc_destroy.argtypes = [vp]
            lib.orc_push.argtypes = [vp, vp, vp, vp, vp, ctypes.c_size_t]
            lib.orc_solve.argtypes = [vp, i]
            lib.orc_get.argtypes = [vp, i, vp]
            lib.orc_set.argtypes = [vp, i, vp]
            lib.orc_stream_energy.argtypes = [vp, _D, _D]
            if omp:
                _lib_omp = lib
            else:
                _lib = lib
        return _lib_omp if omp else _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- operators
def grad(a: np.ndarray):
    """Forward differences (L_x a, L_y a) with zero last column / row."""
    a = _f64(a)
    H, W = a.shape
    ax, ay = np.empty_like(a), np.empty_like(a)
    _lib_handle().orc_grad(W, H, _dp(a), _dp(ax), _dp(ay))
    return ax, ay


def metric(t: np.ndarray):
    """(t_x, t_y, G) of the surface t (Eq. 2)."""
    t = _f64(t)
    H, W = t.shape
    tx, ty, G = np.empty_like(t), np.empty_like(t), np.empty_like(t)
    _lib_handle().orc_metric(W, H, _dp(t), _dp(tx), _dp(ty), _dp(G))
    return tx, ty, G


def Lg(tx, ty, G, u):
    """L_g u as an array of shape (3, H, W) (Eq. 3)."""
    tx, ty, G, u = (_f64(a) for a in (tx, ty, G, u))
    H, W = u.shape
    out = np.empty((3, H, W))
    _lib_handle().orc_Lg(W, H, _dp(tx), _dp(ty), _dp(G), _dp(u),
                         _dp(out[0]), _dp(out[1]), _dp(out[2]))
    return out


def divg(tx, ty, G, p):
    """div_g p = -L_g^* p for p of shape (3, H, W)."""
    tx, ty, G = (_f64(a) for a in (tx, ty, G))
    p = _f64(p)
    H, W = tx.shape
    out = np.empty((H, W))
    _lib_handle().orc_divg(W, H, _dp(tx), _dp(ty), _dp(G), _dp(p[0]), _dp(p[1]), _dp(p[2]),
                           _dp(out))
    return out


def prox_kl(v, beta, f, u_min, u_max) -> float:
    return _lib_handle().orc_prox_kl(float(v), float(beta), float(f), float(u_min), float(u_max))


def project(p3, sqrtG):
    out = np.empty(3)
    _lib_handle().orc_project(float(p3[0]), float(p3[1]), float(p3[2]), float(sqrtG), _dp(out))
    return out


def pd_iterations(tx, ty, G, f, u, p, K, tau, sigma, lam, u_min, u_max):
    """K primal-dual iterations from (u, p); returns new (u, p) copies."""
    tx, ty, G, f = (_f64(a) for a in (tx, ty, G, f))
    u = _f64(u).copy()
    p = _f64(p).copy()
    H, W = u.shape
    _lib_handle().orc_pd_iterations(W, H, _dp(tx), _dp(ty), _dp(G), _dp(f), _dp(u),
                                    _dp(p[0]), _dp(p[1]), _dp(p[2]), int(K), float(tau),
                                    float(sigma), float(lam), float(u_min), float(u_max))
    return u, p


def pd_grad(tx, ty, G, f, u0, p0, K, tau, sigma, lam, u_min, u_max, gu_K):
    """Reverse-mode derivative of pd_iterations for dL/du_K = gu_K:
    returns (dL/du0, dL/dp0 (3,H,W), dL/df, dL/dlambda)."""
    tx, ty, G, f, u0, gu_K = (_f64(a) for a in (tx, ty, G, f, u0, gu_K))
    p0 = _f64(p0)
    H, W = u0.shape
    gu0, gp0, gf = np.empty_like(u0), np.empty((3, H, W)), np.empty_like(u0)
    gl = ctypes.c_double()
    _lib_handle().orc_pd_grad(W, H, _dp(tx), _dp(ty), _dp(G), _dp(f), _dp(u0), _dp(p0), int(K),
                              float(tau), float(sigma), float(lam), float(u_min), float(u_max),
                              _dp(gu_K), _dp(gu0), _dp(gp0), _dp(gf), ctypes.byref(gl))
    return gu0, gp0, gf, gl.value


def prox_l2(v, beta, f) -> float:
    return _lib_handle().orc_prox_l2(float(v), float(beta), float(f))


def tvl1(t0, K, lam):
    """Anisotropic TV-L1 denoising of a surface, K iterations."""
    t0 = _f64(t0)
    H, W = t0.shape
    out = np.empty_like(t0)
    _lib_handle().orc_tvl1(W, H, _dp(t0), int(K), float(lam), _dp(out))
    return out


def pd_iterations_dt(tx, ty, G, f, u, p, K, tau, sigma, lam, u_min, u_max, data_term):
    tx, ty, G, f = (_f64(a) for a in (tx, ty, G, f))
    u = _f64(u).copy()
    p = _f64(p).copy()
    H, W = u.shape
    _lib_handle().orc_pd_iterations_dt(W, H, _dp(tx), _dp(ty), _dp(G), _dp(f), _dp(u),
                                       _dp(p[0]), _dp(p[1]), _dp(p[2]), int(K), float(tau),
                                       float(sigma), float(lam), float(u_min), float(u_max),
                                       int(data_term))
    return u, p


def energy_l2(tx, ty, G, f, u, p, lam):
    tx, ty, G, f, u = (_f64(a) for a in (tx, ty, G, f, u))
    p = _f64(p)
    H, W = u.shape
    pr, du = ctypes.c_double(), ctypes.c_double()
    _lib_handle().orc_energy_l2(W, H, _dp(tx), _dp(ty), _dp(G), _dp(f), _dp(u), _dp(p[0]),
                                _dp(p[1]), _dp(p[2]), float(lam), ctypes.byref(pr),
                                ctypes.byref(du))
    return pr.value, du.value


def energy(tx, ty, G, f, u, p, lam, u_min, u_max):
    """(primal energy of Eq. 5, dual value) at (u, p)."""
    tx, ty, G, f, u = (_f64(a) for a in (tx, ty, G, f, u))
    p = _f64(p)
    H, W = u.shape
    pr, du = ctypes.c_double(), ctypes.c_double()
    _lib_handle().orc_energy(W, H, _dp(tx), _dp(ty), _dp(G), _dp(f), _dp(u), _dp(p[0]),
                             _dp(p[1]), _dp(p[2]), float(lam), float(u_min), float(u_max),
                             ctypes.byref(pr), ctypes.byref(du))
    return pr.value, du.value


# ---------------------------------------------------------------- stream
@dataclass
class OracleParams:
    """Parameters of the model; defaults are the readings used throughout."""
    lam: float = 90.0
    delta_pos: float = 0.15
    delta_neg: float = 0.15
    u_min: float = float(np.exp(-3.0))
    u_max: float = float(np.exp(3.0))
    u_init: float = 1.0
    tau: float = float(1.0 / np.sqrt(8.0 + 4.0 * np.sqrt(2.0)))
    sigma: float = float(1.0 / np.sqrt(8.0 + 4.0 * np.sqrt(2.0)))
    time_scale: float = 1e-3
    t_max_us: int = 100000
    t_init_us: int | None = None  # None: never-fired pixels take the first timestamp
    data_mode: int = 0
    manifold: int = 1
    data_term: int = 0       # 0 KL with box, 1 L2 (Eq. 7)
    tvl1_iters: int = 0      # TV-L1 iterations on the time surface (0 = off)
    tvl1_lambda: float = 1.0

    def _c(self) -> _Params:
        return _Params(self.lam, self.delta_pos, self.delta_neg, self.u_min, self.u_max,
                       self.u_init, self.tau, self.sigma, self.time_scale,
                       int(self.t_max_us), int(self.t_init_us or 0),
                       1 if self.t_init_us is None else 0, int(self.data_mode),
                       int(self.manifold), int(self.data_term), int(self.tvl1_iters),
                       float(self.tvl1_lambda))


class OracleStream:
    """One event stream of a W x H sensor, solved by the FP64 oracle."""

    def __init__(self, W: int, H: int, params: OracleParams | None = None, omp: bool = False):
        """omp=True: the OpenMP build (same results, the host's cores; CPU baseline)."""
        self.W, self.H = int(W), int(H)
        self.params = params or OracleParams()
        self._c_params = self.params._c()
        self._lib = lib = _lib_handle(omp)
        self._h = lib.orc_create(self.W, self.H, ctypes.byref(self._c_params))
        if not self._h:
            raise ValueError("oracle rejected the sensor size or parameters")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    __del__ = close

    def push(self, x, y, t, pol) -> int:
        x = np.ascontiguousarray(x, dtype=np.uint16)
        y = np.ascontiguousarray(y, dtype=np.uint16)
        t = np.ascontiguousarray(t, dtype=np.int64)
        pol = np.ascontiguousarray(pol, dtype=np.int8)
        n = len(x)
        if not (len(y) == len(t) == len(pol) == n):
            raise ValueError("event arrays differ in length")
        return self._lib.orc_push(self._h, x.ctypes.data, y.ctypes.data, t.ctypes.data,
                                      pol.ctypes.data, n)

    def solve(self, K: int) -> int:
        return self._lib.orc_solve(self._h, int(K))

    _DT = {U: np.float64, P1: np.float64, P2: np.float64, P3: np.float64, F: np.float64,
           TAU: np.float64, G: np.float64, TX: np.float64, TY: np.float64,
           TLAST: np.int64, NPOS: np.int32, NNEG: np.int32}

    def get(self, which: int) -> np.ndarray:
        if which in (TREF, TINIT):
            out = np.zeros(1, dtype=np.int64)
        else:
            out = np.empty((self.H, self.W), dtype=self._DT[which])
        rc = self._lib.orc_get(self._h, which, out.ctypes.data)
        if rc:
            raise ValueError(f"orc_get({which}) -> {rc}")
        return out[0] if which in (TREF, TINIT) else out

    def set(self, which: int, value) -> None:
        if which in (TREF, TINIT):
            arr = np.array([value], dtype=np.int64)
        else:
            arr = np.ascontiguousarray(value, dtype=self._DT[which]).reshape(self.H, self.W)
        rc = self._lib.orc_set(self._h, which, arr.ctypes.data)
        if rc:
            raise ValueError(f"orc_set({which}) -> {rc}")

    @property
    def u(self) -> np.ndarray:
        return self.get(U)

    @property
    def p(self) -> np.ndarray:
        return np.stack([self.get(P1), self.get(P2), self.get(P3)])

    def set_up(self, u, p) -> None:
        self.set(U, u)
        for k, w in enumerate((P1, P2, P3)):
            self.set(w, p[k])

    def energy(self):
        pr, du = ctypes.c_double(), ctypes.c_double()
        self._lib.orc_stream_energy(self._h, ctypes.byref(pr), ctypes.byref(du))
        return pr.value, du.value
