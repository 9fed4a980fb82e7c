"""Scene rendering and event emission for synthetic event-camera streams.

Scene model: a log-intensity texture on a toroidal domain twice the sensor size
in each direction, split into one or more layers.  Each layer moves rigidly
(translation, plus a rotation about the sensor centre) and the sensor sees the
sum of the layers, sampled bilinearly at each pixel centre.

Sensor model (the idealised event camera of the paper's Sec. 3): every pixel
keeps a reference level, initialised to its first log intensity.  The scene is
sampled every ``dt_us`` microseconds (steps are subdivided when some pixel
moves by more than C in one step).  Whenever ``L - ref >= C`` the pixel emits a
+1 event and ``ref += C`` (symmetrically -1 events for ``ref - L >= C``); the
event time is interpolated linearly inside the step and floored to whole
microseconds.  A fraction ``noise`` of all events is replaced by uniform noise
(uniform pixel, uniform time, polarity +-1 with probability 1/2).  The merged
stream is stably sorted by (t, y, x, polarity).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np


@dataclass
class EventStream:
    """Structure-of-arrays event stream of a W x H sensor (x = column, y = row)."""
    W: int
    H: int
    x: np.ndarray    # uint16[n]
    y: np.ndarray    # uint16[n]
    t: np.ndarray    # int64[n], microseconds, non-decreasing
    pol: np.ndarray  # int8[n], +1 / -1
    scene: "Scene | None" = field(default=None, repr=False)

    def __len__(self) -> int:
        return int(self.x.shape[0])

    def slice(self, a: int, b: int) -> "EventStream":
        return EventStream(self.W, self.H, self.x[a:b], self.y[a:b], self.t[a:b],
                           self.pol[a:b], self.scene)

    def log_frame(self, t_us: float) -> np.ndarray:
        """Ground-truth log intensity seen by the sensor at time t_us (H x W)."""
        return _CScene(self.scene).sample(t_us).reshape(self.H, self.W)


def packets(stream: EventStream, size: int):
    """Yield consecutive packets of ``size`` events (the last one may be shorter)."""
    for a in range(0, len(stream), size):
        yield stream.slice(a, min(a + size, len(stream)))


# ----------------------------------------------------------------- textures
def _render_rects(rng, DW, DH, n, side_lo, side_hi, ss=4):
    """Axis-aligned rectangles with uniform log values on a uniform background,
    painter's order, toroidal domain, box-filtered from an ss x ss supersample."""
    Sw, Sh = DW * ss, DH * ss
    img = np.full((Sh, Sw), rng.uniform(0.0, 1.0), dtype=np.float64)
    for _ in range(n):
        w = rng.uniform(side_lo, side_hi)
        h = rng.uniform(side_lo, side_hi)
        x0 = rng.uniform(0, DW)
        y0 = rng.uniform(0, DH)
        val = rng.uniform(0.0, 1.0)
        xs = (np.arange(int(round(x0 * ss)), int(round((x0 + w) * ss)))) % Sw
        ys = (np.arange(int(round(y0 * ss)), int(round((y0 + h) * ss)))) % Sh
        img[np.ix_(ys, xs)] = val
    return img.reshape(DH, ss, DW, ss).mean(axis=(1, 3))


def _render_blobs(rng, DW, DH, n, sig_lo, sig_hi, amp_sd):
    """Sum of isotropic Gaussian blobs (sigma U[sig_lo, sig_hi] px, log amplitude
    N(0, amp_sd)) on a toroidal domain, evaluated at texel centres."""
    img = np.zeros((DH, DW), dtype=np.float64)
    for _ in range(n):
        s = rng.uniform(sig_lo, sig_hi)
        a = rng.normal(0.0, amp_sd)
        cx = rng.uniform(0, DW)
        cy = rng.uniform(0, DH)
        r = int(np.ceil(4.0 * s))
        xs = np.arange(int(np.floor(cx)) - r, int(np.floor(cx)) + r + 2)
        ys = np.arange(int(np.floor(cy)) - r, int(np.floor(cy)) + r + 2)
        gx = np.exp(-0.5 * ((xs + 0.5 - cx) / s) ** 2)
        gy = np.exp(-0.5 * ((ys + 0.5 - cy) / s) ** 2)
        np.add.at(img, (ys[:, None] % DH, xs[None, :] % DW), a * gy[:, None] * gx[None, :])
    return img


@dataclass
class Layer:
    tex: np.ndarray        # (DH, DW) log intensity
    vel: tuple             # px/s (vx, vy)
    omega: float           # rad/s about the sensor centre


class Scene:
    """Sum of rigidly moving toroidal texture layers seen by a W x H sensor."""

    def __init__(self, W: int, H: int, layers: list):
        self.W, self.H = W, H
        self.layers = layers
        yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
        self._px = (xx + 0.5 - W / 2.0).ravel()
        self._py = (yy + 0.5 - H / 2.0).ravel()
        # wrap-padded copies (one extra row and column) for branch-free bilinear taps
        self._padded = [np.pad(L.tex, ((0, 1), (0, 1)), mode="wrap").ravel() for L in layers]

    def sample(self, t_us: float) -> np.ndarray:
        ts = float(t_us) * 1e-6
        out = np.zeros(self.W * self.H)
        for L, Tp in zip(self.layers, self._padded):
            DH, DW = L.tex.shape
            th = L.omega * ts
            c, s = np.cos(th), np.sin(th)
            qx = c * self._px - s * self._py
            qx += self.W / 2.0 + L.vel[0] * ts - 0.5
            qx -= DW * np.floor(qx * (1.0 / DW))
            qy = s * self._px + c * self._py
            qy += self.H / 2.0 + L.vel[1] * ts - 0.5
            qy -= DH * np.floor(qy * (1.0 / DH))
            fx = qx.astype(np.int64)
            fy = qy.astype(np.int64)
            np.minimum(fx, DW - 1, out=fx)
            np.minimum(fy, DH - 1, out=fy)
            ax = qx - fx
            ay = qy - fy
            i00 = fy * (DW + 1) + fx
            t0 = Tp[i00]
            t0 += ax * (Tp[i00 + 1] - t0)
            i00 += DW + 1
            t1 = Tp[i00]
            t1 += ax * (Tp[i00 + 1] - t1)
            t0 += ay * (t1 - t0)
            out += t0
        return out.reshape(self.H, self.W)


def make_scene(W, H, kind, n_objects, seed, speed=0.0, omega=0.0, layers=1,
               speed_disc=False):
    """Build a seeded scene.  ``kind`` is 'rects' or 'blobs'.  With ``layers`` > 1
    the objects are split into that many layers, each with its own velocity
    (uniform in a disc of radius ``speed`` when ``speed_disc``)."""
    rng = np.random.default_rng(seed)
    DW, DH = 2 * W, 2 * H
    per = [n_objects // layers + (1 if i < n_objects % layers else 0) for i in range(layers)]
    out = []
    for li in range(layers):
        if kind == "rects":
            tex = _render_rects(rng, DW, DH, per[li], 8.0, 48.0)
            if li > 0:
                tex = tex - tex.mean()
        elif kind == "blobs":
            tex = _render_blobs(rng, DW, DH, per[li], 3.0, 20.0, 0.3)
        else:
            raise ValueError(kind)
        if speed_disc:
            r = speed * np.sqrt(rng.uniform())
            a = rng.uniform(0, 2 * np.pi)
        else:
            r = speed
            a = rng.uniform(0, 2 * np.pi)
        out.append(Layer(tex, (r * np.cos(a), r * np.sin(a)), omega))
    return Scene(W, H, out)


# ------------------------------------------------------------------- events
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "_sim.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libevsim.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the simulator's inner loop (gcc) into evsim/_build/libevsim.so."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
            lib.evsim_sample.argtypes = [i, i, i, vp, vp, vp, vp, vp, vp, d, vp]
            lib.evsim_run.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp, vp, d, d, d, i64, i,
                                      vp, vp, vp, vp, vp, vp, vp]
            lib.evsim_run.restype = i64
            _lib = lib
        return _lib


class _CScene:
    """ctypes view of a Scene's layers (keeps the arrays alive)."""

    def __init__(self, scene: Scene):
        self.scene = scene
        nl = len(scene.layers)
        self.tex = [np.ascontiguousarray(p, dtype=np.float64) for p in scene._padded]
        self.ptrs = (ctypes.c_void_p * nl)(*[t.ctypes.data for t in self.tex])
        self.DW = np.array([L.tex.shape[1] for L in scene.layers], dtype=np.int32)
        self.DH = np.array([L.tex.shape[0] for L in scene.layers], dtype=np.int32)
        self.vx = np.array([L.vel[0] for L in scene.layers], dtype=np.float64)
        self.vy = np.array([L.vel[1] for L in scene.layers], dtype=np.float64)
        self.om = np.array([L.omega for L in scene.layers], dtype=np.float64)
        self.nl = nl

    def args(self):
        return (self.nl, ctypes.cast(self.ptrs, ctypes.c_void_p), self.DW.ctypes.data,
                self.DH.ctypes.data, self.vx.ctypes.data, self.vy.ctypes.data,
                self.om.ctypes.data)

    def sample(self, t_us: float) -> np.ndarray:
        out = np.empty(self.scene.W * self.scene.H)
        _handle().evsim_sample(self.scene.W, self.scene.H, *self.args(), float(t_us),
                               out.ctypes.data)
        return out


def _band_worker(args):
    (lib, W, H, y0, y1, cs_args, C, dt_us, t_stop, ref, L_prev, t_state, max_per_px) = args
    out = []
    while t_state.value + dt_us <= t_stop:
        cap = max(1 << 16, 4 * (y1 - y0) * W * max_per_px)
        bx = np.empty(cap, np.uint16)
        by = np.empty(cap, np.uint16)
        bt = np.empty(cap, np.int64)
        bp = np.empty(cap, np.int8)
        got = lib.evsim_run(W, H, y0, y1, *cs_args, float(C), float(dt_us), float(t_stop), cap,
                            max_per_px, ref.ctypes.data, L_prev.ctypes.data,
                            ctypes.byref(t_state), bx.ctypes.data, by.ctypes.data,
                            bt.ctypes.data, bp.ctypes.data)
        if got < 0:
            raise RuntimeError("scene moves too fast for the simulation step")
        out.append((bx[:got].copy(), by[:got].copy(), bt[:got].copy(), bp[:got].copy()))
    return out


def simulate(scene: Scene, n_events: int, C: float = 0.15, noise: float = 0.01,
             seed: int = 0, dt_us: float = 100.0, t0_us: int = 0,
             threads: int | None = None) -> EventStream:
    """Emit ``n_events`` events from ``scene`` with contrast threshold C.

    The sensor rows are simulated in parallel bands up to a growing time horizon
    until enough signal events exist; the result does not depend on the number
    of bands.  Signal events are cut at the time of the
    ``ceil(n_events * (1 - noise))``-th one, noise events are drawn uniformly up
    to that time, and the first n_events of the sorted merge are returned."""
    W, H = scene.W, scene.H
    rng = np.random.default_rng(seed + 7919)
    cs = _CScene(scene)
    lib = _handle()
    n_signal = int(np.ceil(n_events * (1.0 - noise)))
    ref = cs.sample(0.0)
    L_prev = ref.copy()
    threads = threads or min(16, os.cpu_count() or 1)
    nb = max(1, min(threads, H))
    edges = [H * k // nb for k in range(nb + 1)]
    bands = [(edges[k], edges[k + 1]) for k in range(nb) if edges[k + 1] > edges[k]]
    t_states = [ctypes.c_double(0.0) for _ in bands]
    chunks = []
    count = 0
    horizon = 64 * dt_us
    max_per_px = 8
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=len(bands)) as ex:
        while count < n_signal:
            if horizon > 3.6e9:
                raise RuntimeError("scene produces too few events")
            jobs = [(lib, W, H, y0, y1, cs.args(), C, dt_us, horizon, ref, L_prev, ts,
                     max_per_px) for (y0, y1), ts in zip(bands, t_states)]
            for res in ex.map(_band_worker, jobs):
                for c in res:
                    chunks.append(c)
                    count += c[0].size
            if count < n_signal:
                # grow the horizon towards the expected end, at least by half
                rate = count / horizon if count else 0.0
                need = (n_signal - count) / rate if rate > 0 else horizon
                horizon = horizon + min(max(0.25 * horizon, 1.1 * need), 2.0 * horizon)
                horizon = dt_us * np.ceil(horizon / dt_us)
    x = np.concatenate([c[0] for c in chunks])
    y = np.concatenate([c[1] for c in chunks])
    t = np.concatenate([c[2] for c in chunks])
    p = np.concatenate([c[3] for c in chunks])
    order = np.lexsort((p, x, y, t))
    x, y, t, p = x[order][:n_signal], y[order][:n_signal], t[order][:n_signal], p[order][:n_signal]
    t_cut = int(t[-1]) if t.size else 0
    n_noise = int(round(noise / max(1e-12, 1.0 - noise) * x.size))
    if n_noise:
        nx = rng.integers(0, W, n_noise).astype(np.uint16)
        ny = rng.integers(0, H, n_noise).astype(np.uint16)
        nt = rng.integers(0, t_cut + 1, n_noise).astype(np.int64)
        npol = rng.choice(np.array([-1, 1], dtype=np.int8), n_noise)
        x = np.concatenate([x, nx])
        y = np.concatenate([y, ny])
        t = np.concatenate([t, nt])
        p = np.concatenate([p, npol])
        order = np.lexsort((p, x, y, t))
        x, y, t, p = x[order], y[order], t[order], p[order]
    n = min(n_events, x.size)
    return EventStream(W, H, np.ascontiguousarray(x[:n]), np.ascontiguousarray(y[:n]),
                       np.ascontiguousarray(t[:n] + t0_us), np.ascontiguousarray(p[:n]),
                       scene)
