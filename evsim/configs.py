"""Named synthetic workloads shaped like the paper's DVS128 experiments.

Each configuration fixes the sensor size, scene, event count, packet size and
iterations per packet.  The scenes stand in for the paper's recorded DVS
sequences, which are not available: 1 microsecond integer timestamps, packets of
a few hundred to a few thousand events, and event rates of the order of the
paper's ~5e5 events/s natural scenes.
"""
from __future__ import annotations

from dataclasses import dataclass

from .events import EventStream, make_scene, simulate


@dataclass(frozen=True)
class StreamConfig:
    name: str
    W: int
    H: int
    kind: str             # 'rects' or 'blobs'
    n_objects: int
    seed: int
    n_events: int
    packet: int           # events per packet
    iters: int            # primal-dual iterations per packet
    speed: float = 0.0    # px/s
    omega: float = 0.0    # rad/s
    noise: float = 0.01
    C: float = 0.15
    layers: int = 1
    speed_disc: bool = False
    dt_us: float = 100.0  # simulation step of the sensor model

    @property
    def n_packets(self) -> int:
        return (self.n_events + self.packet - 1) // self.packet

    def with_events(self, n_events: int) -> "StreamConfig":
        d = dict(self.__dict__)
        d["n_events"] = int(n_events)
        return StreamConfig(**d)


CONFIGS = {
    # 128x128, 30 rectangles translating at 40 px/s, 20k events, 500 per packet, 50 it
    "rects128": StreamConfig("rects128", 128, 128, "rects", 30, 1001, 20_000, 500, 50,
                             speed=40.0, noise=0.01),
    # 346x260, 200 Gaussian blobs, 1 rad/s rotation + 100 px/s, 1M events, 1000 per packet
    "blobs346": StreamConfig("blobs346", 346, 260, "blobs", 200, 1002, 1_000_000, 1000, 50,
                             speed=100.0, omega=1.0, noise=0.02, dt_us=250.0),
    # 1280x720, 1000 blobs in 8 layers with velocities in a 500 px/s disc, mild rotation
    "blobs1280": StreamConfig("blobs1280", 1280, 720, "blobs", 1000, 1004, 10_000_000, 5000,
                              100, speed=500.0, omega=0.2, noise=0.02, layers=8,
                              speed_disc=True, dt_us=400.0),
}


def make_stream(cfg: StreamConfig) -> EventStream:
    """Render the configuration's scene and simulate its event stream."""
    scene = make_scene(cfg.W, cfg.H, cfg.kind, cfg.n_objects, cfg.seed, speed=cfg.speed,
                       omega=cfg.omega, layers=cfg.layers, speed_disc=cfg.speed_disc)
    return simulate(scene, cfg.n_events, C=cfg.C, noise=cfg.noise, seed=cfg.seed,
                    dt_us=cfg.dt_us)


# Batched workload: 256 independent streams of mixed sensor sizes (96 at 128x128,
# 96 at 240x180, 64 at 346x260), each a seeded rectangles or blobs scene (alternating),
# with a packet count drawn uniformly in [20, 400]; 500-event packets, 50 iterations.
BATCH_SIZES = [(128, 128)] * 96 + [(240, 180)] * 96 + [(346, 260)] * 64


def batch_configs(n_streams: int = 256, seed_base: int = 3000, packet: int = 500,
                  iters: int = 50, counts_lo: int = 20, counts_hi: int = 400):
    """Per-stream StreamConfig (with the full packet count) of the batched workload."""
    import numpy as np
    sizes = (BATCH_SIZES * ((n_streams + 255) // 256))[:n_streams]
    rng = np.random.default_rng(seed_base)
    counts = rng.integers(counts_lo, counts_hi + 1, n_streams)
    out = []
    for s, ((W, H), cnt) in enumerate(zip(sizes, counts)):
        area = W * H
        if s % 2 == 0:
            cfg = StreamConfig(f"batch{s}", W, H, "rects", max(4, round(30 * area / 16384)),
                               seed_base + s, int(cnt) * packet, packet, iters, speed=40.0,
                               noise=0.01, dt_us=400.0)
        else:
            cfg = StreamConfig(f"batch{s}", W, H, "blobs", max(8, round(200 * area / 89960)),
                               seed_base + s, int(cnt) * packet, packet, iters, speed=100.0,
                               omega=1.0, noise=0.02, dt_us=250.0)
        out.append(cfg)
    return out


def make_batch(cfgs, max_packets: int | None = None, workers: int | None = None):
    """Simulate every stream of a batch (at most max_packets packets each), in parallel
    over streams.  Returns the list of EventStreams."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    def one(cfg):
        n = cfg.n_events if max_packets is None else min(cfg.n_events, max_packets * cfg.packet)
        scene = make_scene(cfg.W, cfg.H, cfg.kind, cfg.n_objects, cfg.seed, speed=cfg.speed,
                           omega=cfg.omega, layers=cfg.layers, speed_disc=cfg.speed_disc)
        return simulate(scene, n, C=cfg.C, noise=cfg.noise, seed=cfg.seed, dt_us=cfg.dt_us,
                        threads=1)

    with ThreadPoolExecutor(max_workers=workers or min(32, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, cfgs))


def batch_step_arrays(streams, packet: int, step: int, t_shift=None):
    """Concatenated events of packet `step` of every stream (empty for streams that
    have run out) and the (n + 1) offsets."""
    import numpy as np
    xs, ys, ts, ps, offs = [], [], [], [], [0]
    for st in streams:
        a = step * packet
        b = min(a + packet, len(st))
        if a >= len(st):
            b = a = 0
        xs.append(st.x[a:b])
        ys.append(st.y[a:b])
        ts.append(st.t[a:b])
        ps.append(st.pol[a:b])
        offs.append(offs[-1] + (b - a))
    return (np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(ps),
            np.array(offs, dtype=np.int64))
