"""The synthetic event generator: well-formed, seeded, independent of threading."""
import numpy as np

from evsim import CONFIGS, make_stream
from evsim.events import make_scene, simulate


def test_stream_is_well_formed_and_seeded():
    cfg = CONFIGS["rects128"].with_events(3000)
    a = make_stream(cfg)
    b = make_stream(cfg)
    assert len(a) == 3000
    for k in ("x", "y", "t", "pol"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.x.dtype == np.uint16 and a.t.dtype == np.int64 and a.pol.dtype == np.int8
    assert np.all(np.diff(a.t) >= 0)
    assert a.x.max() < cfg.W and a.y.max() < cfg.H
    assert set(np.unique(a.pol)) <= {-1, 1}


def test_threads_do_not_change_the_stream():
    sc = make_scene(40, 30, "blobs", 20, 5, speed=200.0, omega=0.5)
    a = simulate(sc, 4000, threads=1, seed=5)
    b = simulate(sc, 4000, threads=5, seed=5)
    for k in ("x", "y", "t", "pol"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))


def test_events_follow_log_intensity():
    """Sum of polarities * C tracks the change of log intensity at each pixel
    (within one threshold, noise-free stream)."""
    sc = make_scene(32, 24, "blobs", 15, 9, speed=150.0)
    s = simulate(sc, 5000, C=0.15, noise=0.0, seed=9)
    t_end = float(s.t[-1])
    L0 = s.log_frame(0.0)
    L1 = s.log_frame(t_end)
    acc = np.zeros((24, 32))
    np.add.at(acc, (s.y.astype(int), s.x.astype(int)), s.pol.astype(float) * 0.15)
    assert np.max(np.abs((L1 - L0) - acc)) <= 0.15 + 0.05
