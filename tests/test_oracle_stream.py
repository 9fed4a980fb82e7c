"""Pins of the oracle's event integration and per-packet solve.

Event integration is integer work with a plain definition (Sec. 3: events
e = (x, y, theta, t) with increasing t; Sec. 3.1: the surface of active events
holds each pixel's most recent timestamp; Eq. intensity_update: one factor c1 or
c2 per event), so it is compared with a brute-force per-event loop written here.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

P = O.OracleParams()


def brute_integrate(W, H, events, t_init=None):
    """Per-event definition: latest timestamp, polarity counts, stream clock."""
    t_last = {}
    npos = np.zeros((H, W), np.int32)
    nneg = np.zeros((H, W), np.int32)
    clock = t_init
    for (x, y, t, p) in events:
        if clock is None:
            clock = t
            t_init = t
        t_last[(y, x)] = max(t_last.get((y, x), t_init), t)
        if p > 0:
            npos[y, x] += 1
        else:
            nneg[y, x] += 1
        clock = max(clock, t)
    tl = np.full((H, W), t_init if t_init is not None else 0, np.int64)
    for (y, x), v in t_last.items():
        tl[y, x] = v
    return tl, npos, nneg, clock


def rand_events(rng, W, H, n, t0=1000, dense=False):
    x = rng.integers(0, W if not dense else 2, n).astype(np.uint16)
    y = rng.integers(0, H if not dense else 2, n).astype(np.uint16)
    t = (t0 + np.sort(rng.integers(0, 50 * n + 1, n))).astype(np.int64)
    p = rng.choice(np.array([-1, 1], np.int8), n)
    return x, y, t, p


@pytest.mark.parametrize("W,H,n,dense", [(7, 5, 40, False), (1, 1, 13, False),
                                         (16, 9, 300, True), (3, 1, 10, False)])
def test_integration_matches_per_event_definition(W, H, n, dense):
    rng = np.random.default_rng(W * 100 + H)
    s = O.OracleStream(W, H)
    x, y, t, p = rand_events(rng, W, H, n, dense=dense)
    half = n // 2
    assert s.push(x[:half], y[:half], t[:half], p[:half]) == 0
    assert s.push(x[half:], y[half:], t[half:], p[half:]) == 0
    tl, npos, nneg, clock = brute_integrate(W, H, list(zip(x, y, t, p)))
    np.testing.assert_array_equal(s.get(O.TLAST), tl)
    np.testing.assert_array_equal(s.get(O.NPOS), npos)
    np.testing.assert_array_equal(s.get(O.NNEG), nneg)
    assert s.get(O.TREF) == clock
    assert s.get(O.TINIT) == t[0]


def test_integration_invariant_to_order_of_equal_timestamps():
    rng = np.random.default_rng(5)
    W, H = 6, 6
    x, y, t, p = rand_events(rng, W, H, 200)
    t = (t // 500) * 500  # many equal timestamps
    perm = np.lexsort((rng.random(len(t)), t))  # shuffle inside equal-t groups
    a, b = O.OracleStream(W, H), O.OracleStream(W, H)
    assert a.push(x, y, t, p) == 0
    assert b.push(x[perm], y[perm], t[perm], p[perm]) == 0
    for w in (O.TLAST, O.NPOS, O.NNEG):
        np.testing.assert_array_equal(a.get(w), b.get(w))
    a.solve(7)
    b.solve(7)
    np.testing.assert_array_equal(a.u, b.u)


@pytest.mark.parametrize("bad,code", [("x", O.ORC_ERR_OUT_OF_RANGE), ("y", O.ORC_ERR_OUT_OF_RANGE),
                                      ("pol", O.ORC_ERR_BAD_POLARITY),
                                      ("t", O.ORC_ERR_NONMONOTONIC)])
def test_rejected_packet_leaves_state_unchanged(bad, code):
    rng = np.random.default_rng(6)
    W, H = 8, 5
    s = O.OracleStream(W, H)
    x, y, t, p = rand_events(rng, W, H, 50)
    assert s.push(x[:20], y[:20], t[:20], p[:20]) == 0
    s.solve(3)
    before = {w: s.get(w) for w in (O.TLAST, O.NPOS, O.NNEG, O.U, O.P1, O.TREF)}
    x2, y2, t2, p2 = (a[20:].copy() for a in (x, y, t, p))
    if bad == "x":
        x2[10] = W
    elif bad == "y":
        y2[10] = H
    elif bad == "pol":
        p2[10] = 0
    else:
        t2[10] = t2[9] - 1
    assert s.push(x2, y2, t2, p2) == code
    for w, v in before.items():
        np.testing.assert_array_equal(s.get(w), v)


def test_first_bad_event_decides_the_code_and_clock_is_checked():
    W, H = 4, 4
    s = O.OracleStream(W, H)
    assert s.push([1], [1], [100], [1]) == 0
    # event 0 is earlier than the clock, event 1 is out of range: the first one wins
    assert s.push([1, 9], [1, 1], [99, 200], [1, 1]) == O.ORC_ERR_NONMONOTONIC
    assert s.push([9, 1], [1, 1], [99, 200], [1, 0]) == O.ORC_ERR_OUT_OF_RANGE
    assert s.push([1, 1], [1, 1], [150, 200], [0, 1]) == O.ORC_ERR_BAD_POLARITY
    # equal to the clock is accepted
    assert s.push([2], [2], [100], [-1]) == 0


def test_explicit_t_init_and_empty_push():
    s = O.OracleStream(3, 2, O.OracleParams(t_init_us=500))
    assert s.push([], [], [], []) == 0
    assert s.get(O.TREF) == 500
    assert s.push([0], [0], [499], [1]) == O.ORC_ERR_NONMONOTONIC
    assert s.push([0], [0], [700], [1]) == 0
    tl = s.get(O.TLAST)
    assert tl[0, 0] == 700 and np.all(tl.ravel()[1:] == 500)


def test_data_image_compounds_one_factor_per_event():
    """f = u^{n-1} * c1^{n+} * c2^{n-} = u^{n-1} exp(Delta+ n+ - Delta- n-) (Eq. intensity_update)."""
    rng = np.random.default_rng(7)
    W, H = 9, 7
    prm = O.OracleParams(delta_pos=0.21, delta_neg=0.13)
    s = O.OracleStream(W, H, prm)
    x, y, t, p = rand_events(rng, W, H, 400)
    s.push(x[:200], y[:200], t[:200], p[:200])
    s.solve(5)
    u_prev = s.u
    s.push(x[200:], y[200:], t[200:], p[200:])
    npos, nneg = s.get(O.NPOS), s.get(O.NNEG)
    s.solve(0)
    want = u_prev * np.exp(0.21 * npos - 0.13 * nneg)
    np.testing.assert_allclose(s.get(O.F), want, rtol=1e-13)
    assert np.all(s.get(O.NPOS) == 0) and np.all(s.get(O.NNEG) == 0)
    np.testing.assert_array_equal(s.u, u_prev)  # K = 0 leaves u alone


def test_persistent_data_mode():
    """data_mode 1: f is stepped from its own previous value, starting at u_init."""
    W, H = 4, 3
    s = O.OracleStream(W, H, O.OracleParams(data_mode=1, u_init=2.0))
    s.push([1, 1, 2], [0, 0, 2], [10, 11, 12], [1, 1, -1])
    s.solve(3)
    f1 = s.get(O.F)
    c1, c2 = math.exp(0.15), math.exp(-0.15)
    want = np.full((H, W), 2.0)
    want[0, 1] *= c1 * c1
    want[2, 2] *= c2
    np.testing.assert_allclose(f1, want, rtol=1e-15)
    s.push([1], [0], [20], [-1])
    s.solve(3)
    want[0, 1] *= c2
    np.testing.assert_allclose(s.get(O.F), want, rtol=1e-15)


def test_time_surface_is_scaled_clamped_time_since_last_event():
    prm = O.OracleParams(time_scale=1e-3, t_max_us=40_000)
    s = O.OracleStream(3, 1, prm)
    s.push([0, 1, 2], [0, 0, 0], [1000, 30_000, 101_000], [1, 1, 1])
    s.solve(0)
    np.testing.assert_allclose(s.get(O.TAU)[0], [40.0, 40.0, 0.0], rtol=0, atol=0)
    prm2 = O.OracleParams(time_scale=1e-3, t_max_us=0)
    s2 = O.OracleStream(3, 1, prm2)
    s2.push([0, 1, 2], [0, 0, 0], [1000, 30_000, 101_000], [1, 1, 1])
    s2.solve(0)
    np.testing.assert_allclose(s2.get(O.TAU)[0], [100.0, 71.0, 0.0], rtol=1e-15)


def test_manifold_off_gives_flat_metric():
    prm = O.OracleParams(manifold=0)
    rng = np.random.default_rng(8)
    s = O.OracleStream(6, 6, prm)
    x, y, t, p = rand_events(rng, 6, 6, 60)
    s.push(x, y, t, p)
    s.solve(4)
    assert np.all(s.get(O.G) == 1.0)
    assert np.all(s.get(O.P3) == 0.0)


def test_invalid_parameters_rejected():
    for bad in (dict(lam=0.0), dict(u_min=0.0), dict(u_min=3.0, u_max=2.0), dict(delta_pos=0.0),
                dict(tau=-1.0), dict(data_mode=3)):
        with pytest.raises(ValueError):
            O.OracleStream(4, 4, O.OracleParams(**bad))
    with pytest.raises(ValueError):
        O.OracleStream(0, 4)


def test_openmp_build_is_bit_identical_to_the_serial_oracle():
    """The CPU baseline's OpenMP build (per-pixel loops over the host's cores) computes the
    same bits as the serial oracle: its loops write only their own pixel."""
    import os
    import subprocess
    import sys
    code = r"""
import numpy as np
from evsim import CONFIGS, make_stream
from oracle import oracle as O
cfg = CONFIGS["rects128"].with_events(3000)
st = make_stream(cfg)
outs = []
for omp in (False, True):
    o = O.OracleStream(cfg.W, cfg.H, omp=omp)
    for a in range(0, len(st), cfg.packet):
        s = st.slice(a, a + cfg.packet)
        assert o.push(s.x, s.y, s.t, s.pol) == 0
        o.solve(cfg.iters)
    outs.append((o.u.copy(), o.get(O.P1).copy(), o.get(O.P3).copy()))
for a, b in zip(*outs):
    assert np.array_equal(a, b)
print("identical")
"""
    env = dict(os.environ, OMP_NUM_THREADS="4")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "identical" in r.stdout, r.stderr[-2000:]
