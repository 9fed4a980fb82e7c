"""Batched streams (evr_batch_*) through the C ABI: every stream bit-identical to the
same stream solved alone with the same solver configuration, per-stream validation,
idle streams untouched, and one stream checked against the FP64 oracle."""
import numpy as np
import pytest

from evsim.configs import batch_step_arrays
from evsim.events import EventStream
from oracle import oracle as O

pytestmark = pytest.mark.gpu

SIZES = [(33, 17), (64, 48), (128, 128), (17, 33), (1, 1), (100, 3), (57, 57), (240, 180),
         (3, 100), (80, 64)]
COUNTS = [6, 3, 8, 1, 5, 7, 2, 6, 4, 8]


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import evr
    return evr


@pytest.fixture(scope="module")
def streams():
    """Random packets (uniform pixels, increasing timestamps with repeats, +-1) for
    sensors down to 1 x 1, with uneven packet counts."""
    out = []
    for s, ((W, H), cnt) in enumerate(zip(SIZES, COUNTS)):
        rng = np.random.default_rng(500 + s)
        n = cnt * 300
        x = rng.integers(0, W, n).astype(np.uint16)
        y = rng.integers(0, H, n).astype(np.uint16)
        t = (1000 + np.sort(rng.integers(0, 40 * n, n))).astype(np.int64)
        p = rng.choice(np.array([-1, 1], np.int8), n)
        out.append(EventStream(W, H, x, y, t, p))
    return out


def run_batch(E, streams, tile, steps, iters=30, grouping=None):
    b = E.Batch(SIZES, tile_config=tile)
    if grouping is not None:
        b.set_grouping(*grouping)
    for k in range(steps):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        b.step(x, y, t, p, off, iters)
    return b


def run_solo(E, st, tile, steps, iters=30):
    g = E.Stream(st.W, st.H, solver=2, tile_config=tile)
    for k in range(steps):
        a = k * 300
        if a >= len(st):
            continue
        s = st.slice(a, a + 300)
        assert g.push(s.x, s.y, s.t, s.pol) == 0
        g.solve(iters)
    return g


@pytest.mark.parametrize("tile", [1, 6, 10])
def test_batch_equals_solo_bit_for_bit(E, streams, tile):
    steps = max(COUNTS)
    b = run_batch(E, streams, tile, steps)
    rc, bad = b.synchronize()
    assert rc == 0 and bad == -1
    for s, st in enumerate(streams):
        g = run_solo(E, st, tile, steps)
        for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P2, E.EVR_STATE_P3,
                  E.EVR_STATE_F, E.EVR_STATE_TLAST, E.EVR_STATE_SQRTG):
            np.testing.assert_array_equal(b.state(s, w), g.state(w), err_msg=f"stream {s} {w}")
        assert int(b.state(s, E.EVR_STATE_CLOCK)) == int(g.state(E.EVR_STATE_CLOCK))
        g.close()
    b.close()


@pytest.mark.parametrize("budget,branches", [(1 << 20, 1), (1 << 20, 2), (3 << 20, 2),
                                             (1 << 20, 4)])
def test_l2_groups_equal_one_group_bit_for_bit(E, streams, budget, branches):
    """Streams cut into groups of at most `budget` bytes of pass working set (the 240 x 180
    stream, 2.4 MB, a group of its own), each group's prologue and passes run before the
    next, on one to four graph branches: every stream's state equals the one-group run."""
    steps = max(COUNTS)
    ref = run_batch(E, streams, 6, steps, grouping=(0, 1))
    b = run_batch(E, streams, 6, steps, grouping=(budget, branches))
    assert "L2 groups" in b.solver_name and "L2 groups" not in ref.solver_name
    for g in (ref, b):
        rc, bad = g.synchronize()
        assert rc == 0 and bad == -1
    for s in range(len(SIZES)):
        for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P2, E.EVR_STATE_P3,
                  E.EVR_STATE_F, E.EVR_STATE_TLAST):
            np.testing.assert_array_equal(b.state(s, w), ref.state(s, w),
                                          err_msg=f"stream {s} {w}")
    ref.close()
    b.close()


def test_grouping_rejects_bad_branches(E):
    b = E.Batch(SIZES[:3])
    for br in (0, 5):
        with pytest.raises(E.EvrError):
            b.set_grouping(1 << 20, br)
    b.close()


def test_autotuned_batch_runs_and_matches_oracle(E, streams):
    """Autotuned configuration; stream 2 (128x128) teacher-forced against the oracle on
    its last packet."""
    b = E.Batch(SIZES)
    s_idx = 2
    st = streams[s_idx]
    steps = COUNTS[s_idx]
    p = b.params
    o = O.OracleStream(st.W, st.H, O.OracleParams(
        lam=float(p.lambda_), delta_pos=float(p.delta_pos), delta_neg=float(p.delta_neg),
        u_min=float(p.u_min), u_max=float(p.u_max), u_init=float(p.u_init), tau=float(p.tau),
        sigma=float(p.sigma), time_scale=float(np.float32(p.time_scale))))
    for k in range(steps):
        x, y, t, pol, off = batch_step_arrays(streams, 300, k)
        s = st.slice(k * 300, k * 300 + 300)
        if k == steps - 1:
            o.set_up(b.state(s_idx, E.EVR_STATE_U).astype(np.float64),
                     np.stack([b.state(s_idx, w) for w in (E.EVR_STATE_P1, E.EVR_STATE_P2,
                                                           E.EVR_STATE_P3)]).astype(np.float64))
            o.set(O.TLAST, b.state(s_idx, E.EVR_STATE_TLAST))
            o.set(O.TREF, int(b.state(s_idx, E.EVR_STATE_CLOCK)))
            o.set(O.TINIT, int(b.state(s_idx, E.EVR_STATE_TINIT)))
            assert o.push(s.x, s.y, s.t, s.pol) == 0
            o.solve(30)
        b.step(x, y, t, pol, off, 30)
    assert "batch of 10" in b.solver_name
    d = np.max(np.abs(b.image(s_idx).astype(np.float64) - o.u))
    assert d <= 1e-4, d
    b.close()


def test_rejection_is_per_stream_and_idle_streams_are_untouched(E, streams):
    b = run_batch(E, streams, 1, 2)
    before = [b.state(s, E.EVR_STATE_U).copy() for s in range(len(SIZES))]
    x, y, t, p, off = batch_step_arrays(streams, 300, 2)
    # stream 4 (1x1, still has packets) gets an out-of-range event; stream 1 (3 packets)
    # stays idle this step by removing its events
    a4, b4 = off[4], off[5]
    x = x.copy()
    x[a4] = 1
    keep = np.ones(len(x), bool)
    keep[off[1]:off[2]] = False
    cnt = np.diff(off)
    cnt[1] = 0
    off2 = np.concatenate([[0], np.cumsum(cnt)])
    b.step(x[keep], y[keep], t[keep], p[keep], off2, 30)
    rc, bad = b.synchronize()
    assert rc == E.EVR_ERR_OUT_OF_RANGE and bad == 4
    np.testing.assert_array_equal(b.state(1, E.EVR_STATE_U), before[1])
    assert b.synchronize() == (0, -1)
    b.close()


def test_gathered_and_async_readback_match_per_stream_images(E, streams):
    """evr_batch_get_images (device gather + one copy) and its asynchronous form, driven
    with two steps in flight, give every stream's own image."""
    import torch
    b = E.Batch(SIZES, tile_config=1)
    n_img = sum(w * h for w, h in SIZES)
    bufs = [torch.empty(n_img, dtype=torch.float32).pin_memory().numpy() for _ in range(2)]
    seen, prev = [], None
    for k in range(4):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        b.step(x, y, t, p, off, 30)
        tk = b.images_async(bufs[k % 2])
        if prev is not None:
            b.wait_images(prev[0])
            seen.append(prev[1].copy())
        prev = (tk, bufs[k % 2])
    b.wait_images(prev[0])
    seen.append(prev[1].copy())
    full = b.images()
    np.testing.assert_array_equal(seen[-1], full)
    a = 0
    for s, (W, H) in enumerate(SIZES):
        np.testing.assert_array_equal(full[a:a + W * H].reshape(H, W), b.image(s))
        a += W * H
    # the earlier asynchronous readbacks hold the earlier steps: replay them
    r = E.Batch(SIZES, tile_config=1)
    for k in range(4):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        r.step(x, y, t, p, off, 30)
        np.testing.assert_array_equal(r.images(), seen[k], err_msg=f"step {k}")
    with pytest.raises(E.EvrError):
        b.wait_images(99)
    b.close()
    r.close()
