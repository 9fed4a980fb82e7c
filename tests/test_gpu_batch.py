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


def run_batch(E, streams, tile, steps, iters=30, grouping=None, schedule=None, **kw):
    b = E.Batch(SIZES, tile_config=tile, **kw)
    if grouping is not None:
        b.set_grouping(*grouping)
    if schedule is not None:
        b.set_schedule(schedule)
    for k in range(steps):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        b.step(x, y, t, p, off, iters)
    return b


def run_solo(E, st, tile, steps, iters=30, **kw):
    g = E.Stream(st.W, st.H, solver=2, tile_config=tile, **kw)
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


# ---------------------------------------------------------------- persistent schedule
# tile_config values whose tiles have a persistent form: 32x32 (256 threads) R2, 32x48
# (384 threads) R4, 32x32 (512 threads) R6
PERSIST_TILES = [1, 36, 31]


@pytest.mark.parametrize("tile", PERSIST_TILES)
@pytest.mark.parametrize("grouping", [(0, 1), (1 << 20, 1)])
def test_persistent_step_equals_solo_bit_for_bit(E, streams, tile, grouping):
    """One persistent launch per step (push, prologue and passes from a work queue, one
    window of all streams or windows of at most 1 MB of pass working set): every stream
    equals its solo run bit for bit.  The first step tunes (and runs as a graph); the
    other seven run persistent, pushes included."""
    steps = max(COUNTS)
    b = run_batch(E, streams, tile, steps, grouping=grouping,
                  schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT)
    assert b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    assert "persistent step" in b.solver_name
    assert b.synchronize() == (0, -1)
    for s, st in enumerate(streams):
        g = run_solo(E, st, tile, steps)
        for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P2, E.EVR_STATE_P3,
                  E.EVR_STATE_F, E.EVR_STATE_TLAST, E.EVR_STATE_SQRTG, E.EVR_STATE_NPOS):
            np.testing.assert_array_equal(b.state(s, w), g.state(w), err_msg=f"stream {s} {w}")
        assert int(b.state(s, E.EVR_STATE_CLOCK)) == int(g.state(E.EVR_STATE_CLOCK))
        g.close()
    b.close()


@pytest.mark.parametrize("storage", [1, 2])
def test_persistent_step_16bit_storage_equals_solo(E, streams, storage):
    steps = 4
    b = run_batch(E, streams, 36, steps, grouping=(0, 1),
                  schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT, storage=storage)
    assert b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    for s in (0, 2, 4, 7):
        g = run_solo(E, streams[s], 36, steps, storage=storage)
        for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P3):
            np.testing.assert_array_equal(b.state(s, w), g.state(w), err_msg=f"stream {s} {w}")
        g.close()
    b.close()


def test_persistent_step_rejection_is_per_stream_and_idle_streams_are_untouched(E, streams):
    b = run_batch(E, streams, 36, 2, schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT)
    assert b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    before = [b.state(s, E.EVR_STATE_U).copy() for s in range(len(SIZES))]
    t_before = b.state(4, E.EVR_STATE_TLAST).copy()
    x, y, t, p, off = batch_step_arrays(streams, 300, 2)
    a4 = off[4]
    x = x.copy()
    x[a4] = 1  # off the 1 x 1 sensor
    keep = np.ones(len(x), bool)
    keep[off[1]:off[2]] = False
    cnt = np.diff(off)
    cnt[1] = 0
    off2 = np.concatenate([[0], np.cumsum(cnt)])
    b.step(x[keep], y[keep], t[keep], p[keep], off2, 30)
    rc, bad = b.synchronize()
    assert rc == E.EVR_ERR_OUT_OF_RANGE and bad == 4
    np.testing.assert_array_equal(b.state(1, E.EVR_STATE_U), before[1])
    np.testing.assert_array_equal(b.state(4, E.EVR_STATE_TLAST), t_before)
    assert b.synchronize() == (0, -1)
    b.close()


def test_persistent_step_is_one_launch_and_schedules_agree(E, streams):
    """Kernel timing counts one launch per persistent step; the graph schedule of the same
    tile gives the same bits; the autotuned schedule is one of the two."""
    steps = 5
    a = run_batch(E, streams, 36, 1, schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT)
    a.enable_kernel_timing(True)
    for k in range(1, steps):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        a.step(x, y, t, p, off, 30)
    ms, launches, _ = a.kernel_time()
    assert launches == steps - 1 and ms > 0
    g = run_batch(E, streams, 36, steps, schedule=E.EVR_BATCH_SCHEDULE_GRAPH)
    assert g.schedule == E.EVR_BATCH_SCHEDULE_GRAPH and "persistent" not in g.solver_name
    for s in range(len(SIZES)):
        np.testing.assert_array_equal(a.state(s, E.EVR_STATE_U), g.state(s, E.EVR_STATE_U))
    auto = run_batch(E, streams, 0, 2)
    assert auto.schedule in (E.EVR_BATCH_SCHEDULE_GRAPH, E.EVR_BATCH_SCHEDULE_PERSISTENT)
    for b in (a, g, auto):
        b.close()


def test_persistent_schedule_rejects_a_tile_without_persistent_form(E):
    b = E.Batch(SIZES[:3], tile_config=6)  # 32 x 64 tile
    with pytest.raises(E.EvrError):
        b.set_schedule(E.EVR_BATCH_SCHEDULE_PERSISTENT)
    with pytest.raises(E.EvrError):
        b.set_schedule(7)
    b.close()


def test_persistent_wait_timeout_is_reported_and_the_batch_continues(E, streams):
    """A work item waits for a count its stream never reaches: its bounded wait runs out,
    the launch reports EVR_ERR_TIMEOUT, the control words are reset (the self-test checks
    them), and later steps still equal the solo runs bit for bit."""
    steps = 4
    b = run_batch(E, streams, 36, 2, schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT)
    assert b.selftest_persist_timeout() == E.EVR_ERR_TIMEOUT
    for k in range(2, steps):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        b.step(x, y, t, p, off, 30)
    assert b.synchronize() == (0, -1)
    for s in (0, 2, 7):
        g = run_solo(E, streams[s], 36, steps)
        np.testing.assert_array_equal(b.state(s, E.EVR_STATE_U), g.state(E.EVR_STATE_U))
        g.close()
    b.close()


@pytest.mark.parametrize("over", [dict(data_term=1), dict(data_mode=1), dict(manifold=0),
                                  dict(t_max_us=0)])
def test_persistent_step_model_variants_equal_solo(E, streams, over):
    """The L2 data term of Eq. 7, the persistent data image, the flat manifold and the
    unclamped time surface through the persistent step: each stream equals its solo run."""
    steps = 4
    b = run_batch(E, streams, 31, steps, grouping=(0, 1),
                  schedule=E.EVR_BATCH_SCHEDULE_PERSISTENT, **over)
    assert b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    for s in (0, 2, 5, 7):
        g = run_solo(E, streams[s], 31, steps, **over)
        for w in (E.EVR_STATE_U, E.EVR_STATE_P2, E.EVR_STATE_F):
            np.testing.assert_array_equal(b.state(s, w), g.state(w), err_msg=f"stream {s} {w}")
        g.close()
    b.close()


def test_persistent_step_host_arrays_equal_device_arrays(E, streams):
    """evr_batch_step (host arrays, copied through the library's pinned staging) and
    evr_batch_step_device give the same persistent steps."""
    import torch
    steps = 4
    a = E.Batch(SIZES, tile_config=36)
    d = E.Batch(SIZES, tile_config=36)
    for b in (a, d):
        b.set_schedule(E.EVR_BATCH_SCHEDULE_PERSISTENT)
    keep = []  # the device copies stay alive until the steps that read them are done
    for k in range(steps):
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        a.step(x, y, t, p, off, 30)
        dev = [torch.from_numpy(v.view(np.int16) if v.dtype == np.uint16 else v).cuda()
               for v in (x, y, t, p, off)]
        torch.cuda.synchronize()
        d.step_device(*dev, 30)
        keep.append(dev)
    assert a.schedule == d.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    np.testing.assert_array_equal(a.images(), d.images())
    a.close()
    d.close()


def test_schedule_switch_mid_stream_keeps_every_stream_bit_identical(E, streams):
    """The schedule switches every two steps (a switch re-tunes the schedule at the next
    step, which runs as a graph; the step after it runs persistent when that was chosen):
    the state equals a run that never switches."""
    steps = 8
    ref = run_batch(E, streams, 36, steps, grouping=(0, 1),
                    schedule=E.EVR_BATCH_SCHEDULE_GRAPH)
    b = E.Batch(SIZES, tile_config=36)
    b.set_grouping(0, 1)
    seen = set()
    for k in range(steps):
        if k % 2 == 0:
            b.set_schedule(E.EVR_BATCH_SCHEDULE_PERSISTENT if k % 4 else
                           E.EVR_BATCH_SCHEDULE_GRAPH)
        x, y, t, p, off = batch_step_arrays(streams, 300, k)
        b.step(x, y, t, p, off, 30)
        seen.add(b.schedule)
    assert seen == {E.EVR_BATCH_SCHEDULE_GRAPH, E.EVR_BATCH_SCHEDULE_PERSISTENT}
    assert b.synchronize() == (0, -1)
    for s in range(len(SIZES)):
        for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_TLAST):
            np.testing.assert_array_equal(b.state(s, w), ref.state(s, w), err_msg=f"{s} {w}")
    ref.close()
    b.close()


@pytest.fixture(scope="module")
def batch256():
    """The 256-stream batched workload at full size (96 x 128x128, 96 x 240x180,
    64 x 346x260; 500-event packets, 50 iterations), its first three packets per stream."""
    from evsim.configs import batch_configs, make_batch
    cfgs = batch_configs()
    return cfgs, make_batch(cfgs, max_packets=3)


@pytest.mark.parametrize("schedule", ["graph", "persistent"])
def test_full_size_batch256_sampled_streams_match_oracle(E, batch256, schedule):
    """Full-size batch in the benchmark's launch configuration (autotuned tile; the graph
    or the persistent schedule): three steps, the last one teacher-forced against the
    FP64 oracle on sampled streams of every size (u within 1e-4, t_last bit-exact)."""
    cfgs, streams = batch256
    sizes = [(c.W, c.H) for c in cfgs]
    iters = cfgs[0].iters
    b = E.Batch(sizes)
    b.set_schedule(E.EVR_BATCH_SCHEDULE_GRAPH if schedule == "graph"
                   else E.EVR_BATCH_SCHEDULE_PERSISTENT)
    sampled = [0, 95, 96, 191, 192, 255]
    p = b.params
    oracles = {}
    for k in range(3):
        x, y, t, pol, off = batch_step_arrays(streams, 500, k)
        if k == 2:
            for s in sampled:
                W, H = sizes[s]
                o = O.OracleStream(W, H, O.OracleParams(
                    lam=float(p.lambda_), delta_pos=float(p.delta_pos),
                    delta_neg=float(p.delta_neg), u_min=float(p.u_min), u_max=float(p.u_max),
                    u_init=float(p.u_init), tau=float(p.tau), sigma=float(p.sigma),
                    time_scale=float(np.float32(p.time_scale))))
                o.set_up(b.state(s, E.EVR_STATE_U).astype(np.float64),
                         np.stack([b.state(s, w) for w in (E.EVR_STATE_P1, E.EVR_STATE_P2,
                                                           E.EVR_STATE_P3)]).astype(np.float64))
                o.set(O.TLAST, b.state(s, E.EVR_STATE_TLAST))
                o.set(O.TREF, int(b.state(s, E.EVR_STATE_CLOCK)))
                o.set(O.TINIT, int(b.state(s, E.EVR_STATE_TINIT)))
                a0, a1 = off[s], off[s + 1]
                assert o.push(x[a0:a1], y[a0:a1], t[a0:a1], pol[a0:a1]) == 0
                o.solve(iters)
                oracles[s] = o
        b.step(x, y, t, pol, off, iters)
    assert b.synchronize() == (0, -1)
    if schedule == "persistent":
        assert b.schedule == E.EVR_BATCH_SCHEDULE_PERSISTENT
    for s, o in oracles.items():
        np.testing.assert_array_equal(b.state(s, E.EVR_STATE_TLAST), o.get(O.TLAST))
        d = np.max(np.abs(b.image(s).astype(np.float64) - o.u))
        assert d <= 1e-4, (s, sizes[s], d)
    b.close()
