"""Checkpoint/resume and failure detection through the C ABI.

Checkpoint: a stream's state read with evr_get_state and written into a fresh stream
with evr_set_state resumes bit-identically.  Failure detection: the persistent
solver's neighbour waits are bounded; the self-test leaves one CTA's progress flag
unset, the waits run out, the device reports EVR_ERR_TIMEOUT, and the stream keeps
working.  No GPU fault is involved: the failure is a flag that nothing sets.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import evr
    return evr


def packets(seed, W, H, n, per):
    rng = np.random.default_rng(seed)
    out, t = [], 5000
    for _ in range(n):
        x = rng.integers(0, W, per).astype(np.uint16)
        y = rng.integers(0, H, per).astype(np.uint16)
        ts = t + np.sort(rng.integers(0, 4000, per)).astype(np.int64)
        t = int(ts[-1])
        out.append((x, y, ts, rng.choice(np.array([-1, 1], np.int8), per)))
    return out


@pytest.mark.parametrize("over", [dict(solver=2, tile_config=2), dict(solver=1),
                                  dict(solver=2, tile_config=8, storage=1),
                                  dict(solver=2, tile_config=12, data_mode=1)])
def test_checkpoint_resume_is_bit_identical(E, over):
    W, H = 90, 70
    pk = packets(1, W, H, 8, 600)
    a = E.Stream(W, H, **over)
    for x, y, t, p in pk[:4]:
        assert a.push(x, y, t, p) == 0
        a.solve(20)
    ckpt = a.save()
    b = E.Stream(W, H, **over)
    b.load(ckpt)
    for g in (a, b):
        for x, y, t, p in pk[4:]:
            assert g.push(x, y, t, p) == 0
            g.solve(20)
    for w in (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P3, E.EVR_STATE_TLAST,
              E.EVR_STATE_F):
        np.testing.assert_array_equal(b.state(w), a.state(w))
    assert int(b.state(E.EVR_STATE_CLOCK)) == int(a.state(E.EVR_STATE_CLOCK))


def test_checkpoint_rejects_wrong_sizes(E):
    g = E.Stream(16, 8)
    with pytest.raises(E.EvrError):
        E.evr_set_state(g.h, E.EVR_STATE_U, np.zeros((8, 15), np.float32))
    with pytest.raises(E.EvrError):
        E.evr_set_state(g.h, E.EVR_STATE_SQRTG, np.zeros((8, 16), np.float32))


def test_wait_timeout_is_detected_and_the_stream_recovers(E):
    W, H = 100, 60
    pk = packets(2, W, H, 6, 500)
    a = E.Stream(W, H, solver=2, tile_config=12)   # persistent configuration
    twin = E.Stream(W, H, solver=2, tile_config=12)
    for g in (a, twin):
        for x, y, t, p in pk[:3]:
            assert g.push(x, y, t, p) == 0
            g.solve(15)
    t0 = time.perf_counter()
    rc = E._lib.evr_selftest_wait_timeout(a.h)
    dt = time.perf_counter() - t0
    assert rc == E.EVR_ERR_TIMEOUT, rc
    assert dt < 10.0
    assert a.synchronize() == 0  # reported once
    np.testing.assert_array_equal(a.image(), twin.image())  # state restored
    for g in (a, twin):
        for x, y, t, p in pk[3:]:
            assert g.push(x, y, t, p) == 0
            g.solve(15)
    assert a.synchronize() == 0
    np.testing.assert_array_equal(a.image(), twin.image())  # solver works after the test


# tile_config 47: one cluster of 4 x 4 CTAs over the sensor (evr_params.tile_config)
@pytest.mark.parametrize("tile", [0, 47])
def test_cluster_wait_timeout_is_detected_and_the_stream_recovers(E, tile):
    """One CTA of the cluster never sends its edges: its neighbours' bounded waits run out,
    the launch reports EVR_ERR_TIMEOUT, and the stream (state saved and restored) goes on
    bit-identically to a twin that never ran the test."""
    W, H = 100, 60
    pk = packets(3, W, H, 6, 500)
    a = E.Stream(W, H, solver=2, tile_config=tile)
    twin = E.Stream(W, H, solver=2, tile_config=tile)
    for g in (a, twin):
        for x, y, t, p in pk[:3]:
            assert g.push(x, y, t, p) == 0
            g.solve(15)
    t0 = time.perf_counter()
    rc = E._lib.evr_selftest_cluster_wait_timeout(a.h)
    dt = time.perf_counter() - t0
    assert rc == E.EVR_ERR_TIMEOUT, rc
    assert dt < 10.0
    assert a.synchronize() == 0  # reported once
    np.testing.assert_array_equal(a.image(), twin.image())  # state restored
    for g in (a, twin):
        for x, y, t, p in pk[3:]:
            assert g.push(x, y, t, p) == 0
            g.solve(15)
    assert a.synchronize() == 0
    np.testing.assert_array_equal(a.image(), twin.image())


# tile_config 73: the resident solver, 32 x 64 tiles with a 9-pixel halo (evr_params)
@pytest.mark.parametrize("tile", [0, 73])
def test_resident_wait_timeout_is_detected_and_the_stream_recovers(E, tile):
    """The resident solver's grid barrier never completes (its arrival count starts far
    below the target): every CTA's bounded wait runs out, the launch reports
    EVR_ERR_TIMEOUT, and the stream (state restored, barrier words cleared) goes on
    bit-identically to a twin that never ran the test."""
    W, H = 100, 60
    pk = packets(4, W, H, 6, 500)
    a = E.Stream(W, H, solver=2, tile_config=tile)
    twin = E.Stream(W, H, solver=2, tile_config=tile)
    for g in (a, twin):
        for x, y, t, p in pk[:3]:
            assert g.push(x, y, t, p) == 0
            g.solve(20)
    t0 = time.perf_counter()
    rc = E._lib.evr_selftest_resident_wait_timeout(a.h)
    dt = time.perf_counter() - t0
    assert rc == E.EVR_ERR_TIMEOUT, rc
    assert dt < 10.0
    assert a.synchronize() == 0  # reported once
    np.testing.assert_array_equal(a.image(), twin.image())  # state restored
    for g in (a, twin):
        for x, y, t, p in pk[3:]:
            assert g.push(x, y, t, p) == 0
            g.solve(20)
    assert a.synchronize() == 0
    np.testing.assert_array_equal(a.image(), twin.image())


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failures_are_reported_and_release_everything(E):
    """Fault injection on the host side: every allocation of evr_create / evr_batch_create
    in turn is made to fail; each attempt reports OOM (or CUDA) and leaves no device
    memory behind, and the library works afterwards."""
    E.Stream(64, 48).close()  # context and module loaded
    free0 = _free_bytes()
    failed = 0
    for n in range(1, 12):
        E._lib.evr_test_fail_alloc_after(n)
        try:
            g = E.Stream(64, 48)
        except E.EvrError as e:
            assert e.code in (E.EVR_ERR_OOM, E.EVR_ERR_CUDA), e.code
            failed += 1
            continue
        g.close()  # n was past the last allocation of evr_create
        break
    for n in range(1, 12):
        E._lib.evr_test_fail_alloc_after(n)
        try:
            b = E.Batch([(40, 30), (17, 9)])
        except E.EvrError as e:
            assert e.code in (E.EVR_ERR_OOM, E.EVR_ERR_CUDA), e.code
            failed += 1
            continue
        b.close()
        break
    E._lib.evr_test_fail_alloc_after(0)
    assert failed >= 4  # every allocation site of both creates was exercised
    assert abs(_free_bytes() - free0) < (8 << 20)
    pk = packets(4, 64, 48, 2, 300)
    g = E.Stream(64, 48)
    for x, y, t, p in pk:
        assert g.push(x, y, t, p) == 0
        g.solve(10)
    assert g.synchronize() == 0


def test_push_staging_allocation_failure_leaves_the_stream_unchanged(E):
    W, H = 80, 40
    small = packets(5, W, H, 1, 200)[0]
    big = packets(6, W, H, 1, 6000)[0]  # grows the pinned slot and the device buffer
    big = (big[0], big[1], big[2] + small[2][-1], big[3])
    a, twin = E.Stream(W, H), E.Stream(W, H)
    for g in (a, twin):
        assert g.push(*small) == 0
        g.solve(10)
    E._lib.evr_test_fail_alloc_after(1)
    with pytest.raises(E.EvrError) as ei:
        E._check(E._lib.evr_push_events(a.h, big[0].ctypes.data, big[1].ctypes.data,
                                        big[2].ctypes.data, big[3].ctypes.data, len(big[0])),
                 "evr_push_events")
    E._lib.evr_test_fail_alloc_after(0)
    assert ei.value.code == E.EVR_ERR_OOM
    for g in (a, twin):
        g.solve(10)
    np.testing.assert_array_equal(a.image(), twin.image())
    for g in (a, twin):  # and the stream takes the packet afterwards
        assert g.push(*big) == 0
        g.solve(10)
    np.testing.assert_array_equal(a.image(), twin.image())


@pytest.mark.parametrize("fail_at", [1, 2])
def test_step_slot_allocation_failure_leaves_the_stream_unchanged(E, fail_at):
    """evr_step grows a staging slot's pinned buffer (first allocation) and then its device
    buffer (second) for a large packet; when either fails the packet is not queued and
    the stream goes on as its twin."""
    W, H = 80, 40
    smalls = packets(7, W, H, 4, 200)  # four packets: every staging slot holds a buffer
    big = packets(8, W, H, 1, 6000)[0]  # past the slot's first 4096 events
    big = (big[0], big[1], big[2] + smalls[-1][2][-1], big[3])
    a, twin = E.Stream(W, H), E.Stream(W, H)
    for g in (a, twin):
        for pk in smalls:
            assert E.evr_step(g.h, *pk, 10) == 0
    E._lib.evr_test_fail_alloc_after(fail_at)
    rc = E._lib.evr_step(a.h, big[0].ctypes.data, big[1].ctypes.data, big[2].ctypes.data,
                         big[3].ctypes.data, len(big[0]), 10)
    E._lib.evr_test_fail_alloc_after(0)
    assert rc == E.EVR_ERR_OOM
    for g in (a, twin):
        g.solve(10)
    np.testing.assert_array_equal(a.image(), twin.image())
    for g in (a, twin):  # and the stream takes the packet afterwards
        assert E.evr_step(g.h, *big, 10) == 0
    np.testing.assert_array_equal(a.image(), twin.image())
