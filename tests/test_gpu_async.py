"""Asynchronous image readback (evr_get_image_async / evr_wait_image) through the C ABI:
a pipelined loop returns the same images as the synchronous one, tickets are validated,
more readbacks than the ring holds stay correct, and a device-side rejection is reported
by the wait that follows it."""
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
    out, t = [], 1000
    for _ in range(n):
        x = rng.integers(0, W, per).astype(np.uint16)
        y = rng.integers(0, H, per).astype(np.uint16)
        ts = t + np.sort(rng.integers(0, 3000, per)).astype(np.int64)
        t = int(ts[-1])
        out.append((x, y, ts, rng.choice(np.array([-1, 1], np.int8), per)))
    return out


def pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float32).pin_memory().numpy()


def test_pipelined_loop_equals_synchronous_loop(E):
    W, H = 97, 61
    pk = packets(1, W, H, 24, 400)
    a = E.Stream(W, H)
    want = []
    for x, y, t, p in pk:
        assert a.push(x, y, t, p) == 0
        a.solve(20)
        want.append(a.image().copy())
    b = E.Stream(W, H)
    bufs = [pinned((H, W)) for _ in range(3)]
    got, prev = [], None
    for k, (x, y, t, p) in enumerate(pk):
        assert E.evr_push_events(b.h, x, y, t, p) == 0
        E.evr_solve(b.h, 20)
        tk = E.evr_get_image_async(b.h, bufs[k % 3])
        if prev is not None:
            assert E.evr_wait_image(b.h, prev[0]) == 0
            got.append(prev[1].copy())
        prev = (tk, bufs[k % 3])
    assert E.evr_wait_image(b.h, prev[0]) == 0
    got.append(prev[1].copy())
    for k in range(len(pk)):
        np.testing.assert_array_equal(got[k], want[k], err_msg=f"packet {k}")


def test_tickets_and_ring_overflow(E):
    W, H = 40, 30
    g = E.Stream(W, H)
    with pytest.raises(E.EvrError):
        E.evr_wait_image(g.h, 1)  # not issued yet
    pk = packets(2, W, H, 40, 100)
    bufs = [pinned((H, W)) for _ in range(40)]
    ref = E.Stream(W, H)
    tickets = []
    for k, (x, y, t, p) in enumerate(pk):  # 40 readbacks queued, more than the ring holds
        assert E.evr_push_events(g.h, x, y, t, p) == 0
        E.evr_solve(g.h, 5)
        tickets.append(E.evr_get_image_async(g.h, bufs[k]))
    assert tickets == list(range(1, 41))
    for tk in tickets:
        assert E.evr_wait_image(g.h, tk) == 0
    for k, (x, y, t, p) in enumerate(pk):
        ref.push(x, y, t, p)
        ref.solve(5)
        np.testing.assert_array_equal(bufs[k], ref.image())
    with pytest.raises(E.EvrError):
        E.evr_wait_image(g.h, 41)
    with pytest.raises(E.EvrError):
        E.evr_wait_image(g.h, 0)


def test_device_rejection_is_reported_by_the_wait(E):
    import torch
    W, H = 50, 20
    g = E.Stream(W, H)
    twin = E.Stream(W, H)
    pk = packets(3, W, H, 3, 200)
    for s in (g, twin):
        x, y, t, p = pk[0]
        assert s.push(x, y, t, p) == 0
        s.solve(10)
    # a device-side push with one out-of-range column: the packet is rejected as a whole
    x, y, t, p = pk[1]
    x = x.copy()
    x[17] = W
    dev = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
           for a in (x, y, t, p)]
    assert g.push_device(*dev) == 0
    g.solve(10)
    buf = pinned((H, W))
    tk = E.evr_get_image_async(g.h, buf)
    assert E.evr_wait_image(g.h, tk) == E.EVR_ERR_OUT_OF_RANGE
    twin.solve(10)  # the twin sees the same solve without the rejected packet
    np.testing.assert_array_equal(buf, twin.image())
    tk = E.evr_get_image_async(g.h, buf)
    assert E.evr_wait_image(g.h, tk) == 0  # reported once
