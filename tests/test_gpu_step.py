"""evr_step_device (push and solve in one call, one CUDA graph once the solver is settled)
through the C ABI: bit-identical to evr_push_events_device + evr_solve over the tuning,
refinement and fused calls, for empty and over-sized packets, and with a rejected
packet."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import evr
    return torch, evr


def packets(seed, W, H, n, per):
    rng = np.random.default_rng(seed)
    out, t = [], 2000
    for _ in range(n):
        x = rng.integers(0, W, per).astype(np.uint16)
        y = rng.integers(0, H, per).astype(np.uint16)
        ts = t + np.sort(rng.integers(0, 2000, per)).astype(np.int64)
        t = int(ts[-1])
        out.append((x, y, ts, rng.choice(np.array([-1, 1], np.int8), per)))
    return out


def dev(torch, pk):
    x, y, t, p = pk
    return [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
            for a in (x, y, t, p)]


# tile_config 55: clusters of 4 x 4 32 x 32 tiles as super-tiles with a 6-pixel halo;
# 73: the resident solver (one cooperative launch, the push inside it)
@pytest.mark.parametrize("over", [{}, dict(tile_config=45), dict(solver=1),
                                  dict(tvl1_iters=3), dict(tile_config=55),
                                  dict(tile_config=73), dict(tile_config=73, data_mode=1),
                                  dict(tile_config=32), dict(tile_config=2)])
def test_step_equals_push_then_solve(T, over):
    torch, E = T
    W, H = 150, 97
    pk = packets(1, W, H, 14, 700)
    a, b = E.Stream(W, H, **over), E.Stream(W, H, **over)
    for k, item in enumerate(pk):
        d = dev(torch, item)
        assert E.evr_step_device(a.h, *d, 20) == 0
        assert b.push_device(*d) == 0
        b.solve(20)
        if k in (0, 3, 8, 13):
            np.testing.assert_array_equal(a.image(), b.image(), err_msg=f"packet {k}")
    for w in (E.EVR_STATE_P1, E.EVR_STATE_P3, E.EVR_STATE_TLAST, E.EVR_STATE_NPOS):
        np.testing.assert_array_equal(a.state(w), b.state(w))
    if "tile_config" in over:  # autotuned streams may settle differently (timing noise);
        assert a.solver_name == b.solver_name  # the results do not depend on it


# tile_config 47: one 4 x 4 cluster over the sensor, the push inside its single launch;
# 73: the resident solver
@pytest.mark.parametrize("tile", [45, 47, 73, 32])
def test_step_with_empty_and_large_packets_and_a_rejection(T, tile):
    torch, E = T
    W, H = 64, 40
    a, b = E.Stream(W, H, tile_config=tile), E.Stream(W, H, tile_config=tile)
    pk = packets(2, W, H, 3, 500)
    big = packets(3, W, H, 1, 40000)[0]  # above one CTA's packet: the two-call path
    big = (big[0], big[1], big[2] + pk[-1][2][-1], big[3])
    empty = tuple(np.zeros(0, a_.dtype) for a_ in pk[0])
    bad = (pk[1][0].copy(),) + pk[1][1:]
    bad[0][5] = W  # out of range: the packet is rejected, the solve still runs
    for item in (pk[0], empty, bad, pk[2], big):
        d = dev(torch, item)
        rc = E.evr_step_device(a.h, *d, 15)
        assert rc == 0
        assert b.push_device(*d) == 0
        b.solve(15)
        ra, rb = a.synchronize(), b.synchronize()
        assert ra == rb
        np.testing.assert_array_equal(a.image(), b.image())
    assert int(a.state(E.EVR_STATE_CLOCK)) == int(b.state(E.EVR_STATE_CLOCK))


@pytest.mark.parametrize("over,iters", [({}, 25), (dict(tile_config=45), 25),
                                        (dict(tile_config=47), 25),
                                        (dict(tile_config=47, data_term=1), 25),
                                        (dict(tile_config=73), 25), (dict(tile_config=73), 7),
                                        (dict(tile_config=76, data_term=1), 25),
                                        (dict(tile_config=78), 8)])
def test_host_step_equals_push_then_solve(T, over, iters):
    """evr_step (host arrays, copied on the copy stream ahead of the packet's graph) against
    evr_push_events + evr_solve; the host-side checks reject a bad packet before anything
    is queued."""
    torch, E = T
    W, H = 120, 77
    pk = packets(4, W, H, 12, 900)
    a, b = E.Stream(W, H, **over), E.Stream(W, H, **over)
    for k, (x, y, t, p) in enumerate(pk):
        assert E.evr_step(a.h, x, y, t, p, iters) == 0
        assert b.push(x, y, t, p) == 0
        b.solve(iters)
        if k in (0, 6, 11):
            np.testing.assert_array_equal(a.image(), b.image(), err_msg=f"packet {k}")
    x, y, t, p = packets(5, W, H, 1, 50)[0]
    x = x.copy()
    x[3] = W
    assert E.evr_step(a.h, x, y, t + pk[-1][2][-1], p, iters) == E.EVR_ERR_OUT_OF_RANGE
    np.testing.assert_array_equal(a.image(), b.image())
