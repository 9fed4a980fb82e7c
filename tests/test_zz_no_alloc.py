"""evr_gap_static: the gap reduction for callers that may not allocate device memory.

Callers such as a real-time event-camera loop (cudaMalloc synchronises the device)
or a host application that owns all device memory through its own pool can use
evr_gap_static, whose scratch is a fixed array inside the library.  This test
feeds it the planes of a live stream and checks it against evr_gap, twice in a row
(the second call reuses the array the first one left behind), for both data terms,
and checks that the calls leave the device's free memory unchanged.  It sits in a
file of its own that pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("data_term", [0, 1])
def test_gap_static_matches_evr_gap_on_consecutive_calls(data_term):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import evr as E

    W, H = 173, 91
    rng = np.random.default_rng(11 + data_term)
    g = E.Stream(W, H, data_term=data_term)
    planes = (E.EVR_STATE_U, E.EVR_STATE_P1, E.EVR_STATE_P2, E.EVR_STATE_P3, E.EVR_STATE_F,
              E.EVR_STATE_TX, E.EVR_STATE_TY)
    t = 1000
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    p = g.params
    for call in range(2):
        n = 3000
        x = rng.integers(0, W, n).astype(np.uint16)
        y = rng.integers(0, H, n).astype(np.uint16)
        ts = t + np.sort(rng.integers(0, 20_000, n)).astype(np.int64)
        t = int(ts[-1])
        pol = rng.choice(np.array([-1, 1], np.int8), n)
        assert g.push(x, y, ts, pol) == 0
        g.solve(20 + 10 * call)
        want = g.gap()
        dev = [torch.from_numpy(np.ascontiguousarray(g.state(w))).cuda() for w in planes]
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        rc = E.evr_gap_static(*dev, W, H, W, p.lambda_, p.u_min, p.u_max, out,
                              stream.cuda_stream, data_term=data_term)
        assert rc == 0
        torch.cuda.synchronize()
        # the entry point's one promise: no device memory taken (the first call on the
        # device may load the library's module lazily; from the second call on, the
        # device's free memory must not move)
        free1, _ = torch.cuda.mem_get_info()
        assert torch.cuda.memory_allocated() == alloc0
        if call:
            assert free1 == free0
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(want[0], rel=1e-5)
        assert got[1] == pytest.approx(want[1], rel=1e-5)
        assert want[0] - want[1] >= -1e-6 * abs(want[0])
    # sizes beyond the array's capacity are refused before anything is queued
    big_w = E.EVR_GAP_STATIC_MAX_PIXELS // 1024 + 1
    big = torch.zeros(big_w * 1024, dtype=torch.float32, device="cuda")
    rc = E.evr_gap_static(*([big] * 7), big_w, 1024, big_w, p.lambda_, p.u_min, p.u_max, out,
                          stream.cuda_stream, data_term=data_term)
    assert rc == E.EVR_ERR_INVALID_ARG
    # planes the library must not read are refused by the binding
    with pytest.raises(ValueError):
        E.evr_gap_static(*(dev[:6] + [dev[6].cpu()]), W, H, W, p.lambda_, p.u_min, p.u_max,
                         out, stream.cuda_stream, data_term=data_term)
    with pytest.raises(ValueError):
        E.evr_gap_static(*dev, W, H + 1, W, p.lambda_, p.u_min, p.u_max, out,
                         stream.cuda_stream, data_term=data_term)
    g.close()
