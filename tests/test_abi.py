"""The C-ABI library builds for sm_103a, loads, and exports what include/evr.h declares.

No compute calls: these run without a GPU.
"""
import ctypes

import numpy as np
import pytest

from paper_1607_06283_gb300 import build


@pytest.fixture(scope="module")
def evr():
    build.build()
    from paper_1607_06283_gb300 import evr as E
    return E


def test_every_declared_function_is_exported(evr):
    names = evr.header_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(evr._lib, n), n


def test_default_params(evr):
    p = evr.evr_default_params()
    assert p.lambda_ == pytest.approx(90.0)
    assert p.tau == pytest.approx(1.0 / np.sqrt(8 + 4 * np.sqrt(2)), rel=1e-7)
    assert p.tau * p.sigma * (8 + 4 * np.sqrt(2)) <= 1 + 1e-6
    assert p.t_init_us == evr.EVR_T_INIT_FIRST
    assert p.u_min == pytest.approx(np.exp(-3), rel=1e-7)


def test_struct_layout_matches_header(evr):
    # 9 floats, pad, 2 int64 (8-byte aligned), 6 ints + 1 float, tail pad to 8
    assert ctypes.sizeof(evr.evr_params) == 9 * 4 + 4 + 2 * 8 + 7 * 4 + 4


def test_argument_errors_need_no_gpu(evr):
    E = evr
    h = ctypes.c_void_p()
    p = E.evr_default_params()
    assert E._lib.evr_create(0, 5, ctypes.byref(p), ctypes.byref(h)) == E.EVR_ERR_INVALID_ARG
    assert E._lib.evr_create(5, 5, None, ctypes.byref(h)) == E.EVR_ERR_INVALID_ARG
    bad = E.evr_default_params()
    bad.tau = 1.0
    bad.sigma = 1.0
    assert E._lib.evr_create(5, 5, ctypes.byref(bad), ctypes.byref(h)) == E.EVR_ERR_INVALID_ARG
    bad = E.evr_default_params()
    bad.u_min = 0.0
    assert E._lib.evr_create(5, 5, ctypes.byref(bad), ctypes.byref(h)) == E.EVR_ERR_INVALID_ARG
    assert E._lib.evr_solve(None, 3) == E.EVR_ERR_INVALID_ARG
    assert E._lib.evr_push_events(None, None, None, None, None, 0) == E.EVR_ERR_INVALID_ARG
    assert E.evr_strerror(E.EVR_ERR_NONMONOTONIC) == "event timestamp decreases"


def test_ptxas_reports_no_spills_in_the_iteration_kernels(evr):
    """Register pressure check on the built kernels (from nvcc -Xptxas -v).  Two
    instantiations are allowed a few bytes: the two-pair FP16 tile held to 80 registers
    (two CTAs per SM; measured faster than one CTA without the spill) and the cluster
    solver's 1024-thread tile (64 registers is the most a 1024-thread CTA can have); the
    persistent batch step's two-pair FP16 tiles share the first allowance."""
    import os
    import re
    allowed = {"ILi1ELi4ELi12E6__half": 8, "ILi1ELi4ELi8E6__half": 8,
               "k_clusterILi1ELi2ELi32E": 8}
    text = ""
    for f in ("evr_kernels.ptxas.txt", "evr_solvers.ptxas.txt", "evr_grad.ptxas.txt",
              "evr_cluster.ptxas.txt", "evr_staged.ptxas.txt", "evr_persist.ptxas.txt"):
        text += open(os.path.join(os.path.dirname(build.LIB), f)).read()
    blocks = text.split("Compiling entry function")
    seen = 0
    for b in blocks[1:]:
        name = b.split("'")[1]
        if any(k in name for k in ("k_tiled", "k_prologue", "k_push", "k_rev_tiled",
                                   "k_cluster", "k_staged", "k_resident",
                                   "k_batch_persist")):
            seen += 1
            spill = int(re.search(r"(\d+) bytes spill stores", b).group(1))
            limit = max([v for k, v in allowed.items() if k in name], default=0)
            assert spill <= limit, (name, spill)
    assert seen >= 40


def test_unrolled_workspace_sizing_needs_no_gpu(evr):
    """Workspace of the differentiation calls: checkpoints every `every` iterations, the
    forward's tape of the last segment and, with several segments, a replay tape of
    `every` iterations (5 planes per tape iteration); invalid sizes give 0."""
    E = evr
    ws = E._lib.evr_unrolled_workspace_bytes
    W, H, n, K = 37, 23, 3, 30
    plane = (W * H * n * 4 + 255) // 256 * 256
    # every >= K: one checkpoint and the whole tape, whatever `every` is
    assert ws(W, H, W, n, K, K) == ws(W, H, W, n, K, 2 * K) == ws(W, H, W, n, K, 1000)
    # every 10: 3 checkpoints, 10 + 10 tape slots; every 30: 1 checkpoint, 30 tape slots
    assert ws(W, H, W, n, K, 30) - ws(W, H, W, n, K, 10) == ((4 + 150) - (12 + 100)) * plane
    # every 7 (segments 7, 7, 7, 7, 2): 5 checkpoints, the last segment's 2 slots + 7
    assert ws(W, H, W, n, K, 10) - ws(W, H, W, n, K, 7) == ((12 + 100) - (20 + 45)) * plane
    # a larger pitch grows every plane
    assert ws(W, H, W + 64, n, K, 10) > ws(W, H, W, n, K, 10)
    for bad in [(0, H, W, n, K, 10), (W, H, W - 1, n, K, 10), (W, H, W, 0, K, 10),
                (W, H, W, n, 0, 10), (W, H, W, n, K, 0)]:
        assert ws(*bad) == 0, bad


def test_gap_static_binding_refuses_planes_before_the_call(evr):
    # host tensors, wrong dtypes or short planes never reach the library (no GPU needed:
    # the binding raises before calling it)
    import torch
    W, H = 8, 4
    planes = [torch.zeros(W * H, dtype=torch.float32) for _ in range(7)]
    out = torch.zeros(2, dtype=torch.float64)
    with pytest.raises(ValueError):
        evr.evr_gap_static(*planes, W, H, W, 90.0, 0.05, 20.0, out)
    with pytest.raises(ValueError):
        evr.evr_gap_static(*planes, W, H, W, 90.0, 0.05, 20.0, out.float())
