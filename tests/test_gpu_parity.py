"""GPU (libevr, through the C ABI) against the FP64 oracle.

Integer integration (t_last, counts, clock) must be bit-exact.  The image u must
stay within max-abs 1e-4 of the oracle after K FP32 iterations, checked
teacher-forced per packet: the oracle starts each packet from the GPU's (u, p)
widened to FP64 and the same integer state.
"""
import numpy as np
import pytest

from evsim import CONFIGS, make_stream
from oracle import oracle as O

pytestmark = pytest.mark.gpu

TOL_U = 1e-4


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import evr
    return evr


def oracle_params(p, **kw):
    return O.OracleParams(
        lam=float(p.lambda_), delta_pos=float(p.delta_pos), delta_neg=float(p.delta_neg),
        u_min=float(p.u_min), u_max=float(p.u_max), u_init=float(p.u_init), tau=float(p.tau),
        sigma=float(p.sigma), time_scale=float(np.float32(p.time_scale)),
        t_max_us=int(p.t_max_us),
        t_init_us=None if p.t_init_us == -(2 ** 63) else int(p.t_init_us),
        data_mode=int(p.data_mode), manifold=int(p.manifold), data_term=int(p.data_term),
        tvl1_iters=int(p.tvl1_iters), tvl1_lambda=float(np.float32(p.tvl1_lambda)), **kw)


N_CFGS = 80  # solver configurations selectable with evr_params.tile_config = 1..N_CFGS
SOLVERS = [("unfused", 1, 0)] + [(f"cfg{k}", 2, k) for k in range(1, N_CFGS + 1)]
# tile_config of the cluster solver: one 4 x 4 cluster of 32 x 32 tiles over a sensor of
# up to 128 x 128 (one launch per packet), and 2 x 2 clusters as super-tiles with a
# 4-pixel halo
CLUSTER_ONE = 47
CLUSTER_SUPER = 59
# tile_config of the tensor-copy staged persistent passes: 32 x 32 tiles with a 4-pixel
# halo (512 threads) and 32 x 48 tiles with a 5-pixel halo (384 threads)
STAGED_32 = 63
STAGED_48 = 69
# tile_config of the resident solver (one cooperative launch per packet, grid barrier
# every R iterations): 32 x 64 tiles with a 9-pixel halo, 32 x 32 tiles with 6
RESIDENT_64 = 73
RESIDENT_32 = 76


def make_pair(E, W, H, solver=2, tile=0, **over):
    p = E.evr_default_params()
    p.solver = solver
    p.tile_config = tile
    for k, v in over.items():
        setattr(p, k, v)
    try:
        g = E.Stream(W, H, p)
    except E.EvrError as e:
        if tile and e.code == E.EVR_ERR_NOT_SUPPORTED:
            pytest.skip(f"tile_config {tile} does not fit a {W} x {H} sensor")
        raise
    o = O.OracleStream(W, H, oracle_params(p))
    return g, o


def integer_state_equal(E, g, o):
    for w_g, w_o in ((E.EVR_STATE_TLAST, O.TLAST), (E.EVR_STATE_NPOS, O.NPOS),
                     (E.EVR_STATE_NNEG, O.NNEG)):
        np.testing.assert_array_equal(g.state(w_g), o.get(w_o))
    assert int(g.state(E.EVR_STATE_CLOCK)) == int(o.get(O.TREF))


def teacher_forced_packet(E, g, o, x, y, t, pol, K):
    """Returns max |u_gpu - u_oracle| after one packet started from the GPU state."""
    o.set_up(g.state(E.EVR_STATE_U).astype(np.float64), g.p().astype(np.float64))
    assert g.push(x, y, t, pol) == 0
    assert o.push(x, y, t, pol) == 0
    integer_state_equal(E, g, o)
    g.solve(K)
    o.solve(K)
    return float(np.max(np.abs(g.image().astype(np.float64) - o.u)))


def rand_packets(rng, W, H, n_packets, per, t0=10_000, dense=False):
    out = []
    t = t0
    for _ in range(n_packets):
        k = per
        xs = rng.integers(0, 2 if dense else W, k).astype(np.uint16) % W
        ys = rng.integers(0, 2 if dense else H, k).astype(np.uint16) % H
        ts = t + np.sort(rng.integers(0, 3000, k)).astype(np.int64)
        t = int(ts[-1])
        ps = rng.choice(np.array([-1, 1], np.int8), k)
        out.append((xs, ys, ts, ps))
    return out


# ----------------------------------------------------------------- integration
@pytest.mark.parametrize("path", ["host", "device"])
@pytest.mark.parametrize("W,H,per,dense", [(128, 128, 500, False), (37, 11, 700, True),
                                           (1, 1, 64, False), (346, 260, 40000, False)])
def test_scatter_bit_exact(E, path, W, H, per, dense):
    import torch
    rng = np.random.default_rng(W + H + per)
    g, o = make_pair(E, W, H)
    for pk in rand_packets(rng, W, H, 3, per, dense=dense):
        if path == "host":
            assert g.push(*pk) == 0
        else:
            dev = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
                   for a in pk]
            assert g.push_device(*dev) == 0
            assert g.synchronize() == 0
        assert o.push(*pk) == 0
        integer_state_equal(E, g, o)
    assert int(g.state(E.EVR_STATE_TINIT)) == int(o.get(O.TINIT))
    g.solve(0)
    o.solve(0)
    np.testing.assert_array_equal(g.state(E.EVR_STATE_NPOS), 0)
    np.testing.assert_allclose(g.state(E.EVR_STATE_F), o.get(O.F), rtol=2e-6)
    np.testing.assert_allclose(g.state(E.EVR_STATE_SQRTG), np.sqrt(o.get(O.G)), rtol=2e-6)
    np.testing.assert_allclose(g.state(E.EVR_STATE_TX), o.get(O.TX), rtol=2e-6, atol=1e-5)
    np.testing.assert_allclose(g.state(E.EVR_STATE_TY), o.get(O.TY), rtol=2e-6, atol=1e-5)


@pytest.mark.parametrize("bad,code", [("x", -2), ("y", -2), ("pol", -3), ("t", -4), ("clock", -4)])
@pytest.mark.parametrize("path", ["host", "device"])
def test_rejected_packet_changes_nothing(E, bad, code, path):
    import torch
    rng = np.random.default_rng(3)
    W, H = 20, 12
    g, o = make_pair(E, W, H)
    pk = rand_packets(rng, W, H, 2, 300)
    assert g.push(*pk[0]) == 0 and o.push(*pk[0]) == 0
    g.solve(5)
    o.solve(5)
    x, y, t, p = (a.copy() for a in pk[1])
    if bad == "x":
        x[100] = W
    elif bad == "y":
        y[100] = H
    elif bad == "pol":
        p[100] = 0
    elif bad == "t":
        t[100] = t[99] - 1
    else:
        t[:] = pk[0][2][-1] - 5
    u_before = g.image()
    if path == "host":
        assert g.push(x, y, t, p) == code
    else:
        dev = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
               for a in (x, y, t, p)]
        assert g.push_device(*dev) == 0
        assert g.synchronize() == code
        assert g.synchronize() == 0  # reported once
    assert o.push(x, y, t, p) == code
    integer_state_equal(E, g, o)
    np.testing.assert_array_equal(g.image(), u_before)


# ----------------------------------------------------------------- solver parity
@pytest.fixture(scope="module")
def rects128():
    return make_stream(CONFIGS["rects128"])


@pytest.mark.parametrize("name,solver,tile", SOLVERS)
def test_teacher_forced_parity_rects128(E, rects128, name, solver, tile):
    cfg = CONFIGS["rects128"]
    g, o = make_pair(E, cfg.W, cfg.H, solver=solver, tile=tile)
    worst = 0.0
    for a in range(0, len(rects128), cfg.packet):
        s = rects128.slice(a, a + cfg.packet)
        worst = max(worst, teacher_forced_packet(E, g, o, s.x, s.y, s.t, s.pol, cfg.iters))
    assert worst <= TOL_U, (name, worst)


def test_free_running_drift_rects128(E, rects128):
    """Both sides run the whole 40-packet stream on their own."""
    cfg = CONFIGS["rects128"]
    g, o = make_pair(E, cfg.W, cfg.H)
    for a in range(0, len(rects128), cfg.packet):
        s = rects128.slice(a, a + cfg.packet)
        assert g.push(s.x, s.y, s.t, s.pol) == 0 and o.push(s.x, s.y, s.t, s.pol) == 0
        g.solve(cfg.iters)
        o.solve(cfg.iters)
    drift = float(np.max(np.abs(g.image().astype(np.float64) - o.u)))
    assert drift <= TOL_U, drift


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (33, 17), (65, 31), (100, 3),
                                 (3, 100), (57, 57)])
@pytest.mark.parametrize("name,solver,tile", [SOLVERS[0], SOLVERS[1], SOLVERS[11], SOLVERS[20],
                                              SOLVERS[24], SOLVERS[CLUSTER_ONE],
                                              SOLVERS[CLUSTER_SUPER], SOLVERS[STAGED_32],
                                              SOLVERS[STAGED_48], SOLVERS[RESIDENT_64],
                                              SOLVERS[RESIDENT_32]])
def test_ragged_sizes(E, W, H, name, solver, tile):
    rng = np.random.default_rng(W * 1000 + H)
    g, o = make_pair(E, W, H, solver=solver, tile=tile)
    worst = 0.0
    for pk in rand_packets(rng, W, H, 4, max(1, W * H // 4)):
        worst = max(worst, teacher_forced_packet(E, g, o, *pk, 23))
    assert worst <= TOL_U, worst


@pytest.mark.parametrize("over", [dict(manifold=0), dict(data_mode=1), dict(t_max_us=0),
                                  dict(t_init_us=0), dict(lambda_=5.0), dict(time_scale=0.02),
                                  dict(data_term=1), dict(data_term=1, lambda_=3.0, solver=1),
                                  dict(tvl1_iters=10), dict(tvl1_iters=10, tvl1_lambda=0.5),
                                  dict(tvl1_iters=5, data_term=1, solver=1)])
def test_parameter_variants(E, over):
    rng = np.random.default_rng(17)
    W, H = 70, 45
    g, o = make_pair(E, W, H, **over)
    worst = 0.0
    for pk in rand_packets(rng, W, H, 5, 400):
        worst = max(worst, teacher_forced_packet(E, g, o, *pk, 30))
    assert worst <= TOL_U, worst


def test_empty_packet_and_zero_iterations(E):
    rng = np.random.default_rng(4)
    W, H = 40, 30
    g, o = make_pair(E, W, H)
    e = np.zeros(0)
    assert g.push(e, e, e, e) == 0
    g.solve(0)
    o.solve(0)
    np.testing.assert_array_equal(g.image(), np.float32(o.u))
    for pk in rand_packets(rng, W, H, 2, 200):
        d = teacher_forced_packet(E, g, o, *pk, 0)
        assert d == 0.0
        assert g.push(e, e, e, e) == 0
        assert teacher_forced_packet(E, g, o, e, e, e, e, 12) <= TOL_U


def test_tiled_is_deterministic_and_matches_unfused(E, rects128):
    cfg = CONFIGS["rects128"]
    imgs = []
    for solver, tile in ((2, 2), (2, 2), (1, 0)):
        g, _ = make_pair(E, cfg.W, cfg.H, solver=solver, tile=tile)
        for a in range(0, 10 * cfg.packet, cfg.packet):
            s = rects128.slice(a, a + cfg.packet)
            g.push(s.x, s.y, s.t, s.pol)
            g.solve(cfg.iters)
        imgs.append(g.image())
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_allclose(imgs[0], imgs[2], rtol=0, atol=1e-5)


# ----------------------------------------------------------------- FP64 gap
@pytest.mark.parametrize("data_term", [0, 1])
def test_gap_matches_oracle_and_shrinks(E, rects128, data_term):
    """data_mode 1 keeps f fixed across solve calls, so the checkpoints see one problem."""
    cfg = CONFIGS["rects128"]
    g, o = make_pair(E, cfg.W, cfg.H, data_mode=1, data_term=data_term)
    s = rects128.slice(0, 4 * cfg.packet)
    g.push(s.x, s.y, s.t, s.pol)
    o.push(s.x, s.y, s.t, s.pol)
    gaps = []
    done = 0
    for K in (10, 20, 40, 80, 160, 320):
        g.solve(K - done)
        done = K
        pr, du = g.gap()
        gaps.append(pr - du)
        # the oracle evaluates the same (u, p) with its own FP64 metric and f
        o.solve(0)
        o.set_up(g.state(E.EVR_STATE_U).astype(np.float64), g.p().astype(np.float64))
        opr, odu = o.energy()
        assert pr == pytest.approx(opr, rel=1e-5)
        assert du == pytest.approx(odu, rel=1e-5)
        assert pr - du >= -1e-6 * abs(pr)
    assert gaps[-1] < gaps[0]


# ----------------------------------------------------------------- full size
def test_full_size_blobs346_sampled_packets(E):
    """346 x 260, 1M events, 1000-event packets, 50 iterations, the solver the
    benchmark uses: every packet on the GPU, four of them teacher-forced against
    the oracle."""
    cfg = CONFIGS["blobs346"]
    st = make_stream(cfg)
    g, o = make_pair(E, cfg.W, cfg.H)
    sample = {0, 137, 500, cfg.n_packets - 1}
    worst = 0.0
    for k in range(cfg.n_packets):
        s = st.slice(k * cfg.packet, (k + 1) * cfg.packet)
        if k in sample:
            if k:  # the oracle's integer state follows the GPU's (both fresh at k = 0)
                oracle_follow_integer_state(E, g, o, cfg)
            worst = max(worst, teacher_forced_packet(E, g, o, s.x, s.y, s.t, s.pol, cfg.iters))
        else:
            assert g.push(s.x, s.y, s.t, s.pol) == 0
            g.solve(cfg.iters)
    assert worst <= TOL_U, worst
    u = g.image()
    assert np.all(np.isfinite(u)) and u.min() >= np.float32(np.exp(-3)) * 0.999999


def oracle_follow_integer_state(E, g, o, cfg):
    o.set(O.TLAST, g.state(E.EVR_STATE_TLAST))
    o.set(O.TREF, int(g.state(E.EVR_STATE_CLOCK)))
    o.set(O.TINIT, int(g.state(E.EVR_STATE_TINIT)))
    o.set(O.NPOS, np.zeros((cfg.H, cfg.W), np.int32))
    o.set(O.NNEG, np.zeros((cfg.H, cfg.W), np.int32))
