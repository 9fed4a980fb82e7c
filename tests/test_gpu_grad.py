"""Differentiation of one packet's solve on the GPU (adjoint kernels through the C ABI,
behind torch.autograd.Function), against the FP64 oracle's adjoint and FP64 central
finite differences of the oracle's forward iterations."""
import math

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

TAU = float(np.float32(1.0 / math.sqrt(8.0 + 4.0 * math.sqrt(2.0))))
UMIN, UMAX = float(np.float32(math.exp(-3.0))), float(np.float32(math.exp(3.0)))
# FP32 forward/adjoint through K iterations against FP64: relative to the largest entry
GRAD_RTOL = 2e-3


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_06283_gb300 import build
    build.build()
    from paper_1607_06283_gb300 import autograd, evr
    return torch, autograd, evr


def problem(seed, H, W, tscale=3.0):
    rng = np.random.default_rng(seed)
    t = rng.uniform(0, tscale, (H, W)).astype(np.float32)
    tx = np.zeros((H, W), np.float32)
    ty = np.zeros((H, W), np.float32)
    tx[:, :-1] = np.diff(t, axis=1)
    ty[:-1, :] = np.diff(t, axis=0)
    f = rng.uniform(0.5, 2.0, (H, W)).astype(np.float32)
    u0 = rng.uniform(0.5, 2.0, (H, W)).astype(np.float32)
    p0 = (rng.normal(scale=0.3, size=(3, H, W))).astype(np.float32)
    w = rng.normal(size=(H, W)).astype(np.float32)
    return tx, ty, f, u0, p0, w


def oracle_metric(tx, ty):
    tx = tx.astype(np.float64)
    ty = ty.astype(np.float64)
    return tx, ty, 1.0 + tx * tx + ty * ty


def cuda(torch, *arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-30, np.max(np.abs(b))))


# widths that are a multiple of 4 (rows of a multiple of 16 bytes) take the reverse pass
# that stages its tape slots with tensor copies; the others read the tape directly
@pytest.mark.parametrize("H,W,K,every,lam", [(23, 37, 30, 10, 9.0), (40, 33, 30, 7, 90.0),
                                             (1, 50, 12, 5, 20.0), (17, 1, 9, 2, 20.0),
                                             (29, 36, 30, 10, 30.0), (33, 64, 23, 6, 90.0),
                                             (1, 8, 9, 3, 20.0)])
def test_forward_and_gradients_match_oracle(T, H, W, K, every, lam):
    torch, AG, E = T
    tx, ty, f, u0, p0, w = problem(H * 100 + W, H, W)
    ttx, tty, tf, tu0, tp0, tw = cuda(torch, tx, ty, f, u0, p0, w)
    tf.requires_grad_(True)
    tu0.requires_grad_(True)
    tp0.requires_grad_(True)
    tlam = torch.tensor(lam, dtype=torch.float32, device="cuda", requires_grad=True)
    u, p = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
    loss = (u * tw).sum()
    loss.backward()
    otx, oty, oG = oracle_metric(tx, ty)
    uo, po = O.pd_iterations(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX)
    assert np.max(np.abs(u.detach().cpu().numpy() - uo)) <= 1e-4
    gu0, gp0, gf, gl = O.pd_grad(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX, w)
    assert rel_err(tf.grad.cpu().numpy(), gf) <= GRAD_RTOL
    assert rel_err(tu0.grad.cpu().numpy(), gu0) <= GRAD_RTOL
    assert rel_err(tp0.grad.cpu().numpy(), gp0) <= GRAD_RTOL
    assert float(tlam.grad) == pytest.approx(gl, rel=GRAD_RTOL, abs=1e-6)


def test_checkpoint_spacing_does_not_change_gradients(T):
    torch, AG, E = T
    H, W, K = 31, 29, 24
    tx, ty, f, u0, p0, w = problem(5, H, W)
    ttx, tty, tu0, tp0, tw = cuda(torch, tx, ty, u0, p0, w)
    grads = []
    for every in (1, 3, 8, 24, 100):
        tf = torch.from_numpy(f).cuda().requires_grad_(True)
        tlam = torch.tensor(30.0, device="cuda", requires_grad=True)
        u, _ = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
        (u * tw).sum().backward()
        grads.append((tf.grad.cpu().numpy(), float(tlam.grad)))
    for gf, gl in grads[1:]:
        np.testing.assert_array_equal(gf, grads[0][0])
        assert gl == grads[0][1]


def test_contrast_threshold_and_lambda_against_finite_differences(T):
    """dL/dC and dL/dlambda of L = sum w * u_K with f = u_prev exp(C (n+ - n-)), against
    FP64 central differences of the oracle forward."""
    torch, AG, E = T
    H, W, K = 24, 30, 30
    rng = np.random.default_rng(9)
    tx, ty, _, u0, p0, w = problem(9, H, W)
    u_prev = rng.uniform(0.5, 2.0, (H, W)).astype(np.float32)
    npos = rng.poisson(0.6, (H, W)).astype(np.int32)
    nneg = rng.poisson(0.6, (H, W)).astype(np.int32)
    C0, lam0 = 0.15, 40.0
    ttx, tty, tu0, tp0, tw, tup, tnp, tnn = cuda(torch, tx, ty, u0, p0, w, u_prev, npos, nneg)
    tC = torch.tensor(C0, device="cuda", requires_grad=True)
    tlam = torch.tensor(lam0, device="cuda", requires_grad=True)
    f = AG.data_image(tup, tnp, tnn, tC, tC)
    u, _ = AG.packet_solve(f, tlam, tu0, tp0, ttx, tty, K, 10)
    (u * tw).sum().backward()
    otx, oty, oG = oracle_metric(tx, ty)

    def L(C, lam):
        fo = u_prev.astype(np.float64) * np.exp(C * (npos - nneg))
        uo, _ = O.pd_iterations(otx, oty, oG, fo, u0, p0, K, TAU, TAU, lam, UMIN, UMAX)
        return float(np.sum(w * uo))

    h = 1e-5
    dC = (L(C0 + h, lam0) - L(C0 - h, lam0)) / (2 * h)
    dl = (L(C0, lam0 + h) - L(C0, lam0 - h)) / (2 * h)
    assert float(tC.grad) == pytest.approx(dC, rel=GRAD_RTOL)
    assert float(tlam.grad) == pytest.approx(dl, rel=GRAD_RTOL, abs=1e-6)


def test_fit_lambda_and_threshold_to_target(T):
    """Gradient descent through the GPU adjoint moves (lambda, C) towards the values
    that produced a target image and lowers the loss."""
    torch, AG, E = T
    H, W, K = 32, 40, 30
    rng = np.random.default_rng(21)
    tx, ty, _, u0, _, _ = problem(21, H, W, tscale=1.0)
    u_prev = rng.uniform(0.6, 1.6, (H, W)).astype(np.float32)
    npos = rng.poisson(1.0, (H, W)).astype(np.int32)
    nneg = rng.poisson(1.0, (H, W)).astype(np.int32)
    p0 = np.zeros((3, H, W), np.float32)
    ttx, tty, tu0, tp0, tup, tnp, tnn = cuda(torch, tx, ty, u0, p0, u_prev, npos, nneg)
    with torch.no_grad():
        target, _ = AG.packet_solve(AG.data_image(tup, tnp, tnn, 0.2, 0.2), 25.0, tu0, tp0, ttx,
                                    tty, K, 10)
    logl = torch.tensor(math.log(60.0), device="cuda", requires_grad=True)
    C = torch.tensor(0.1, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([logl, C], lr=0.05)
    losses = []
    for _ in range(60):
        opt.zero_grad()
        u, _ = AG.packet_solve(AG.data_image(tup, tnp, tnn, C, C), logl.exp(), tu0, tp0, ttx,
                               tty, K, 10)
        loss = ((u - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.05 * losses[0]
    c_fit, l_fit = float(C.detach()), float(logl.detach().exp())
    assert abs(c_fit - 0.2) < abs(0.1 - 0.2) * 0.5
    assert abs(math.log(l_fit / 25.0)) < abs(math.log(60.0 / 25.0))


def test_diff64_shape_gradients_match_oracle(T):
    """The differentiation workload's shape: 64 stacked 240 x 180 packets, 30 unrolled
    iterations, checkpoints every 10.  Two members' dL/df and dL/du0 against the FP64
    oracle adjoint of those members alone, and dL/dlambda summed over all 64 members
    against the sum of the oracle's."""
    torch, AG, E = T
    n, H, W, K, every, lam = 64, 180, 240, 30, 10, 90.0
    probs = [problem(5000 + b, H, W) for b in range(n)]
    stk = [np.stack([pr[k] for pr in probs]) for k in range(6)]
    ttx, tty, tf, tu0, tp0, tw = cuda(torch, *stk)
    tf.requires_grad_(True)
    tu0.requires_grad_(True)
    tlam = torch.tensor(lam, dtype=torch.float32, device="cuda", requires_grad=True)
    u, _ = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
    (u * tw).sum().backward()
    gl_sum = 0.0
    for b, (tx, ty, f, u0, p0, w) in enumerate(probs):
        otx, oty, oG = oracle_metric(tx, ty)
        gu0, _, gf, gl = O.pd_grad(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX, w)
        gl_sum += gl
        if b in (0, n - 1):
            uo, _ = O.pd_iterations(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX)
            assert np.max(np.abs(u[b].detach().cpu().numpy() - uo)) <= 1e-4
            assert rel_err(tf.grad[b].cpu().numpy(), gf) <= GRAD_RTOL, b
            assert rel_err(tu0.grad[b].cpu().numpy(), gu0) <= GRAD_RTOL, b
    assert float(tlam.grad) == pytest.approx(gl_sum, rel=GRAD_RTOL, abs=1e-6)


def test_fit_to_ground_truth_frames_of_a_simulated_scene(T):
    """(lambda, C) fitted by gradient descent through the GPU adjoint to the simulator's
    ground-truth frames of a rectangles scene: each packet starts from the true image at
    its first event, its events give f = u_prev exp(C (n+ - n-)) and the metric, and the
    loss is the mean square error against the true image at its last event.  The loss
    falls and the fitted contrast threshold moves towards the simulator's C = 0.15."""
    torch, AG, E = T
    from evsim.configs import StreamConfig, make_stream
    W, H, K, per, n_pk = 64, 48, 30, 1500, 4
    cfg = StreamConfig("fit", W, H, "rects", 8, 4242, per * (n_pk + 1), per, K, speed=60.0,
                       noise=0.0, dt_us=100.0)
    st = make_stream(cfg)
    o = O.OracleStream(W, H)
    items = []
    a0 = per  # the first packet sets the time surface up
    s = st.slice(0, a0)
    assert o.push(s.x, s.y, s.t, s.pol) == 0
    o.solve(0)
    L0 = st.log_frame(float(st.t[0]))
    for k in range(n_pk):
        a, b = a0 + k * per, a0 + (k + 1) * per
        s = st.slice(a, b)
        assert o.push(s.x, s.y, s.t, s.pol) == 0
        npos, nneg = o.get(O.NPOS).copy(), o.get(O.NNEG).copy()
        o.solve(0)  # metric of this packet (oracle prologue)
        u_prev = np.exp(st.log_frame(float(st.t[a])) - L0)
        target = np.exp(st.log_frame(float(st.t[b - 1])) - L0)
        items.append((u_prev, npos, nneg, o.get(O.TX), o.get(O.TY), target))
    u_prev, npos, nneg, tx, ty, target = [
        torch.from_numpy(np.ascontiguousarray(np.stack([it[j] for it in items]).astype(
            np.int32 if j in (1, 2) else np.float32))).cuda() for j in range(6)]
    p0 = torch.zeros((n_pk, 3, H, W), device="cuda")
    logl = torch.tensor(math.log(30.0), device="cuda", requires_grad=True)
    C = torch.tensor(0.06, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([logl, C], lr=0.03)
    losses, cs = [], []
    for _ in range(80):
        opt.zero_grad()
        f = AG.data_image(u_prev, npos, nneg, C, C)
        u, _ = AG.packet_solve(f, logl.exp(), u_prev, p0, tx, ty, K, 10)
        loss = ((u - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
        cs.append(float(C.detach()))
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    assert abs(cs[-1] - 0.15) < 0.5 * abs(0.06 - 0.15), cs[-1]


def test_batched_solve_equals_single_solves_bit_for_bit(T):
    """n packets in one call: each image's forward state and every gradient are those of
    the same packet solved alone; dL/dlambda is the sum over the batch."""
    torch, AG, E = T
    n, H, W, K, every, lam = 5, 19, 23, 21, 6, 35.0
    probs = [problem(700 + b, H, W) for b in range(n)]
    single = []
    for tx, ty, f, u0, p0, w in probs:
        ttx, tty, tf, tu0, tp0, tw = cuda(torch, tx, ty, f, u0, p0, w)
        for t in (tf, tu0, tp0):
            t.requires_grad_(True)
        tlam = torch.tensor(lam, device="cuda", requires_grad=True)
        u, p = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
        ((u * tw).sum() + 0.1 * p.sum()).backward()
        single.append([a.detach().cpu().numpy() for a in (u, p, tf.grad, tu0.grad, tp0.grad)] +
                      [float(tlam.grad)])
    stk = [np.stack([pr[k] for pr in probs]) for k in range(6)]
    ttx, tty, tf, tu0, tp0, tw = cuda(torch, *stk)
    for t in (tf, tu0, tp0):
        t.requires_grad_(True)
    tlam = torch.tensor(lam, device="cuda", requires_grad=True)
    u, p = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
    assert u.shape == (n, H, W) and p.shape == (n, 3, H, W)
    ((u * tw).sum() + 0.1 * p.sum()).backward()
    got = [a.detach().cpu().numpy() for a in (u, p, tf.grad, tu0.grad, tp0.grad)]
    for b in range(n):
        for k in range(5):
            np.testing.assert_array_equal(got[k][b], single[b][k], err_msg=f"image {b} out {k}")
    assert float(tlam.grad) == pytest.approx(sum(s[5] for s in single), rel=1e-5)


def test_mixed_size_members_equal_their_own_calls(T):
    """packet_solve_many groups members by size (one library call per size); every
    member's forward result and gradients are those of its own call, and dL/dlambda is
    the sum over the members."""
    torch, AG, E = T
    K, every, lam = 17, 5, 30.0
    shapes = [(19, 23), (12, 40), (19, 23), (12, 40), (19, 23)]
    probs = [problem(900 + b, H, W) for b, (H, W) in enumerate(shapes)]
    single = []
    for tx, ty, f, u0, p0, w in probs:
        ttx, tty, tf, tu0, tp0, tw = cuda(torch, tx, ty, f, u0, p0, w)
        tf.requires_grad_(True)
        tlam = torch.tensor(lam, device="cuda", requires_grad=True)
        u, p = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, every)
        (u * tw).sum().backward()
        single.append((u.detach().cpu().numpy(), tf.grad.cpu().numpy(), float(tlam.grad)))
    members, ws, fs = [], [], []
    for tx, ty, f, u0, p0, w in probs:
        ttx, tty, tf, tu0, tp0, tw = cuda(torch, tx, ty, f, u0, p0, w)
        tf.requires_grad_(True)
        members.append((tf, tu0, tp0, ttx, tty))
        ws.append(tw)
        fs.append(tf)
    tlam = torch.tensor(lam, device="cuda", requires_grad=True)
    res = AG.packet_solve_many(members, tlam, K, every)
    sum((u * w).sum() for (u, _), w in zip(res, ws)).backward()
    for b, ((u, _), tf) in enumerate(zip(res, fs)):
        np.testing.assert_array_equal(u.detach().cpu().numpy(), single[b][0])
        np.testing.assert_array_equal(tf.grad.cpu().numpy(), single[b][1])
    assert float(tlam.grad) == pytest.approx(sum(s[2] for s in single), rel=1e-5)


def test_batched_gradients_match_oracle_on_a_ragged_member(T):
    """A batch of 3 images of 1 row each (every row is a member's first and last row):
    no y-coupling between members, gradients against the FP64 oracle per member."""
    torch, AG, E = T
    n, H, W, K, lam = 3, 1, 41, 15, 20.0
    probs = [problem(800 + b, H, W) for b in range(n)]
    stk = [np.stack([pr[k] for pr in probs]) for k in range(6)]
    ttx, tty, tf, tu0, tp0, tw = cuda(torch, *stk)
    tf.requires_grad_(True)
    tlam = torch.tensor(lam, device="cuda", requires_grad=True)
    u, _ = AG.packet_solve(tf, tlam, tu0, tp0, ttx, tty, K, 4)
    (u * tw).sum().backward()
    gl_sum = 0.0
    for b, (tx, ty, f, u0, p0, w) in enumerate(probs):
        otx, oty, oG = oracle_metric(tx, ty)
        uo, _ = O.pd_iterations(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX)
        assert np.max(np.abs(u[b].detach().cpu().numpy() - uo)) <= 1e-4
        _, _, gf, gl = O.pd_grad(otx, oty, oG, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX, w)
        assert rel_err(tf.grad[b].cpu().numpy(), gf) <= GRAD_RTOL
        gl_sum += gl
    assert float(tlam.grad) == pytest.approx(gl_sum, rel=GRAD_RTOL, abs=1e-6)


def test_batched_call_rejects_bad_sizes(T):
    torch, AG, E = T
    assert E._lib.evr_unrolled_workspace_bytes(16, 8, 16, 0, 10, 5) == 0
    assert E._lib.evr_unrolled_workspace_bytes(16, 8, 16, 70000, 10, 5) == 0
    assert E._lib.evr_unrolled_workspace_bytes(16, 8, 16, 4, 10, 5) > 0


def test_launch_timing_counts_every_launch(T):
    """evr_unrolled_timing_start/stop: every kernel of the differentiation calls counted,
    every reverse-pass launch timed (each reverses at most a few iterations)."""
    torch, AG, E = T
    H, W, K, every = 23, 37, 30, 10
    segs = K // every
    tx, ty, f, u0, p0, w = problem(11, H, W)
    ttx, tty, tf, tu0, tp0, tw = cuda(torch, tx, ty, f, u0, p0, w)
    tf.requires_grad_(True)
    E.evr_unrolled_timing_start()
    u, _ = AG.packet_solve(tf, 30.0, tu0, tp0, ttx, tty, K, every)
    torch.cuda.synchronize()
    *_, fwd = E.evr_unrolled_timing_stop()
    # forward: metric, 4 copies (checkpoint 0), then the same number of passes per segment
    passes, rem = divmod(fwd - 5, segs)
    assert rem == 0 and every // 8 <= passes <= every
    E.evr_unrolled_timing_start()
    (u * tw).sum().backward()
    ms, n_rev, px_iters, px_launches, bwd = E.evr_unrolled_timing_stop()
    assert n_rev % segs == 0 and every // 8 <= n_rev // segs <= every
    assert px_iters == H * W * K and px_launches == H * W * n_rev
    # backward: metric, zero, the replay passes of all but the last segment (the forward
    # wrote its tape), the reverse launches, dL/dp0, the two-stage lambda reduction
    assert bwd == 2 + (segs - 1) * passes + n_rev + 1 + 2
    assert ms > 0.0


def test_backward_can_repeat(T):
    """The backward leaves the checkpoints and the forward's tape intact: a second
    backward through the same graph gives the same gradients bit for bit."""
    torch, AG, E = T
    H, W, K, every = 21, 19, 25, 7
    tx, ty, f, u0, p0, w = problem(13, H, W)
    ttx, tty, tu0, tp0, tw = cuda(torch, tx, ty, u0, p0, w)
    tf = torch.from_numpy(f).cuda().requires_grad_(True)
    u, _ = AG.packet_solve(tf, 30.0, tu0, tp0, ttx, tty, K, every)
    loss = (u * tw).sum()
    loss.backward(retain_graph=True)
    g1 = tf.grad.clone()
    tf.grad = None
    loss.backward()
    assert torch.equal(tf.grad, g1)
