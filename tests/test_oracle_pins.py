"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
differential-geometry definitions of Sec. 3.1 evaluated with numpy's linear
algebra, exact identities (adjoint, duality), closed forms (Neumann-Laplacian
spectrum, prox root on perfect squares), brute-force scalar minimisation and an
independent Newton minimisation of the discrete energy (Eq. 5) on 8x8 images.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

TAU = 1.0 / math.sqrt(8.0 + 4.0 * math.sqrt(2.0))
UMIN, UMAX = math.exp(-3.0), math.exp(3.0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fwd(a):
    """Forward differences with zero last column / row, built with np.diff."""
    ax = np.zeros_like(a)
    ay = np.zeros_like(a)
    ax[:, :-1] = np.diff(a, axis=1)
    ay[:-1, :] = np.diff(a, axis=0)
    return ax, ay


def surface_frames(t):
    """phi_x, phi_y (Eq. 1 differentiated) and g (Eq. 2 as dot products), per pixel."""
    tx, ty = fwd(t)
    n = t.size
    phx = np.stack([np.ones(n), np.zeros(n), tx.ravel()], axis=1)
    phy = np.stack([np.zeros(n), np.ones(n), ty.ravel()], axis=1)
    g = np.empty((n, 2, 2))
    g[:, 0, 0] = np.einsum("ij,ij->i", phx, phx)
    g[:, 0, 1] = g[:, 1, 0] = np.einsum("ij,ij->i", phx, phy)
    g[:, 1, 1] = np.einsum("ij,ij->i", phy, phy)
    return phx, phy, g


# ----------------------------------------------------------------- geometry
@pytest.mark.parametrize("shape", [(6, 9), (1, 5), (5, 1), (2, 2)])
def test_metric_is_det_of_first_fundamental_form(shape):
    rng = np.random.default_rng(1)
    t = rng.normal(scale=2.0, size=shape)
    tx, ty, G = O.metric(t)
    _, _, g = surface_frames(t)
    np.testing.assert_allclose(G.ravel(), np.linalg.det(g), rtol=1e-13)
    ex, ey = fwd(t)
    np.testing.assert_array_equal(tx, ex)
    np.testing.assert_array_equal(ty, ey)


@pytest.mark.parametrize("shape", [(7, 5), (4, 11), (1, 6), (6, 1), (2, 2), (1, 1)])
def test_Lg_equals_pullback_gradient(shape):
    """Eq. 3 must be Eq. 4 (grad_g = (g^11 f_x + g^12 f_y) phi_x + (g^21 f_x + g^22 f_y)
    phi_y) evaluated with forward differences; g^-1 from numpy.linalg.inv."""
    rng = np.random.default_rng(2)
    t = rng.normal(scale=3.0, size=shape)
    u = rng.normal(size=shape)
    tx, ty, G = O.metric(t)
    got = O.Lg(tx, ty, G, u).reshape(3, -1).T
    phx, phy, g = surface_frames(t)
    gi = np.linalg.inv(g)
    ux, uy = fwd(u)
    gradu = np.stack([ux.ravel(), uy.ravel()], axis=1)
    c = np.einsum("nij,nj->ni", gi, gradu)
    want = c[:, :1] * phx + c[:, 1:] * phy
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


def test_Lg_norm_is_inverse_metric_quadratic_form():
    """|L_g u|^2 = grad u^T g^-1 grad u (M = J g^-1, J^T J = g)."""
    rng = np.random.default_rng(3)
    t = rng.normal(scale=5.0, size=(9, 8))
    u = rng.normal(size=(9, 8))
    tx, ty, G = O.metric(t)
    L = O.Lg(tx, ty, G, u).reshape(3, -1)
    _, _, g = surface_frames(t)
    ux, uy = fwd(u)
    a = np.stack([ux.ravel(), uy.ravel()], axis=1)
    q = np.einsum("ni,nij,nj->n", a, np.linalg.inv(g), a)
    np.testing.assert_allclose((L ** 2).sum(0), q, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("shape", [(8, 8), (13, 7), (1, 9), (9, 1), (2, 3), (1, 1)])
def test_adjoint_identity(shape):
    """<L_g u, p> = -<u, div_g p> (L_g^* in Eq. cont_iterates is the exact adjoint)."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        t = rng.normal(scale=4.0, size=shape)
        u = rng.normal(size=shape)
        p = rng.normal(size=(3,) + shape)
        tx, ty, G = O.metric(t)
        lhs = float(np.sum(O.Lg(tx, ty, G, u) * p))
        rhs = -float(np.sum(u * O.divg(tx, ty, G, p)))
        scale = float(np.sum(np.abs(O.Lg(tx, ty, G, u) * p))) + 1e-300
        assert abs(lhs - rhs) <= 1e-13 * scale


def _power_norm(tx, ty, G, iters=3000, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.normal(size=tx.shape)
    lam = 0.0
    for _ in range(iters):
        v = -O.divg(tx, ty, G, O.Lg(tx, ty, G, u))
        lam = float(np.sum(u * v) / np.sum(u * u))
        u = v / np.linalg.norm(v)
    return lam


def test_operator_norm_flat_matches_neumann_spectrum():
    """t = const: L_g^* L_g is the Neumann Laplacian, whose largest eigenvalue is
    4 cos^2(pi/2W) + 4 cos^2(pi/2H); it stays below the paper's bound 8 + 4 sqrt 2."""
    W, H = 12, 9
    z = np.zeros((H, W))
    tx, ty, G = O.metric(z)
    lam = _power_norm(tx, ty, G, iters=4000)
    exact = 4 * math.cos(math.pi / (2 * W)) ** 2 + 4 * math.cos(math.pi / (2 * H)) ** 2
    assert abs(lam - exact) < 1e-6
    assert lam <= 8.0 + 4.0 * math.sqrt(2.0)


def test_operator_norm_curved_below_eight():
    """M^T M = g^-1 <= I, so ||L_g||^2 <= ||grad||^2 <= 8 < 8 + 4 sqrt 2 (Sec. 3.2)."""
    rng = np.random.default_rng(5)
    for s in (0.3, 3.0, 30.0):
        t = rng.normal(scale=s, size=(10, 10))
        tx, ty, G = O.metric(t)
        assert _power_norm(tx, ty, G, iters=800, seed=1) <= 8.0 + 1e-9


# ----------------------------------------------------------------- proximal maps
def _golden_min(fun, a, b, tol=1e-14):
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = fun(c), fun(d)
    while b - a > tol * max(1.0, abs(a)):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = fun(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = fun(d)
    return 0.5 * (a + b)


def test_prox_kl_matches_scalar_minimisation():
    """prox of Eq. update_rules = argmin_u (u - v)^2/2 + beta (u - f log u) on the box."""
    rng = np.random.default_rng(6)
    for _ in range(300):
        v = rng.uniform(-30, 30)
        beta = 10 ** rng.uniform(-3, 3)
        f = 10 ** rng.uniform(-2, 1.5)
        want = _golden_min(lambda u: 0.5 * (u - v) ** 2 + beta * (u - f * math.log(u)),
                           UMIN, UMAX)
        got = O.prox_kl(v, beta, f, UMIN, UMAX)
        assert abs(got - want) <= 2e-7 * max(1.0, abs(want))
        if UMIN < got < UMAX:
            # stationarity: u^2 + (beta - v) u - beta f = 0
            assert abs(got * got + (beta - v) * got - beta * f) <= 1e-9 * (got * got + beta * f
                                                                         + abs(v * got))


def test_prox_kl_golden_cases():
    """Hand-solved roots of u^2 + (beta - v) u - beta f = 0 (perfect squares)."""
    with open(os.path.join(GOLDEN, "prox_kl_cases.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        got = O.prox_kl(c["v"], c["beta"], c["f"], c["u_min"], c["u_max"])
        assert got == pytest.approx(c["u"], rel=0, abs=1e-15), c


def test_projection_is_metric_ball_projection():
    """p / max(1, |p|/sqrt G) is the Euclidean projection onto {|q| <= sqrt G}:
    feasible, idempotent, identity inside, and <p - P(p), q - P(p)> <= 0 for q in the ball."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        sG = 10 ** rng.uniform(-0.0, 2.0)
        p = rng.normal(scale=sG * rng.uniform(0.1, 3.0), size=3)
        pp = O.project(p, sG)
        assert np.linalg.norm(pp) <= sG * (1 + 1e-15)
        np.testing.assert_allclose(O.project(pp, sG), pp, rtol=1e-15, atol=0)
        if np.linalg.norm(p) <= sG:
            np.testing.assert_array_equal(pp, p)
        for _ in range(5):
            q = rng.normal(size=3)
            q = q / np.linalg.norm(q) * sG * rng.uniform() ** (1 / 3)
            assert np.dot(p - pp, q - pp) <= 1e-12 * sG * sG


# ----------------------------------------------------------------- solver
def tv_kl_numpy(f, u, p2, K, tau, sigma, lam):
    """Ordinary TV-KL primal-dual (flat image domain, 2-vector dual), written
    independently of the oracle (Steidl-Teuber data term, Chambolle-Pock)."""
    u = u.copy()
    p = p2.copy()
    beta = tau * lam
    for _ in range(K):
        div = np.zeros_like(u)
        div[:, :-1] += p[0][:, :-1]
        div[:, 1:] -= p[0][:, :-1]
        div[:-1, :] += p[1][:-1, :]
        div[1:, :] -= p[1][:-1, :]
        v = u + tau * div
        un = np.clip(0.5 * (v - beta + np.sqrt((v - beta) ** 2 + 4 * beta * f)), UMIN, UMAX)
        ub = 2 * un - u
        gx, gy = fwd(ub)
        q = np.stack([p[0] + sigma * gx, p[1] + sigma * gy])
        nrm = np.maximum(1.0, np.sqrt(q[0] ** 2 + q[1] ** 2))
        p = q / nrm
        u = un
    return u, p


@pytest.mark.parametrize("shape", [(10, 14), (1, 8), (7, 1)])
def test_flat_manifold_is_standard_tv_kl(shape):
    """t = const gives g = I and TV_g = TV (Sec. 3.1 after Eq. regularisation_term)."""
    rng = np.random.default_rng(8)
    f = rng.uniform(0.2, 5.0, size=shape)
    u0 = rng.uniform(0.5, 2.0, size=shape)
    t = np.full(shape, 3.7)
    tx, ty, G = O.metric(t)
    p0 = np.zeros((3,) + shape)
    u, p = O.pd_iterations(tx, ty, G, f, u0, p0, 150, TAU, TAU, 2.0, UMIN, UMAX)
    ur, pr = tv_kl_numpy(f, u0, np.zeros((2,) + shape), 150, TAU, TAU, 2.0)
    np.testing.assert_allclose(u, ur, rtol=0, atol=1e-12)
    np.testing.assert_allclose(p[:2], pr, rtol=0, atol=1e-12)
    assert np.all(p[2] == 0.0)


def test_surface_orientation_does_not_change_the_image():
    """t and -t (time since last event vs. latest timestamp) give the same metric; L_g's
    third row flips sign, p3 with it, and u is bit-identical."""
    rng = np.random.default_rng(9)
    t = rng.uniform(0, 20, size=(9, 11))
    f = rng.uniform(0.3, 3.0, size=t.shape)
    u0 = np.ones_like(t)
    p0 = np.zeros((3,) + t.shape)
    a = O.metric(t)
    b = O.metric(-t)
    np.testing.assert_array_equal(a[2], b[2])
    ua, pa = O.pd_iterations(*a, f, u0, p0, 40, TAU, TAU, 90.0, UMIN, UMAX)
    ub, pb = O.pd_iterations(*b, f, u0, p0, 40, TAU, TAU, 90.0, UMIN, UMAX)
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(pa[2], -pb[2])


def test_constant_data_is_a_fixed_point():
    """Constant f inside the box: L_g f = 0 and the KL term is minimal at u = f."""
    rng = np.random.default_rng(10)
    t = rng.uniform(0, 50, size=(6, 7))
    tx, ty, G = O.metric(t)
    f = np.full(t.shape, 1.7)
    u, p = O.pd_iterations(tx, ty, G, f, f, np.zeros((3,) + t.shape), 25, TAU, TAU, 90.0,
                           UMIN, UMAX)
    # the root is evaluated with cancellation when beta >> f: rounding only
    np.testing.assert_allclose(u, f, rtol=0, atol=1e-12)
    assert np.max(np.abs(p)) < 1e-11


def test_huge_lambda_returns_clamped_data():
    """lambda -> infinity: u -> clamp(f), with an O(1/lambda) residual from the TV term."""
    rng = np.random.default_rng(11)
    t = rng.uniform(0, 5, size=(5, 6))
    tx, ty, G = O.metric(t)
    f = rng.uniform(0.01, 40.0, size=t.shape)
    errs = []
    for lam in (1e5, 1e6):
        u, _ = O.pd_iterations(tx, ty, G, f, np.ones_like(f), np.zeros((3,) + f.shape), 6,
                               TAU, TAU, lam, UMIN, UMAX)
        errs.append(np.max(np.abs(u - np.clip(f, UMIN, UMAX))))
    assert errs[1] < 1e-4
    assert 5.0 < errs[0] / errs[1] < 20.0


def test_single_pixel_converges_to_data():
    """1x1 image: no differences, p stays 0, u_{k+1} = prox(u_k) -> f."""
    f = np.array([[2.5]])
    z = np.zeros((1, 1))
    tx, ty, G = O.metric(z)
    u, p = O.pd_iterations(tx, ty, G, f, np.array([[1.0]]), np.zeros((3, 1, 1)), 500, TAU, TAU,
                           5.0, UMIN, UMAX)
    assert abs(u[0, 0] - 2.5) < 1e-12 and np.all(p == 0)


# ----------------------------------------------------------------- energy / duality
def energy_numpy(t, f, u, lam, eps=0.0):
    """Eq. 5 written with |L_g u| = sqrt(grad u^T g^-1 grad u) (independent of Eq. 3)."""
    _, _, g = surface_frames(t)
    sG = np.sqrt(np.linalg.det(g))
    ux, uy = fwd(u)
    a = np.stack([ux.ravel(), uy.ravel()], axis=1)
    q = np.einsum("ni,nij,nj->n", a, np.linalg.inv(g), a)
    return float(np.sum(sG * np.sqrt(q + eps * eps))
                 + lam * np.sum(sG * (u.ravel() - f.ravel() * np.log(u.ravel()))))


def test_primal_energy_matches_definition():
    rng = np.random.default_rng(12)
    t = rng.uniform(0, 4, size=(7, 9))
    f = rng.uniform(0.2, 3, size=t.shape)
    u = rng.uniform(UMIN, UMAX, size=t.shape)
    tx, ty, G = O.metric(t)
    pr, _ = O.energy(tx, ty, G, f, u, np.zeros((3,) + t.shape), 90.0, UMIN, UMAX)
    assert pr == pytest.approx(energy_numpy(t, f, u, 90.0), rel=1e-13)


def test_dual_value_matches_pixelwise_minimisation():
    """Dual function = sum over pixels of min_{u in box} a(u - f log u) - u div_g p."""
    rng = np.random.default_rng(13)
    t = rng.uniform(0, 4, size=(4, 5))
    tx, ty, G = O.metric(t)
    f = rng.uniform(0.2, 3, size=t.shape)
    p = rng.normal(scale=2.0, size=(3,) + t.shape)
    for i in range(t.size):  # make p feasible
        p[:, i // 5, i % 5] = O.project(p[:, i // 5, i % 5], math.sqrt(G.ravel()[i]))
    lam = 0.7
    _, du = O.energy(tx, ty, G, f, np.ones_like(f), p, lam, UMIN, UMAX)
    div = O.divg(tx, ty, G, p).ravel()
    acc = 0.0
    for i in range(t.size):
        a = lam * math.sqrt(G.ravel()[i])
        fi = f.ravel()[i]
        fun = lambda u: a * (u - fi * math.log(u)) - u * div[i]  # noqa: E731
        us = _golden_min(fun, UMIN, UMAX)
        acc += min(fun(us), fun(UMIN), fun(UMAX))
    assert du == pytest.approx(acc, rel=1e-10, abs=1e-10)


def test_weak_duality_random_pairs():
    rng = np.random.default_rng(14)
    for _ in range(20):
        t = rng.uniform(0, 10, size=(6, 6))
        tx, ty, G = O.metric(t)
        f = rng.uniform(0.1, 10, size=t.shape)
        u = rng.uniform(UMIN, UMAX, size=t.shape)
        p = rng.normal(size=(3, 6, 6)) * np.sqrt(G) / np.sqrt(3.0) * rng.uniform(0, 1)
        pr, du = O.energy(tx, ty, G, f, u, p, 90.0, UMIN, UMAX)
        assert pr - du >= -1e-9 * abs(pr)


def _newton_minimise(t, f, lam, eps_list=(1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12)):
    """Damped Newton on the smoothed Eq. 5 energy (sqrt(q + eps^2)), eps -> 0."""
    H, W = t.shape
    n = H * W
    _, _, g = surface_frames(t)
    gi = np.linalg.inv(g)
    sG = np.sqrt(np.linalg.det(g))
    Dx = np.zeros((n, n))
    Dy = np.zeros((n, n))
    for y in range(H):
        for x in range(W):
            i = y * W + x
            if x < W - 1:
                Dx[i, i], Dx[i, i + 1] = -1.0, 1.0
            if y < H - 1:
                Dy[i, i], Dy[i, i + W] = -1.0, 1.0
    fv = f.ravel()
    u = fv.copy()

    def fgh(u, eps, need_h=True):
        a = np.stack([Dx @ u, Dy @ u], axis=1)
        Aa = np.einsum("nij,nj->ni", gi, a)
        r = np.sqrt(np.einsum("ni,ni->n", a, Aa) + eps * eps)
        val = np.sum(sG * r) + lam * np.sum(sG * (u - fv * np.log(u)))
        w = sG / r
        grad = Dx.T @ (w * Aa[:, 0]) + Dy.T @ (w * Aa[:, 1]) + lam * sG * (1 - fv / u)
        if not need_h:
            return val, grad, None
        Hm = np.diag(lam * sG * fv / u ** 2)
        B = gi / r[:, None, None] - np.einsum("ni,nj->nij", Aa, Aa) / (r ** 3)[:, None, None]
        B *= sG[:, None, None]
        for (P, i), (Q, j) in [((Dx, 0), (Dx, 0)), ((Dx, 0), (Dy, 1)), ((Dy, 1), (Dx, 0)),
                               ((Dy, 1), (Dy, 1))]:
            Hm += P.T @ (B[:, i, j][:, None] * Q)
        return val, grad, Hm

    for eps in eps_list:
        for _ in range(100):
            val, grad, Hm = fgh(u, eps)
            step = np.linalg.solve(Hm, grad)
            s = 1.0
            while np.any(u - s * step <= 0) or fgh(u - s * step, eps, False)[0] > val:
                s *= 0.5
                if s < 1e-12:
                    break
            u = u - s * step
            if np.max(np.abs(s * step)) < 1e-15 * np.max(np.abs(u)):
                break
    return u.reshape(H, W), (Dx, Dy)


@pytest.mark.parametrize("surface", ["random", "ramp", "sine", "flat"])
def test_8x8_matches_independent_energy_minimisation(surface):
    """The K-step oracle reaches the minimiser of Eq. 5 found by Newton's method on
    the energy written from g^-1 (surfaces after Fig. 2: flat, ramp, sine)."""
    rng = np.random.default_rng({"random": 20, "ramp": 21, "sine": 22, "flat": 23}[surface])
    H = W = 8
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    t = {"random": rng.uniform(0, 3, (H, W)), "ramp": 0.8 * xx,
         "sine": 2.0 * np.sin(xx / 2.0) + 0.5 * np.cos(yy / 3.0), "flat": np.zeros((H, W))}[surface]
    f = rng.uniform(0.5, 2.0, (H, W))
    lam = 9.0
    un, (Dx, Dy) = _newton_minimise(t, f, lam)
    assert np.all((un > UMIN) & (un < UMAX))
    tx, ty, G = O.metric(t)
    u, p = O.pd_iterations(tx, ty, G, f, np.ones_like(f), np.zeros((3, H, W)), 20000, TAU, TAU,
                           lam, UMIN, UMAX)
    np.testing.assert_allclose(u, un, rtol=0, atol=1e-9)
    pr, du = O.energy(tx, ty, G, f, u, p, lam, UMIN, UMAX)
    en = energy_numpy(t, f, un, lam)
    assert pr == pytest.approx(en, rel=1e-9)
    assert abs(pr - du) <= 1e-9 * abs(pr)


def test_gap_shrinks_at_geometric_checkpoints():
    """Primal-dual gap at K = 10, 20, 40, ... on a fixed packet is non-negative and does
    not grow (Chambolle-Pock convergence; the paper's k <= 50 budget is a statistic)."""
    rng = np.random.default_rng(30)
    t = rng.uniform(0, 3, (24, 24))
    tx, ty, G = O.metric(t)
    f = np.exp(rng.normal(scale=0.4, size=t.shape))
    u, p = np.ones_like(f), np.zeros((3,) + f.shape)
    gaps = []
    done = 0
    for K in (10, 20, 40, 80, 160, 320, 640, 1280, 2560):
        u, p = O.pd_iterations(tx, ty, G, f, u, p, K - done, TAU, TAU, 90.0, UMIN, UMAX)
        done = K
        pr, du = O.energy(tx, ty, G, f, u, p, 90.0, UMIN, UMAX)
        gaps.append(pr - du)
    assert all(gp >= -1e-9 * abs(pr) for gp in gaps)
    assert all(b <= a * (1 + 1e-9) + 1e-9 for a, b in zip(gaps, gaps[1:]))
    assert gaps[-1] <= 1e-6 * gaps[0]
