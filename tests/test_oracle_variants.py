"""Pins of the oracle's model variants: the L2 data term of Eq. 7 (ROF on the event
manifold, Fig. 2) and the TV-L1 denoising of the time surface (Sec. 4)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_pins import (TAU, UMAX, UMIN, _golden_min, fwd, surface_frames)


def test_prox_l2_matches_scalar_minimisation():
    rng = np.random.default_rng(1)
    for _ in range(200):
        v, beta, f = rng.uniform(-5, 5), 10 ** rng.uniform(-3, 3), rng.uniform(-3, 3)
        want = _golden_min(lambda u: 0.5 * (u - v) ** 2 + 0.5 * beta * (u - f) ** 2,
                           -50.0, 50.0)
        assert O.prox_l2(v, beta, f) == pytest.approx(want, abs=1e-7)


def rof_numpy(f, u, K, tau, sigma, lam):
    """Standard ROF primal-dual on the image domain, written independently."""
    u = u.copy()
    p = np.zeros((2,) + f.shape)
    for _ in range(K):
        div = np.zeros_like(u)
        div[:, :-1] += p[0][:, :-1]
        div[:, 1:] -= p[0][:, :-1]
        div[:-1, :] += p[1][:-1, :]
        div[1:, :] -= p[1][:-1, :]
        v = u + tau * div
        un = (v + tau * lam * f) / (1 + tau * lam)
        gx, gy = fwd(2 * un - u)
        q = np.stack([p[0] + sigma * gx, p[1] + sigma * gy])
        p = q / np.maximum(1.0, np.sqrt(q[0] ** 2 + q[1] ** 2))
        u = un
    return u


def test_rof_flat_manifold_is_standard_rof():
    rng = np.random.default_rng(2)
    f = rng.normal(size=(9, 13))
    tx, ty, G = O.metric(np.full(f.shape, 2.0))
    u, p = O.pd_iterations_dt(tx, ty, G, f, np.zeros_like(f), np.zeros((3,) + f.shape), 120,
                              TAU, TAU, 3.0, UMIN, UMAX, 1)
    np.testing.assert_allclose(u, rof_numpy(f, np.zeros_like(f), 120, TAU, TAU, 3.0), atol=1e-12)


def _newton_rof(t, f, lam, eps_list=(1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12)):
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

    def fgh(u, eps):
        a = np.stack([Dx @ u, Dy @ u], axis=1)
        Aa = np.einsum("nij,nj->ni", gi, a)
        r = np.sqrt(np.einsum("ni,ni->n", a, Aa) + eps * eps)
        val = np.sum(sG * r) + 0.5 * lam * np.sum(sG * (u - fv) ** 2)
        w = sG / r
        grad = Dx.T @ (w * Aa[:, 0]) + Dy.T @ (w * Aa[:, 1]) + lam * sG * (u - fv)
        Hm = np.diag(lam * sG)
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
            while fgh(u - s * step, eps)[0] > val and s > 1e-12:
                s *= 0.5
            u = u - s * step
            if np.max(np.abs(s * step)) < 1e-15 * max(1.0, np.max(np.abs(u))):
                break
    return u.reshape(H, W)


@pytest.mark.parametrize("surface", ["ramp", "sine"])
def test_rof_8x8_matches_newton(surface):
    """Eq. 7 on 8x8 images with the ramp and sine surfaces of Fig. 2."""
    rng = np.random.default_rng(3)
    yy, xx = np.mgrid[0:8, 0:8].astype(float)
    t = 0.8 * xx if surface == "ramp" else 2.0 * np.sin(xx / 2.0) + 0.5 * np.cos(yy / 3.0)
    f = rng.normal(size=(8, 8))
    lam = 4.0
    un = _newton_rof(t, f, lam)
    tx, ty, G = O.metric(t)
    u, p = O.pd_iterations_dt(tx, ty, G, f, np.zeros_like(f), np.zeros((3, 8, 8)), 20000, TAU,
                              TAU, lam, UMIN, UMAX, 1)
    np.testing.assert_allclose(u, un, atol=1e-8)
    pr, du = O.energy_l2(tx, ty, G, f, u, p, lam)
    assert abs(pr - du) <= 1e-9 * abs(pr)


def test_rof_ramp_regularises_along_the_level_lines():
    """Fig. 2(b): on a ramp t = c x the surface gradient is zero in y, so TV_g penalises
    y-variation sqrt(1 + c^2) times more than x-variation: ROF denoising of noise leaves
    more variation along x than along y."""
    rng = np.random.default_rng(4)
    H = W = 48
    yy, xx = np.mgrid[0:H, 0:W].astype(float)
    f = rng.normal(size=(H, W))
    tx, ty, G = O.metric(3.0 * xx)
    u, _ = O.pd_iterations_dt(tx, ty, G, f, f, np.zeros((3, H, W)), 400, TAU, TAU, 2.0, UMIN,
                              UMAX, 1)
    gx, gy = fwd(u)
    assert np.mean(np.abs(gx[:, :-1])) > 1.3 * np.mean(np.abs(gy[:-1, :]))
    tx0, ty0, G0 = O.metric(np.zeros((H, W)))
    u0, _ = O.pd_iterations_dt(tx0, ty0, G0, f, f, np.zeros((3, H, W)), 400, TAU, TAU, 2.0,
                               UMIN, UMAX, 1)
    gx0, gy0 = fwd(u0)
    assert 0.8 < np.mean(np.abs(gx0[:, :-1])) / np.mean(np.abs(gy0[:-1, :])) < 1.25


# ----------------------------------------------------------------- TV-L1
def test_tvl1_constant_is_fixed_point():
    t = np.full((7, 9), 12.5)
    np.testing.assert_array_equal(O.tvl1(t, 50, 1.0), t)


@pytest.mark.parametrize("lam,kept", [(2.0, False), (6.0, True)])
def test_tvl1_single_pixel_spike_threshold(lam, kept):
    """Anisotropic TV of a height-h one-pixel spike is 4h (four forward differences)
    and its data cost lam h: the minimiser removes it for lam < 4 and keeps it above."""
    t = np.zeros((9, 9))
    t[4, 4] = 10.0
    s = O.tvl1(t, 4000, lam)
    assert abs(s[4, 4] - (10.0 if kept else 0.0)) < 1e-3
    assert np.max(np.abs(np.delete(s.ravel(), 40))) < 1e-3


def _tvl1_energy(s, t0, lam):
    gx, gy = fwd(s)
    return float(np.sum(np.abs(gx)) + np.sum(np.abs(gy)) + lam * np.sum(np.abs(s - t0)))


def test_tvl1_reaches_the_linear_programme_optimum():
    """min sum |L_x s| + |L_y s| + lam |s - t0| is a linear programme; its optimum value
    (scipy linprog) is what the oracle's iterations approach."""
    sp = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(5)
    H, W, lam = 5, 6, 0.7
    t0 = rng.uniform(0, 10, (H, W))
    n = H * W
    rows = []
    for y in range(H):
        for x in range(W):
            i = y * W + x
            if x < W - 1:
                rows.append((i, i + 1))
            if y < H - 1:
                rows.append((i, i + W))
    m = len(rows)
    # variables: s (n), a_k >= |s_j - s_i| (m), b_i >= |s_i - t0_i| (n)
    c = np.concatenate([np.zeros(n), np.ones(m), lam * np.ones(n)])
    A, bvec = [], []
    for k, (i, j) in enumerate(rows):
        for sgn in (1, -1):
            r = np.zeros(2 * n + m)
            r[j], r[i], r[n + k] = sgn, -sgn, -1
            A.append(r)
            bvec.append(0.0)
    for i in range(n):
        for sgn in (1, -1):
            r = np.zeros(2 * n + m)
            r[i], r[n + m + i] = sgn, -1
            A.append(r)
            bvec.append(sgn * t0.ravel()[i])
    res = sp.linprog(c, A_ub=np.array(A), b_ub=np.array(bvec),
                     bounds=[(None, None)] * n + [(0, None)] * (m + n), method="highs")
    assert res.status == 0
    s = O.tvl1(t0, 20000, lam)
    assert _tvl1_energy(s, t0, lam) == pytest.approx(res.fun, rel=1e-6)


def test_stream_with_denoised_surface_and_l2_term():
    """Stream level: the solve uses TV-L1 of the raw time surface, then the metric."""
    rng = np.random.default_rng(6)
    W, H = 12, 10
    raw = O.OracleStream(W, H)
    den = O.OracleStream(W, H, O.OracleParams(tvl1_iters=30, tvl1_lambda=1.5, data_term=1))
    x = rng.integers(0, W, 200).astype(np.uint16)
    y = rng.integers(0, H, 200).astype(np.uint16)
    t = (1000 + np.sort(rng.integers(0, 50_000, 200))).astype(np.int64)
    p = rng.choice(np.array([-1, 1], np.int8), 200)
    for s in (raw, den):
        assert s.push(x, y, t, p) == 0
        s.solve(5)
    np.testing.assert_allclose(den.get(O.TAU), O.tvl1(raw.get(O.TAU), 30, 1.5), rtol=0,
                               atol=1e-12)
    tx, ty, G = O.metric(den.get(O.TAU))
    np.testing.assert_allclose(den.get(O.G), G, rtol=1e-15)
