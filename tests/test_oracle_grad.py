"""Pin of the oracle's reverse-mode derivative of the unrolled solve against FP64
central finite differences of the oracle's forward iterations."""
import math

import numpy as np
import pytest

from oracle import oracle as O

TAU = 1.0 / math.sqrt(8.0 + 4.0 * math.sqrt(2.0))
UMIN, UMAX = math.exp(-3.0), math.exp(3.0)


@pytest.mark.parametrize("shape,K,lam", [((6, 7), 12, 9.0), ((1, 9), 8, 30.0), ((5, 1), 5, 2.0),
                                         ((8, 8), 25, 90.0)])
def test_adjoint_matches_central_differences(shape, K, lam):
    rng = np.random.default_rng(sum(shape) + K)
    H, W = shape
    t = rng.uniform(0, 3, shape)
    tx, ty, G = O.metric(t)
    f = rng.uniform(0.5, 2.0, shape)
    u0 = rng.uniform(0.5, 2.0, shape)
    p0 = rng.normal(scale=0.3, size=(3,) + shape)
    w = rng.normal(size=shape)

    def loss(f_, u0_, p0_, lam_):
        u, _ = O.pd_iterations(tx, ty, G, f_, u0_, p0_, K, TAU, TAU, lam_, UMIN, UMAX)
        return float(np.sum(w * u))

    gu0, gp0, gf, gl = O.pd_grad(tx, ty, G, f, u0, p0, K, TAU, TAU, lam, UMIN, UMAX, w)
    h = 1e-6
    fd = (loss(f, u0, p0, lam + h) - loss(f, u0, p0, lam - h)) / (2 * h)
    assert gl == pytest.approx(fd, rel=1e-5, abs=1e-8)
    for _ in range(6):
        i, j = rng.integers(0, H), rng.integers(0, W)
        e = np.zeros(shape)
        e[i, j] = h
        fd_f = (loss(f + e, u0, p0, lam) - loss(f - e, u0, p0, lam)) / (2 * h)
        fd_u = (loss(f, u0 + e, p0, lam) - loss(f, u0 - e, p0, lam)) / (2 * h)
        assert gf[i, j] == pytest.approx(fd_f, rel=1e-5, abs=1e-8)
        assert gu0[i, j] == pytest.approx(fd_u, rel=1e-5, abs=1e-8)
        c = rng.integers(0, 3)
        E = np.zeros((3,) + shape)
        E[c, i, j] = h
        fd_p = (loss(f, u0, p0 + E, lam) - loss(f, u0, p0 - E, lam)) / (2 * h)
        assert gp0[c, i, j] == pytest.approx(fd_p, rel=1e-5, abs=1e-8)


def test_adjoint_of_zero_iterations_is_identity():
    rng = np.random.default_rng(3)
    t = rng.uniform(0, 3, (4, 5))
    tx, ty, G = O.metric(t)
    f = rng.uniform(0.5, 2, (4, 5))
    w = rng.normal(size=(4, 5))
    gu0, gp0, gf, gl = O.pd_grad(tx, ty, G, f, f, np.zeros((3, 4, 5)), 0, TAU, TAU, 9.0, UMIN,
                                 UMAX, w)
    np.testing.assert_array_equal(gu0, w)
    assert np.all(gp0 == 0) and np.all(gf == 0) and gl == 0.0
