"""Pins for the constant disturbance w_d of Eq. first_order_integration in
the oracle's condensed form, adjoint and closed loop.  The rollout with w_d
is pinned to the closed form in test_oracle_model.py; here the other
functions are pinned to that rollout (the condensed form and the adjoint
reproduce its cost and its central differences) and the loop to a plant
whose states have a closed form."""
import numpy as np

import oracle as O
import workloads as W
from helpers import oracle_model


def _model_with_w(seed=0, T=40, p=5):
    wl = W.small(dof=3, T=T, p=p, P=40, E=4)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    rng = np.random.default_rng(seed)
    w = 0.05 * rng.standard_normal(wl.n)
    b = wl.bounds()
    return wl, O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p, w=w), rng


def test_condensed_form_carries_the_disturbance():
    wl, M, rng = _model_with_w(1)
    x0, g = wl.start_goal()
    H, f, c0 = M.condensed(x0, g)
    H0, f0, c00 = oracle_model(wl).condensed(x0, g)
    np.testing.assert_allclose(H, H0, rtol=1e-13, atol=1e-15)  # w_d is affine: H unchanged
    assert np.abs(f - f0).max() > 0
    for _ in range(5):
        U = rng.uniform(-1, 1, wl.m * wl.p)
        np.testing.assert_allclose(M.cost(x0, g, U), U @ H @ U + 2 * f @ U + c0, rtol=1e-11)


def test_adjoint_with_disturbance_matches_central_differences():
    wl, M, rng = _model_with_w(2, T=30, p=4)
    x0, g = wl.start_goal()
    h = 1e-6
    for _ in range(3):
        U = rng.uniform(-1, 1, wl.m * wl.p)
        J, gr = M.grad(x0, g, U)
        assert abs(J - M.cost(x0, g, U)) <= 1e-13 * abs(J)
        fd = np.zeros_like(U)
        for q in range(U.size):
            e = np.zeros_like(U)
            e[q] = h
            fd[q] = (M.cost(x0, g, U + e) - M.cost(x0, g, U - e)) / (2 * h)
        np.testing.assert_allclose(gr, fd, rtol=1e-6, atol=1e-7 * np.abs(gr).max())


def test_closed_loop_plant_drifts_by_the_disturbance():
    """Ad = I, Bd = 0: the inputs cannot act, so x_k = x_0 + k w_d exactly
    (w_d and x_0 dyadic), and the actual cost has a closed form."""
    wl = W.small(dof=2, T=20, p=3, P=120, E=10)
    b = wl.bounds()
    w = np.array([0.125, -0.25, 0.0625, 0.5])[: wl.n]
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    M = O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p, w=w)
    x0 = np.array([0.5, -0.5, 0.25, 0.0])[: wl.n]
    g = np.zeros(wl.n)
    steps = 5
    ga = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma)
    xs, us, J, _ = O.closed_loop(ga, np.eye(wl.n), np.zeros((wl.n, wl.m)), wl.Q(), wl.R(),
                                 x0, g, steps, 1)
    for k in range(steps + 1):
        np.testing.assert_array_equal(xs[k], x0 + k * w)
    Q, R = wl.Q(), wl.R()
    ref = sum((x0 + k * w) @ Q @ (x0 + k * w) for k in range(steps + 1))
    ref += sum(u @ R @ u for u in us)
    assert abs(J - ref) <= 1e-12 * ref
