"""Pins for the oracle's receding-horizon loop (Sec. III-A, Sec. V; actual
cost by Eq. actual_cost): a plant that inputs cannot move gives a closed-form
actual cost, the first applied input is the first knot of the first solve's
best candidate, and on a chain that starts away from its goal the loop beats
applying no input at all."""
import numpy as np

import oracle as O
import workloads as W
from helpers import oracle_model


def _setup(**kw):
    wl = W.small(dof=2, T=20, p=3, P=120, E=10, **kw)
    M = oracle_model(wl)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    return wl, M, A, B


def test_frozen_plant_actual_cost_closed_form():
    wl, M, A, B = _setup()
    x0, g = wl.start_goal()
    ga = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma)
    steps = 6
    xs, us, J, _ = O.closed_loop(ga, np.eye(wl.n), np.zeros((wl.n, wl.m)), wl.Q(), wl.R(), x0,
                                 g, steps, 2)
    np.testing.assert_array_equal(xs, np.tile(x0, (steps + 1, 1)))
    e = g - x0
    state_term = e @ wl.Q() @ e
    input_term = sum(u @ wl.R() @ u for u in us)
    assert abs(J - ((steps + 1) * state_term + input_term)) <= 1e-12 * J


def test_first_input_is_first_knot_of_best():
    wl, M, A, B = _setup()
    x0, g = wl.start_goal()
    ga = O.EMPC(M, wl.P, wl.E, seed=4, sigma=wl.sigma)
    ref = O.EMPC(M, wl.P, wl.E, seed=4, sigma=wl.sigma)
    knots, _ = ref.solve(x0, g, 3)
    xs, us, _, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, 1, 3)
    np.testing.assert_array_equal(us[0], knots.astype(np.float64)[::wl.p])
    np.testing.assert_allclose(xs[1], A @ x0 + B @ us[0], rtol=0, atol=0)


def test_loop_beats_no_input():
    wl = W.small(dof=2, T=60, p=3, P=200, E=12)
    M = oracle_model(wl)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    x0 = np.zeros(wl.n)
    g = np.r_[np.full(wl.dof, 0.05), np.zeros(wl.dof)]  # holdable within the input bounds
    ga = O.EMPC(M, wl.P, wl.E, seed=5, sigma=wl.sigma)
    steps = 300
    xs, _, J, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, steps, 2)
    x, J0 = x0.copy(), 0.0
    for _ in range(steps):
        e = g - x
        J0 += e @ wl.Q() @ e
        x = A @ x
    e = g - x
    J0 += e @ wl.Q() @ e
    assert J < 0.5 * J0
    assert np.abs(xs[-1] - g).max() < 0.2 * np.abs(x0 - g).max()


def test_distance_scaled_sigma():
    """At the goal the exploration noise is the floor; far away it is the
    configured sigma; with a zero floor at the goal, children only recombine
    their parents' knots (no value outside the previous population appears)."""
    wl, M, A, B = _setup()
    g = np.zeros(wl.n)
    ga = O.EMPC(M, wl.P, wl.E, seed=8, sigma=wl.sigma)
    _, _, _, sig = O.closed_loop(ga, np.eye(wl.n), np.zeros((wl.n, wl.m)), wl.Q(), wl.R(), g, g,
                                 4, 1, sigma_min=0.0, sigma_dref=1.0)
    assert (sig == 0.0).all()
    prev = ga.pop.copy()
    ga.sigma = 0.0
    ga.generation(g, g)
    for q in range(prev.shape[0]):
        assert np.isin(ga.pop[q], prev[q]).all()
    far = np.full(wl.n, 10.0)
    ga2 = O.EMPC(M, wl.P, wl.E, seed=8, sigma=wl.sigma)
    _, _, _, sig2 = O.closed_loop(ga2, np.eye(wl.n), np.zeros((wl.n, wl.m)), wl.Q(), wl.R(), far,
                                  g, 3, 1, sigma_min=0.01, sigma_dref=1.0)
    assert (sig2 == np.float32(wl.sigma)).all()
