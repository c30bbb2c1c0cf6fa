"""Pins for the oracle's state-box hook (Sec. V, simulation and cost
calculation: with every state of every step simulated, hard stops and
non-convex state costs go into the simulation as if/else).

The hook, per state i after each update: d_i = max(0, lo_i - x_i, x_i - hi_i);
the penalty adds rho_i d_i^2, the clamp stops x_i at the box, and the stage
cost sees the stopped state.  Pinned by a hand-worked integrator, by the
special case of a box that never binds, by a state held at a single value,
and by the plain (pinned) trajectory plus the hinge distances it implies."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import oracle_model


def _integrator(T=6):
    # x_{k+1} = x_k + u_k, Q = 1, R = 0, two equal knots: u_k = 1 every step
    return O.Model([[1.0]], [[1.0]], [[1.0]], [[0.0]], [-5.0], [5.0], T, 2)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_integrator_hand_worked(sign):
    """x_0 = 0, u = 1: free states 1..6 and J = 1 + 4 + ... + 36 = 91.
    Stopped at 2.5: states 1, 2, 2.5, 2.5, 2.5, 2.5, J = 1 + 4 + 4 * 6.25 = 30.
    Penalty only (rho = 10, states free): d = 0, 0, .5, 1.5, 2.5, 3.5, so
    J = 91 + 10 (.25 + 2.25 + 6.25 + 12.25) = 301.
    Stop and penalty: each step from 2.5 attempts 3.5, d = 0, 0, .5, 1, 1, 1,
    J = 30 + 10 (.25 + 3) = 62.5.  Mirrored (u = -1, lower bound -2.5) the
    same values hold."""
    M = _integrator()
    U = np.array([sign, sign])
    lo, hi = ([-10.0], [2.5]) if sign > 0 else ([-2.5], [10.0])
    assert M.cost([0.0], [0.0], U) == 91.0
    cases = [(True, False, 30.0, [1, 2, 2.5, 2.5, 2.5, 2.5]),
             (False, True, 301.0, [1, 2, 3, 4, 5, 6]),
             (True, True, 62.5, [1, 2, 2.5, 2.5, 2.5, 2.5])]
    for clamp, penalty, J, xs in cases:
        box = O.StateBox(lo, hi, [10.0], clamp=clamp, penalty=penalty)
        got, traj = M.cost([0.0], [0.0], U, box=box, return_traj=True)
        assert got == J
        np.testing.assert_array_equal(traj[1:, 0], sign * np.array(xs, dtype=float))


def _chain(T=25, p=4, dof=3):
    wl = W.small(dof=dof, T=T, p=p, P=40, E=4)
    return wl, oracle_model(wl)


def test_box_that_never_binds_is_the_plain_cost():
    wl, M = _chain()
    x0, g = wl.start_goal()
    rng = np.random.default_rng(3)
    big = np.full(wl.n, 1e300)
    for mode in range(4):
        box = O.StateBox(-big, big, rng.uniform(0, 5, wl.n), clamp=mode & 1, penalty=mode & 2)
        for _ in range(5):
            U = rng.uniform(-1, 1, wl.m * wl.p)
            assert M.cost(x0, g, U, box=box) == M.cost(x0, g, U)


def test_state_held_at_one_value():
    """lo_i = hi_i = c with the clamp: x_i = c after every step, exactly."""
    wl, M = _chain()
    x0, g = wl.start_goal()
    lo, hi = np.full(wl.n, -1e300), np.full(wl.n, 1e300)
    lo[1] = hi[1] = 0.125
    box = O.StateBox(lo, hi, clamp=True)
    U = np.random.default_rng(4).uniform(-1, 1, wl.m * wl.p)
    _, traj = M.cost(x0, g, U, box=box, return_traj=True)
    assert (traj[1:, 1] == 0.125).all()
    assert traj[0, 1] == x0[1]


def test_stopped_trajectory_obeys_the_stopped_dynamics():
    """Every recorded step is the plain update of the previous recorded state
    (through the pinned knot expansion), stopped at the box."""
    wl, M = _chain()
    x0, g = wl.start_goal()
    lo, hi = np.full(wl.n, -0.4), np.full(wl.n, 0.3)
    box = O.StateBox(lo, hi, clamp=True)
    U = np.random.default_rng(5).uniform(-1, 1, wl.m * wl.p)
    _, traj = M.cost(x0, g, U, box=box, return_traj=True)
    u = O.expand(U, wl.m, wl.T, wl.p)
    for k in range(wl.T):
        step = M.A @ traj[k] + M.B @ u[k]
        np.testing.assert_allclose(traj[k + 1], np.clip(step, lo, hi), rtol=0, atol=1e-14)
    assert ((traj[1:] >= lo) & (traj[1:] <= hi)).all()
    assert ((traj[1:] == lo) | (traj[1:] == hi)).any()  # the stop acted


def test_penalty_is_the_hinge_distance_of_the_free_trajectory():
    """Without the clamp the states are the plain ones, and the cost grows by
    sum_k sum_i rho_i d_ik^2 taken on them."""
    wl, M = _chain()
    x0, g = wl.start_goal()
    rng = np.random.default_rng(6)
    lo, hi = np.full(wl.n, -0.4), np.full(wl.n, 0.3)
    rho = rng.uniform(1, 20, wl.n)
    box = O.StateBox(lo, hi, rho, penalty=True)
    U = rng.uniform(-1, 1, wl.m * wl.p)
    J0, free = M.cost(x0, g, U, return_traj=True)
    J1, traj = M.cost(x0, g, U, box=box, return_traj=True)
    np.testing.assert_array_equal(traj, free)
    d = np.maximum(np.maximum(lo - free[1:], free[1:] - hi), 0.0)
    extra = float((rho * d * d).sum())
    assert extra > 0
    assert abs((J1 - J0) - extra) <= 1e-12 * J1


def test_population_matches_single_candidate():
    wl, M = _chain()
    x0, g = wl.start_goal()
    rng = np.random.default_rng(7)
    box = O.StateBox(np.full(wl.n, -0.5), np.full(wl.n, 0.5), rng.uniform(1, 9, wl.n),
                     clamp=True, penalty=True)
    pop = rng.uniform(-1, 1, (wl.m * wl.p, 9)).astype(np.float32)
    got = M.cost_population(x0, g, pop, box=box)
    ref = [M.cost(x0, g, pop[:, c].astype(np.float64), box=box) for c in range(9)]
    np.testing.assert_array_equal(got, ref)


def test_closed_loop_plant_stays_in_the_box():
    wl = W.small(dof=2, T=20, p=3, P=120, E=10)
    M = oracle_model(wl)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    x0, g = wl.start_goal()
    lo, hi = np.full(wl.n, -0.6), np.full(wl.n, 0.6)
    x0 = np.clip(x0, lo, hi)
    box = O.StateBox(lo, hi, np.full(wl.n, 10.0), clamp=True, penalty=True)
    ga = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma, box=box)
    xs, _, _, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, 8, 2)
    assert ((xs >= lo) & (xs <= hi)).all()
    # a box that never binds leaves the loop as it is without one
    big = np.full(wl.n, 1e300)
    ga1 = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma,
                 box=O.StateBox(-big, big, np.ones(wl.n), clamp=True, penalty=True))
    ga2 = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma)
    r1 = O.closed_loop(ga1, A, B, wl.Q(), wl.R(), x0, g, 4, 2)
    r2 = O.closed_loop(ga2, A, B, wl.Q(), wl.R(), x0, g, 4, 2)
    np.testing.assert_array_equal(r1[0], r2[0])
    assert r1[2] == r2[2]
