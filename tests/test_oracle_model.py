"""Pins for the oracle's parameterization, rollout, cost, condensed form,
gradient, discretization and selection against the paper's worked example,
closed forms, invariants and library routines."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_model(n, m, T, p, seed, diag=False):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.05 * rng.standard_normal((n, n))
    B = rng.standard_normal((n, m))
    if diag:
        Q = np.diag(rng.uniform(0.5, 2, n))
        R = np.diag(rng.uniform(0.01, 0.1, m))
    else:
        L = rng.standard_normal((n, n))
        Q = L @ L.T / n + 0.1 * np.eye(n)
        L = rng.standard_normal((m, m))
        R = L @ L.T / m + 0.01 * np.eye(m)
    return O.Model(A, B, Q, R, -np.ones(m), np.ones(m), T, p), rng


def _weights(T, p):
    idx1, num, den = O.knot_table(T, p)
    Wt = np.zeros((T, p))
    for k in range(T):
        c = num[k] / den
        Wt[k, idx1[k]] += 1 - c
        if p > 1:
            Wt[k, idx1[k] + 1] += c
    return Wt


# ------------------------------------------------------------------ knots
def test_knot_weights_match_paper_T5_p3():
    gold = np.loadtxt(os.path.join(GOLD, "knot_weights_T5_p3.txt"))
    np.testing.assert_array_equal(_weights(5, 3), gold[:, 1:])


@pytest.mark.parametrize("T,p", [(50, 4), (100, 5), (200, 8), (23, 4), (7, 7), (9, 2)])
def test_knot_table_is_exact_paper_formula(T, p):
    """idx1 = floor(k / dT), c = (k - idx1 dT)/dT with dT = (T-1)/(p-1) in exact
    rationals; the last step (idx1 = p-1, c = 0) is the same input as the
    oracle's (p-2, c = 1)."""
    idx1, num, den = O.knot_table(T, p)
    dT = Fraction(T - 1, p - 1)
    for k in range(T):
        a = int(Fraction(k) / dT)  # floor
        c = (Fraction(k) - a * dT) / dT
        if a == p - 1:
            assert c == 0 and idx1[k] == p - 2 and Fraction(int(num[k]), den) == 1
        else:
            assert idx1[k] == a and Fraction(int(num[k]), den) == c


def test_p_equals_T_reproduces_per_step_inputs():
    T = 12
    U = np.random.default_rng(0).standard_normal(3 * T)
    u = O.expand(U, 3, T, T)
    np.testing.assert_array_equal(u, U.reshape(3, T).T)


def test_p_one_is_constant_input():
    U = np.array([0.3, -0.7])
    u = O.expand(U, 2, 17, 1)
    np.testing.assert_array_equal(u, np.tile(U, (17, 1)))


def test_expanded_inputs_stay_in_knot_hull():
    rng = np.random.default_rng(3)
    U = rng.uniform(-1, 1, 5 * 4)
    u = O.expand(U, 5, 50, 4)
    Um = U.reshape(5, 4)
    assert (u <= Um.max(1) + 1e-15).all() and (u >= Um.min(1) - 1e-15).all()
    np.testing.assert_array_equal(u[0], Um[:, 0])  # u* = first knot (Alg. 1 end)
    np.testing.assert_array_equal(u[-1], Um[:, -1])


# ------------------------------------------------------------------ rollout
@pytest.mark.parametrize("seed", [0, 1])
def test_rollout_matches_closed_form(seed):
    """x_T = A^T x0 + sum_k A^(T-1-k) (B u_k + w) (Eq. small_matrix_sz_v)."""
    n, m, T, p = 5, 2, 30, 4
    M, rng = _rand_model(n, m, T, p, seed)
    w = 0.01 * rng.standard_normal(n)
    M = O.Model(M.A, M.B, M.Q, M.R, M.umin, M.umax, T, p, w=w)
    x0, g = rng.standard_normal(n), rng.standard_normal(n)
    U = rng.uniform(-1, 1, m * p)
    _, traj = M.cost(x0, g, U, return_traj=True)
    u = O.expand(U, m, T, p)
    for k in [1, 7, T]:
        ref = np.linalg.matrix_power(M.A, k) @ x0
        for j in range(k):
            ref = ref + np.linalg.matrix_power(M.A, k - 1 - j) @ (M.B @ u[j] + w)
        np.testing.assert_allclose(traj[k], ref, rtol=1e-12, atol=1e-12)


def test_S_matches_paper_printed_example():
    gold = np.loadtxt(os.path.join(GOLD, "S_T5_p3.txt"))
    n, m, T, p = 3, 2, 5, 3
    M, rng = _rand_model(n, m, T, p, 5)
    _, _, _, S = M.condensed(np.zeros(n), np.zeros(n), return_S=True)
    for r, j, *coef in gold:
        r, j = int(r), int(j)
        poly = sum(c * np.linalg.matrix_power(M.A, d) for d, c in enumerate(coef))
        for i in range(m):
            np.testing.assert_allclose(S[r * n:(r + 1) * n, i * p + j], poly @ M.B[:, i],
                                       rtol=1e-13, atol=1e-14)


def test_S_columns_are_unit_knot_rollouts():
    n, m, T, p = 4, 2, 11, 4
    M, _ = _rand_model(n, m, T, p, 6)
    _, _, _, S = M.condensed(np.zeros(n), np.zeros(n), return_S=True)
    for q in range(m * p):
        U = np.zeros(m * p)
        U[q] = 1.0
        _, traj = M.cost(np.zeros(n), np.zeros(n), U, return_traj=True)
        np.testing.assert_allclose(S[:, q], traj[1:].reshape(-1), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("seed,diag", [(0, False), (1, True), (2, False)])
def test_cost_equals_condensed_quadratic(seed, diag):
    n, m, T, p = 6, 3, 40, 5
    M, rng = _rand_model(n, m, T, p, seed, diag)
    x0, g = rng.standard_normal(n), rng.standard_normal(n)
    H, f, c0 = M.condensed(x0, g)
    for _ in range(5):
        U = rng.uniform(-1, 1, m * p)
        J = M.cost(x0, g, U)
        np.testing.assert_allclose(J, U @ H @ U + 2 * f @ U + c0, rtol=1e-11)


def test_zero_cost_invariant_and_nonnegativity():
    n, m, T, p = 6, 3, 40, 5
    M, rng = _rand_model(n, m, T, p, 4)
    assert M.cost(np.zeros(n), np.zeros(n), np.zeros(m * p)) == 0.0
    pop = rng.uniform(-1, 1, (m * p, 64)).astype(np.float32)
    assert (M.cost_population(rng.standard_normal(n), rng.standard_normal(n), pop) >= 0).all()
    # zero input from the goal at rest: cost is exactly the drift of x0 = g
    x0 = rng.standard_normal(n)
    J = M.cost(x0, x0, np.zeros(m * p))
    _, traj = M.cost(x0, x0, np.zeros(m * p), return_traj=True)
    e = traj[1:] - x0
    np.testing.assert_allclose(J, np.einsum("ki,ij,kj->", e, M.Q, e), rtol=1e-13)


def test_cost_conventions_differ_by_end_terms():
    n, m, T, p = 4, 2, 25, 3
    M, rng = _rand_model(n, m, T, p, 8)
    x0, g = rng.standard_normal(n), rng.standard_normal(n)
    U = rng.uniform(-1, 1, m * p)
    J0, traj = M.cost(x0, g, U, conv=0, return_traj=True)
    J1 = M.cost(x0, g, U, conv=1)
    e0, eT = x0 - g, traj[-1] - g
    np.testing.assert_allclose(J1 - J0, e0 @ M.Q @ e0 - eT @ M.Q @ eT, rtol=1e-10, atol=1e-12)


def test_population_cost_matches_single():
    n, m, T, p = 4, 2, 25, 3
    M, rng = _rand_model(n, m, T, p, 9)
    x0, g = rng.standard_normal(n), rng.standard_normal(n)
    pop = rng.uniform(-1, 1, (m * p, 37)).astype(np.float32)
    got = M.cost_population(x0, g, pop)
    for c in [0, 13, 36]:
        assert got[c] == M.cost(x0, g, pop[:, c].astype(np.float64))


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("seed", [0, 1])
def test_adjoint_gradient_equals_condensed(seed):
    n, m, T, p = 6, 3, 40, 5
    M, rng = _rand_model(n, m, T, p, seed)
    x0, g = rng.standard_normal(n), rng.standard_normal(n)
    H, f, c0 = M.condensed(x0, g)
    U = rng.uniform(-1, 1, m * p)
    J, gr = M.grad(x0, g, U)
    np.testing.assert_allclose(gr, 2 * H @ U + 2 * f, rtol=1e-10, atol=1e-10 * np.abs(f).max())
    np.testing.assert_allclose(J, M.cost(x0, g, U), rtol=1e-14)


def test_adjoint_gradient_matches_central_differences():
    wl = W.small(dof=3, T=30, p=4)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    M = O.Model(Ad, Bd, wl.Q(), wl.R(), -np.ones(wl.m), np.ones(wl.m), wl.T, wl.p)
    x0, g = wl.start_goal()
    rng = np.random.default_rng(0)
    h = 1e-6
    for _ in range(4):
        U = rng.uniform(-1, 1, wl.m * wl.p)
        _, gr = M.grad(x0, g, U)
        fd = np.zeros_like(U)
        for q in range(U.size):
            e = np.zeros_like(U)
            e[q] = h
            fd[q] = (M.cost(x0, g, U + e) - M.cost(x0, g, U - e)) / (2 * h)
        np.testing.assert_allclose(gr, fd, rtol=1e-6, atol=1e-7 * np.abs(gr).max())


def test_refine_descends_and_stays_in_bounds():
    wl = W.small(dof=3, T=30, p=4)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    M = O.Model(Ad, Bd, wl.Q(), wl.R(), -np.ones(wl.m), np.ones(wl.m), wl.T, wl.p)
    x0, g = wl.start_goal()
    eta = M.lipschitz_step()
    U = np.random.default_rng(1).uniform(-1, 1, wl.m * wl.p)
    J = M.cost(x0, g, U)
    for _ in range(5):
        U2 = M.refine(x0, g, U, 1, eta)
        J2 = M.cost(x0, g, U2)
        assert J2 <= J + 1e-12 and (np.abs(U2) <= 1).all()
        U, J = U2, J2


@pytest.mark.parametrize("eta_scale,steps", [(1.0, 1), (1.0, 3), (40.0, 1), (40.0, 2)])
def test_refine_is_the_projected_step_of_the_condensed_form(eta_scale, steps):
    """orc_refine against projected gradient written out in numpy from the
    condensed form J = U'HU + 2f'U + c0 (Sec. IV-E), whose S is pinned to the
    printed example: each step is U <- clip(U - eta (2 H U + 2 f)) with each
    knot clipped to its own input's bounds.  The large step makes clipping
    bind on many knots, so a clip taken before the step, a missing factor 2,
    a wrong step count or a wrong input index for the bounds all fail."""
    wl = W.small(dof=3, T=30, p=4)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    lo = np.array([-1.0, -0.3, -0.7])
    hi = np.array([0.9, 0.4, 1.0])
    M = O.Model(Ad, Bd, wl.Q(), wl.R(), lo, hi, wl.T, wl.p)
    x0, g = wl.start_goal()
    H, f, _ = M.condensed(x0, g)
    eta = eta_scale * M.lipschitz_step()
    lo_q, hi_q = np.repeat(lo, wl.p), np.repeat(hi, wl.p)
    U0 = np.random.default_rng(5).uniform(lo_q, hi_q)
    U = U0.copy()
    clipped = 0
    for _ in range(steps):
        free = U - eta * (2.0 * H @ U + 2.0 * f)
        U = np.minimum(np.maximum(free, lo_q), hi_q)
        clipped += int(np.count_nonzero(U != free))
    got = M.refine(x0, g, U0, steps, eta)
    np.testing.assert_allclose(got, U, rtol=1e-10, atol=1e-12)
    if eta_scale > 1.0:
        assert clipped >= 3  # the bounds bind, so the clip's place in the step matters


# ------------------------------------------------------------------ ZOH
def test_zoh_matches_scipy_expm():
    plant = W.chain_plant(4, seed=3, radius=3)
    for dt in [0.005, 0.01, 0.3]:
        Ad, Bd = O.zoh(plant.Ac, plant.Bc, dt)
        n, m = plant.Bc.shape
        Mbig = np.zeros((n + m, n + m))
        Mbig[:n, :n] = plant.Ac
        Mbig[:n, n:] = plant.Bc
        E = scipy.linalg.expm(Mbig * dt)
        np.testing.assert_allclose(Ad, E[:n, :n], rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(Bd, E[:n, n:], rtol=1e-13, atol=1e-15)


def test_zoh_closed_forms():
    # double integrator (nilpotent): Ad = [[1, dt], [0, 1]], Bd = [dt^2/2, dt]
    Ad, Bd = O.zoh(np.array([[0.0, 1.0], [0.0, 0.0]]), np.array([[0.0], [1.0]]), 0.1)
    np.testing.assert_allclose(Ad, [[1, 0.1], [0, 1]], rtol=0, atol=1e-16)
    np.testing.assert_allclose(Bd[:, 0], [0.005, 0.1], rtol=1e-15)
    # diagonal: Ad = exp(a dt), Bd = (exp(a dt) - 1)/a * b
    a = np.array([-2.0, 0.5, -7.0])
    Ad, Bd = O.zoh(np.diag(a), np.eye(3), 0.2)
    np.testing.assert_allclose(np.diag(Ad), np.exp(a * 0.2), rtol=1e-14)
    np.testing.assert_allclose(np.diag(Bd), np.expm1(a * 0.2) / a, rtol=1e-13)


def test_zoh_small_dt_limit():
    plant = W.chain_plant(3, seed=1)
    dt = 1e-7
    Ad, Bd = O.zoh(plant.Ac, plant.Bc, dt)
    np.testing.assert_allclose(Ad, np.eye(6) + plant.Ac * dt, atol=1e-12)
    np.testing.assert_allclose(Bd, plant.Bc * dt, atol=1e-12)


# ------------------------------------------------------------------ select
def test_select_is_lexicographic_cost_index():
    rng = np.random.default_rng(0)
    cost = np.round(rng.uniform(0, 10, 1000), 1)  # many exact ties
    cost[[3, 17, 900]] = np.nan
    cost[5] = np.inf
    for E in [1, 32, 999, 1000]:
        got = O.select(cost, E)
        key = np.where(np.isnan(cost), np.inf, cost)
        ref = np.lexsort((np.arange(1000), key))[:E]
        np.testing.assert_array_equal(got, ref)
