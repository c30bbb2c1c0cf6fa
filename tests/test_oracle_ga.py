"""Pins for the oracle's breeding and Algorithm 1 loop: statistical laws of the
draws, elitism invariants, and brute force / exact box-QP optimum on 1-DoF."""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle as O
import workloads as W


def test_cold_start_uniform_in_bounds_and_counter_based():
    umin = np.array([-1.0, 0.0, -3.0], np.float32)
    umax = np.array([1.0, 0.5, 3.0], np.float32)
    pop = O.breed_cold(7, 0, umin, umax, 3, 4, 4000)
    for i in range(3):
        v = pop[i * 4:(i + 1) * 4].ravel()
        assert v.min() >= umin[i] and v.max() <= umax[i]
        assert stats.kstest((v - umin[i]) / (umax[i] - umin[i]), "uniform").pvalue > 1e-4
    # candidate c's draws do not depend on the population size
    small = O.breed_cold(7, 0, umin, umax, 3, 4, 100)
    np.testing.assert_array_equal(small, pop[:, :100])
    assert not np.array_equal(O.breed_cold(7, 1, umin, umax, 3, 4, 100), small)
    assert not np.array_equal(O.breed_cold(8, 0, umin, umax, 3, 4, 100), small)


def test_warm_keeps_elites_in_rank_order():
    m, p, P, E = 3, 4, 300, 20
    rng = np.random.default_rng(0)
    old = rng.uniform(-1, 1, (m * p, P)).astype(np.float32)
    elite = rng.permutation(P)[:E].astype(np.int32)
    new = O.breed_warm(1, 5, old, elite, -np.ones(m), np.ones(m), m, p, 0.1)
    np.testing.assert_array_equal(new[:, :E], old[:, elite])


def test_crossover_takes_each_parameter_from_a_parent():
    """No mutation: every child parameter equals one of the elites' values
    at that parameter, each child has exactly two parents, and about half the
    parameters come from each."""
    m, p, P, E = 4, 5, 2000, 8
    D = m * p
    old = np.zeros((D, P), np.float32)
    elite = np.arange(E, dtype=np.int32) * 7
    for e in range(E):  # distinct per elite and per parameter
        old[:, elite[e]] = (e + 1) * 0.01 + np.arange(D) * 0.1
    new = O.breed_warm(3, 2, old, elite, -10 * np.ones(m), 10 * np.ones(m), m, p, 0.1,
                       pm256=0)
    par = np.rint((new[:, E:] - (np.arange(D) * 0.1)[:, None]) / 0.01).astype(int) - 1
    assert par.min() >= 0 and par.max() < E
    npar = np.array([len(set(par[:, c])) for c in range(P - E)])
    assert npar.max() <= 2
    # parent draws uniform over the E elites (chi-square, one parameter per child)
    counts = np.bincount(par[0], minlength=E)
    assert stats.chisquare(counts).pvalue > 1e-4
    # with two distinct parents, the share taken from either is about 1/2
    two = npar == 2
    frac = np.array([np.mean(par[:, c] == par[0, c]) for c in np.nonzero(two)[0]])
    assert abs(frac.mean() - 0.5) < 0.03
    # pc256 = 0: always the first parent, so one parent per child
    new0 = O.breed_warm(3, 2, old, elite, -10 * np.ones(m), 10 * np.ones(m), m, p, 0.1,
                        pc256=0, pm256=0)
    par0 = np.rint((new0[:, E:] - (np.arange(D) * 0.1)[:, None]) / 0.01).astype(int) - 1
    assert max(len(set(par0[:, c])) for c in range(P - E)) == 1


def test_mutation_gate_per_input_and_gaussian_noise():
    """E = 1 (both parents the single elite): child - elite is sigma * N(0,1) on
    gated inputs (all p knots of a gated input), zero elsewhere; about half of
    the inputs are gated."""
    m, p, P, sigma = 6, 4, 3000, 0.25
    old = np.zeros((m * p, P), np.float32)
    old[:, 0] = np.linspace(-0.5, 0.5, m * p)
    new = O.breed_warm(11, 4, old, np.array([0], np.int32), -100 * np.ones(m),
                       100 * np.ones(m), m, p, sigma)
    d = (new[:, 1:] - old[:, :1]).reshape(m, p, P - 1)
    gated = np.abs(d).sum(1) > 0
    assert ((np.abs(d) > 0).sum(1) == gated * p).all()  # all-or-none per input
    assert abs(gated.mean() - 0.5) < 0.02
    z = (d[:, :, :][np.broadcast_to(gated[:, None, :], d.shape)]) / sigma
    assert abs(z.std() - 1) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # per-parameter gate: about half of all parameters mutated, independently
    new1 = O.breed_warm(11, 4, old, np.array([0], np.int32), -100 * np.ones(m),
                        100 * np.ones(m), m, p, sigma, gate_mode=1)
    d1 = new1[:, 1:] - old[:, :1]
    assert abs((d1 != 0).mean() - 0.5) < 0.02
    # always-mutate
    new2 = O.breed_warm(11, 4, old, np.array([0], np.int32), -100 * np.ones(m),
                        100 * np.ones(m), m, p, sigma, gate_mode=2)
    assert ((new2[:, 1:] - old[:, :1]) != 0).mean() > 0.999


def test_children_clipped_to_bounds():
    m, p, P = 2, 3, 500
    old = np.full((m * p, P), 0.95, np.float32)
    new = O.breed_warm(2, 1, old, np.arange(4, dtype=np.int32), -np.ones(m), np.ones(m), m,
                       p, 1.0, gate_mode=2)
    assert new.max() == 1.0 and new.min() >= -1.0


def _model_1dof(T=20, p=2, seed=0):
    wl = W.small(dof=1, T=T, p=p, seed=seed, q_pos=1.0, q_vel=0.1, r=1e-2)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, 0.05)
    return O.Model(Ad, Bd, wl.Q(), wl.R(), -np.ones(1), np.ones(1), T, p), wl


def _box_qp_exact(H, f, lo, hi):
    """min U'HU + 2f'U on the box, by enumerating active sets (each coordinate
    at lo, at hi, or free) and keeping the feasible KKT point of least value."""
    D = f.size
    best, bestU = np.inf, None
    for pat in itertools.product(range(3), repeat=D):
        U = np.zeros(D)
        free = [q for q in range(D) if pat[q] == 2]
        for q in range(D):
            if pat[q] == 0:
                U[q] = lo
            elif pat[q] == 1:
                U[q] = hi
        if free:
            fixed = [q for q in range(D) if pat[q] != 2]
            rhs = -f[free] - H[np.ix_(free, fixed)] @ U[fixed]
            U[free] = np.linalg.solve(H[np.ix_(free, free)], rhs)
        if (U < lo - 1e-12).any() or (U > hi + 1e-12).any():
            continue
        val = U @ H @ U + 2 * f @ U
        if val < best:
            best, bestU = val, U
    return best, bestU


@pytest.mark.parametrize("p", [2, 3])
def test_empc_reaches_brute_force_optimum_1dof(p):
    M, wl = _model_1dof(T=20, p=p)
    x0, g = np.array([0.8, 0.0]), np.array([-0.6, 0.0])
    # brute force over a 101^p knot grid
    grid = np.linspace(-1, 1, 101)
    pts = np.array(list(itertools.product(grid, repeat=p)), np.float32).T
    costs = M.cost_population(x0, g, pts)
    gmin = costs.min()
    H, f, c0 = M.condensed(x0, g)
    qp, Uqp = _box_qp_exact(H, f, -1.0, 1.0)
    assert qp + c0 <= gmin + 1e-12  # the exact optimum lower-bounds the grid
    ga = O.EMPC(M, P=256, E=16, seed=5, sigma=0.05)
    U, J = ga.solve(x0, g, 25)
    assert J >= qp + c0 - 1e-9 * abs(qp + c0)  # cannot beat the optimum
    # grid spacing 0.02: the grid minimum is within half a cell of the optimum
    assert J <= gmin + 1e-6 * abs(gmin)


def test_elitism_best_cost_non_increasing():
    wl = W.small(dof=3, T=30, p=4, P=128, E=8)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    M = O.Model(Ad, Bd, wl.Q(), wl.R(), -np.ones(wl.m), np.ones(wl.m), wl.T, wl.p)
    x0, g = wl.start_goal()
    ga = O.EMPC(M, P=wl.P, E=wl.E, seed=1, sigma=0.1)
    best = []
    for _ in range(12):
        ga.generation(x0, g)
        best.append(ga.cost[ga.elite[0]])
        # the elite slots hold the previous elites, re-evaluated to the same cost
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))
    assert best[-1] < best[0]


def test_refined_empc_not_worse_than_plain():
    wl = W.small(dof=3, T=30, p=4, P=128, E=8)
    Ad, Bd = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    M = O.Model(Ad, Bd, wl.Q(), wl.R(), -np.ones(wl.m), np.ones(wl.m), wl.T, wl.p)
    x0, g = wl.start_goal()
    eta = M.lipschitz_step()
    plain = O.EMPC(M, P=wl.P, E=wl.E, seed=1, sigma=0.1)
    ref = O.EMPC(M, P=wl.P, E=wl.E, seed=1, sigma=0.1, refine_steps=3, refine_eta=eta)
    _, Jp = plain.solve(x0, g, 6)
    _, Jr = ref.solve(x0, g, 6)
    H, f, c0 = M.condensed(x0, g)
    assert Jr <= Jp * 1.0001
    assert Jr >= c0 - f @ np.linalg.solve(H, f) - 1e-9  # unconstrained optimum bound
