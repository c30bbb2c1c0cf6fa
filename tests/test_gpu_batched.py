"""Batched persistent launch against the FP64 oracle and against independent
single-problem solves, plus its bounded waits."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, oracle_model, rel_err

pytestmark = pytest.mark.gpu


def _problems(wls):
    import paper_2001_04931_gb300 as E
    out = []
    for wl in wls:
        A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
        x0, g = wl.start_goal()
        out.append(dict(A=A, B=B, Q=wl.Q(), R=wl.R(), bounds=wl.bounds(), x0=x0, x_goal=g,
                        horizon=wl.T, knots=wl.p, pop=wl.P, elite=wl.E, seed=wl.seed + 100,
                        sigma=wl.sigma))
    return out


def _small_batch():
    # uneven sizes: every compiled state class up to 64, ragged populations
    specs = [dict(dof=2, T=20, p=3, P=96, E=6), dict(dof=5, T=33, p=4, P=130, E=8),
             dict(dof=12, T=17, p=5, P=64, E=4), dict(dof=24, radius=3, dt=0.005, T=40, p=5,
                                                          P=200, E=12),
             dict(dof=32, T=12, p=3, P=70, E=5), dict(dof=1, T=7, p=2, P=33, E=3)]
    return [W.small(name=f"s{i}", seed=i, **kw) for i, kw in enumerate(specs)]


def test_batched_lockstep_against_oracle():
    import torch
    import paper_2001_04931_gb300 as E
    wls = _small_batch()
    probs = _problems(wls)
    bt = E.Batch(probs)
    prev = [None] * len(wls)
    for gen in range(3):
        knots, costs = bt.solve(1)
        for i, (wl, pr) in enumerate(zip(wls, probs)):
            D = wl.m * wl.p
            pop = torch.empty((D, wl.P), device="cuda")
            cost = torch.empty(wl.P, device="cuda")
            el = torch.empty(wl.E, device="cuda", dtype=torch.int32)
            bt.get_state(i, pop, cost, el)
            pop, cost, el = pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()
            b = wl.bounds().astype(np.float32)
            if prev[i] is None:
                ref = O.breed_cold(pr["seed"], gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P)
            else:
                ref = O.breed_warm(pr["seed"], gen, prev[i][0], prev[i][2], b[:, 0], b[:, 1],
                                   wl.m, wl.p, wl.sigma)
            np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
            M = oracle_model(wl)
            oc = M.cost_population(pr["x0"], pr["x_goal"], pop)
            assert rel_err(cost, oc).max() <= 1e-5
            check_elites(el, oc, wl.E)
            assert costs[i] == cost[el[0]]
            np.testing.assert_array_equal(knots[i], pop[:, el[0]])
            prev[i] = (pop, cost, el)
    bt.close()


def test_batched_matches_single_problem_solves():
    """Same seeds: the batch reproduces independent warp-family solves."""
    import paper_2001_04931_gb300 as E
    wls = _small_batch()
    probs = _problems(wls)
    bt = E.Batch(probs)
    bk, bc = bt.solve(4)
    for i, pr in enumerate(probs):
        single = E.Problem(pr["A"], pr["B"], pr["Q"], pr["R"], pr["bounds"], pr["horizon"],
                           pr["knots"], pr["pop"], seed=pr["seed"], elite=pr["elite"],
                           sigma=pr["sigma"], tile=1)  # first warp-family shape
        assert single.info().tile_kind == 1
        k, c = single.solve(pr["x0"], pr["x_goal"], 4)
        assert c == bc[i]
        np.testing.assert_array_equal(k, bk[i])
        single.close()
    bt.close()


def test_batched_wait_runs_out_and_reports_timeout():
    import paper_2001_04931_gb300 as E
    wls = _small_batch()[:3]
    bt = E.Batch(_problems(wls))
    bt.inject_stall(1, 0.5)
    with pytest.raises(E.EmpcError) as ei:
        bt.solve(3)
    assert ei.value.status == E.EMPC_ETIMEOUT
    # the context stays usable: clear the fault and solve again (cold)
    bt.inject_stall(-1, 1.0)
    knots, costs = bt.solve(2)
    assert np.isfinite(costs).all()
    bt.close()


def test_batched_new_targets_warm_start_matches_single_problems():
    """A receding-horizon step: new start states and goals, populations kept.
    Each problem must follow the single-problem API given the same sequence of
    (x0, goal) pairs, bit for bit."""
    import paper_2001_04931_gb300 as E
    wls = _small_batch()
    probs = _problems(wls)
    rng = np.random.default_rng(7)
    x1 = [rng.uniform(-1, 1, pr["A"].shape[0]) for pr in probs]
    g1 = [rng.uniform(-1, 1, pr["A"].shape[0]) for pr in probs]
    bt = E.Batch(probs)
    bt.solve(2)
    bt.set_targets(x1, g1)
    bk, bc = bt.solve(3)
    for i, pr in enumerate(probs):
        single = E.Problem(pr["A"], pr["B"], pr["Q"], pr["R"], pr["bounds"], pr["horizon"],
                           pr["knots"], pr["pop"], seed=pr["seed"], elite=pr["elite"],
                           sigma=pr["sigma"], tile=1)
        single.solve(pr["x0"], pr["x_goal"], 2)
        k, c = single.solve(x1[i], g1[i], 3)
        assert c == bc[i]
        np.testing.assert_array_equal(k, bk[i])
        single.close()
    with pytest.raises(ValueError):
        bt.set_targets(x1[:-1], g1[:-1])
    bad = [v.copy() for v in x1]
    bad[0][0] = np.nan
    with pytest.raises(E.EmpcError) as ei:
        bt.set_targets(bad, g1)
    assert ei.value.status == E.EMPC_EINVAL
    bt.close()


def test_a_second_batch_does_not_lower_the_first_ones_shared_memory_limit():
    # Both batches use the same launch shape; the first needs more than 48 KiB
    # of shared memory (its 8192-candidate key array alone is 32 KiB), the
    # second much less.  Configuring the second must leave the kernel's limit
    # high enough for the first to keep launching.
    import paper_2001_04931_gb300 as E
    big = E.Batch(_problems([W.small(name="big", seed=1, dof=2, T=20, p=3, P=8192, E=64)]),
                  tile=1)
    small = E.Batch(_problems([W.small(name="small", seed=2, dof=2, T=20, p=3, P=64, E=4)]),
                    tile=1)
    _, c_small = small.solve(2)
    _, c_big = big.solve(2)
    assert np.isfinite(c_small).all() and np.isfinite(c_big).all()
    big.close()
    small.close()
