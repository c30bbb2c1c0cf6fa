"""CUDA path vs the FP64 oracle, through the C ABI.

Bars: candidate costs within 1e-5 relative (FP32 against FP64); elite sets
equal wherever the FP64 cost gap exceeds that tolerance; bred populations
(draws, crossover, mutation, clipping) equal bit for bit given the same
previous population and elite indices (lockstep replay)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, gpu_problem, oracle_model, rel_err, report

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-5


def _torch():
    import torch
    return torch


def _state(prob):
    torch = _torch()
    pop = torch.empty((prob.D, prob.P), device="cuda", dtype=torch.float32)
    cost = torch.empty(prob.P, device="cuda", dtype=torch.float32)
    elite = torch.empty(prob.E, device="cuda", dtype=torch.int32)
    prob.get_state(pop, cost, elite)
    torch.cuda.synchronize()
    return pop.cpu().numpy(), cost.cpu().numpy(), elite.cpu().numpy()


def _evaluate(prob, x0, g, pop_np):
    torch = _torch()
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    cost = torch.empty(pop.shape[1], device="cuda", dtype=torch.float32)
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    prob.evaluate(x0d, gd, pop, cost)
    torch.cuda.synchronize()
    return cost.cpu().numpy()


def _lockstep(wl, generations, seed=3, sample=None, **cfg):
    prob = gpu_problem(wl, seed=seed, **cfg)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    b = wl.bounds().astype(np.float32)
    prev = None
    best_hist = []
    for gen in range(generations):
        knots, best = prob.solve(x0, g, 1)
        pop, cost, elite = _state(prob)
        # breeding: bit-exact against the oracle's draws
        if prev is None:
            ref = O.breed_cold(seed, gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P)
        else:
            ref = O.breed_warm(seed, gen, prev[0], prev[2], b[:, 0], b[:, 1], wl.m, wl.p,
                               wl.sigma, gate_mode=cfg.get("gate", 0))
        np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
        # costs within tolerance
        cols = np.arange(wl.P) if sample is None else np.unique(
            np.r_[sample, elite, np.arange(min(wl.E, wl.P))])
        oc = M.cost_population(x0, g, pop[:, cols])
        err = rel_err(cost[cols], oc)
        report(f"lockstep_n{wl.n}_P{wl.P}_gen{gen}", max_rel=err.max())
        assert err.max() <= COST_RTOL
        if sample is None:
            check_elites(elite, oc, wl.E)
        # the reported best is rank 0
        assert best == cost[elite[0]]
        np.testing.assert_array_equal(knots, pop[:, elite[0]])
        best_hist.append(best)
        prev = (pop, cost, elite)
    # elitism: the best cost never increases
    assert all(b2 <= b1 for b1, b2 in zip(best_hist, best_hist[1:]))
    prob.close()
    return best_hist


def test_lockstep_small_ragged():
    # P = 200 spans several tiles with a ragged last tile
    _lockstep(W.small(dof=3, T=23, p=4, P=200, E=16), 4)


def test_lockstep_c1_full_size():
    _lockstep(W.config("c1"), 5)


def test_lockstep_breeding_at_a_million_knot_groups():
    """8192 candidates of 512 knots (the 64-DoF chain's knot count): 2^20
    four-knot groups, one breeding thread each; the bred populations equal
    the oracle's draws bit for bit (cold, then two warm generations)."""
    wl = W.small(dof=64, radius=3, dt=0.005, T=8, p=8, P=8192, E=64, q_pos=10.0, q_vel=1.0,
                 r=1e-4)
    assert wl.P * (wl.m * wl.p // 4) == 1 << 20
    _lockstep(wl, 3, seed=4, sample=np.arange(0, wl.P, 97))


@pytest.mark.parametrize("gate", [0, 1, 2])
def test_lockstep_gate_modes(gate):
    _lockstep(W.small(dof=2, T=17, p=3, P=96, E=8, sigma=0.3), 3, gate=gate)


def test_lockstep_c2_full_size():
    # every one of the 4096 candidates costed by the FP64 oracle, and the
    # elite set checked, in each of three lockstep generations
    _lockstep(W.config("c2"), 3)


def _c5_fp32_workload(P=512, T=200):
    """The 64-DoF chain of the large workload (n = 128, m = 64, 8 knots) at a
    population the oracle costs in seconds: four tiles of 128 plus a ragged
    tail when P is not a multiple of 128."""
    return W.small(dof=64, radius=3, dt=0.005, T=T, p=8, P=P, E=16, q_pos=10.0, q_vel=1.0,
                   r=1e-4)


def test_fp32_block_family_n128_costs():
    """n = 128 runs in the block family with one state row per thread (R = 1):
    the plain-FP32 path the BF16 rollout of the 64-DoF chain is compared with.
    Horizon 200 as in that workload; 4.5 tiles of candidates."""
    wl = _c5_fp32_workload(P=577)
    prob = gpu_problem(wl)
    inf = prob.info()
    assert inf.tile_kind == 0 and inf.tile_nx == 128 and inf.tile_rows == 1
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(3).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    err = rel_err(_evaluate(prob, x0, g, pop), M.cost_population(x0, g, pop))
    report("fp32_block_n128_T200", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= COST_RTOL, (float(err.max()), float(np.median(err)))
    prob.close()


def test_lockstep_fp32_n128():
    """Two lockstep generations of the 64-DoF chain in FP32 (block family):
    bred populations bit-exact, every cost within 1e-5, elites checked."""
    _lockstep(_c5_fp32_workload(P=384, T=120), 2)


@pytest.mark.parametrize("kw", [
    dict(dof=1, T=1, p=1, P=7, E=1),      # one step, one knot, tiny population
    dict(dof=2, T=9, p=9, P=33, E=33),    # p = T (per-step inputs), E = P
    dict(dof=5, T=40, p=1, P=65, E=4),    # constant input
    dict(dof=16, T=31, p=6, P=130, E=9),  # n = 32
    dict(dof=32, T=12, p=3, P=70, E=5),   # n = 64
])
def test_costs_edge_shapes(kw):
    wl = W.small(**kw)
    prob = gpu_problem(wl)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    rng = np.random.default_rng(1)
    pop = rng.uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    got = _evaluate(prob, x0, g, pop)
    assert rel_err(got, M.cost_population(x0, g, pop)).max() <= COST_RTOL
    prob.close()


@pytest.mark.parametrize("n,m", [(5, 3), (7, 9), (12, 1)])
def test_costs_random_models_odd_dims(n, m):
    """Non-chain models: odd n, m > n, single input; dense A, diagonal Q/R."""
    rng = np.random.default_rng(n * 31 + m)
    T, p, P = 37, 4, 150
    A = np.eye(n) + 0.02 * rng.standard_normal((n, n))
    B = 0.1 * rng.standard_normal((n, m))
    Q = np.diag(rng.uniform(0.1, 3, n))
    R = np.diag(rng.uniform(0.0, 0.1, m))
    bounds = np.tile([-2.0, 1.5], (m, 1))
    import paper_2001_04931_gb300 as E
    prob = E.Problem(A, B, Q, R, bounds, T, p, P, seed=5, elite=8)
    M = O.Model(A, B, Q, R, bounds[:, 0], bounds[:, 1], T, p)
    x0, g = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    pop = rng.uniform(-2, 1.5, (m * p, P)).astype(np.float32)
    got = _evaluate(prob, x0, g, pop)
    assert rel_err(got, M.cost_population(x0, g, pop)).max() <= COST_RTOL
    prob.close()


def test_tile_shapes_give_identical_costs():
    """Within one kernel family (block or warp) a candidate's arithmetic does
    not depend on the tile shape (bitwise); the families agree within the
    tolerance."""
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=24, radius=3, dt=0.005, T=60, p=5, P=300, E=16)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(2).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    by_kind = {}
    for tile in range(1, 64):
        try:
            prob = gpu_problem(wl, tile=tile)
        except E.EmpcError as e:
            assert e.status == E.EMPC_EINVAL
            break
        inf = prob.info()
        by_kind.setdefault(inf.tile_kind, []).append(
            _evaluate(prob, x0, g, pop))
        prob.close()
    assert set(by_kind) == {0, 1}
    for outs in by_kind.values():
        assert len(outs) >= 3
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])
    fams = list(by_kind.values())
    for o in fams[1:]:
        assert rel_err(o[0], fams[0][0]).max() <= 2e-6


def test_nonfinite_costs_sort_last_and_are_reported():
    torch = _torch()
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=2, T=10, p=3, P=64, E=4)
    prob = gpu_problem(wl)
    x0, g = wl.start_goal()
    prob.solve(x0, g, 1)
    pop, cost, elite = _state(prob)
    pop[:, :10] = np.nan  # ten poisoned candidates
    cost_t = torch.from_numpy(cost).cuda()
    prob.set_state(torch.from_numpy(pop).cuda(), cost_t,
                   torch.from_numpy(np.arange(4, dtype=np.int32)).cuda())
    c = _evaluate(prob, x0, g, pop)
    assert np.isinf(c[:10]).all() and np.isfinite(c[10:]).all()
    # an exploding model gives a non-finite best cost -> EMPC_ENONFINITE
    A = np.eye(4) * 1e30
    B = np.ones((4, 2))
    bad = E.Problem(A, B, np.eye(4), np.eye(2), wl.bounds(), 50, 3, 64, seed=1, elite=4)
    with pytest.raises(E.EmpcError) as ei:
        bad.solve(np.ones(4), np.zeros(4), 2)
    assert ei.value.status == E.EMPC_ENONFINITE
    bad.close()
    prob.close()


def test_warm_start_persists_and_reset_starts_cold():
    wl = W.small(dof=2, T=20, p=3, P=128, E=8)
    prob = gpu_problem(wl, seed=9)
    b = wl.bounds().astype(np.float32)
    x0, g = wl.start_goal()
    prob.solve(x0, g, 3)  # generations 0, 1, 2
    assert prob.info().generation == 3
    prob.reset()
    prob.solve(x0, g, 1)  # generation 3, cold
    pop, _, _ = _state(prob)
    ref = O.breed_cold(9, 3, b[:, 0], b[:, 1], wl.m, wl.p, wl.P)
    np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
    prob.close()


def _same_state(a, b):
    for x, y in zip(_state(a), _state(b)):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))


@pytest.mark.parametrize("case", ["ragged", "gate1", "c2", "condensed"])
def test_multi_generation_solve_equals_single_generation_solves(case):
    # One captured graph of G generations against G graphs of one generation
    # (each of which the lockstep tests check against the oracle): the same
    # populations, costs, elites, best plan and generation counter, bit for
    # bit, from a cold start and again from the warm start that follows.
    import paper_2001_04931_gb300 as E
    cfg = {}
    if case == "ragged":
        wl = W.small(dof=3, T=23, p=4, P=200, E=16)
    elif case == "gate1":
        wl = W.small(dof=2, T=17, p=3, P=96, E=8, sigma=0.3)
        cfg = {"gate": 1}
    elif case == "c2":
        wl = W.config("c2")
    else:
        wl = W.small(dof=3, T=30, p=4, P=700, E=32)
        cfg = {"evaluator": E.EMPC_EVAL_CONDENSED}
    x0, g = wl.start_goal()
    a = gpu_problem(wl, seed=6, **cfg)
    b = gpu_problem(wl, seed=6, **cfg)
    for G in (4, 3):
        ka, ca = a.solve(x0, g, G)
        for _ in range(G):
            kb, cb = b.solve(x0, g, 1)
        np.testing.assert_array_equal(ka.view(np.uint32), kb.view(np.uint32))
        assert np.float32(ca).view(np.uint32) == np.float32(cb).view(np.uint32)
        assert a.info().generation == b.info().generation
        _same_state(a, b)
    a.close()
    b.close()


def test_solve_device_matches_host_solve():
    torch = _torch()
    wl = W.small(dof=3, T=25, p=4, P=256, E=16)
    x0, g = wl.start_goal()
    a = gpu_problem(wl, seed=4)
    b = gpu_problem(wl, seed=4)
    k1, c1 = a.solve(x0, g, 4)
    kd = torch.empty(wl.m * wl.p, device="cuda")
    cd = torch.empty(1, device="cuda")
    b.solve_device(torch.tensor(x0, dtype=torch.float32, device="cuda"),
                   torch.tensor(g, dtype=torch.float32, device="cuda"), 4, kd, cd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(kd.cpu().numpy(), k1)
    assert cd.item() == c1
    a.close()
    b.close()
