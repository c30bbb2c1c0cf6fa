"""The state-box hook in the FP32 rollout (Sec. V: hard stops and non-convex
state costs written into the simulation as if/else) against the FP64
oracle, through the C ABI.

Bars: candidate costs within 1e-5 relative of the oracle's hooked costs (the
hinge and the stop are continuous, so FP32 rounding near a bound moves the
cost by a rounding-sized amount), in both kernel families; a box that never
binds gives costs bit-identical to no hook (the hook adds exact zeros and
changes no state); the elite sets of a hooked solve agree with the FP64 costs
wherever those are separated by more than the tolerance; a closed loop with
the stop keeps the plant inside the box."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, gpu_problem, oracle_model, rel_err

pytestmark = pytest.mark.gpu
COST_RTOL = 1e-5


def _evaluate(prob, x0, g, pop_np):
    import torch
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    cost = torch.empty(pop.shape[1], device="cuda", dtype=torch.float32)
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    prob.evaluate(x0d, gd, pop, cost)
    torch.cuda.synchronize()
    return cost.cpu().numpy()


def _box(n, seed):
    """Bounds and weights exact in FP32, so both sides hold the same box."""
    rng = np.random.default_rng(seed)
    lo = -np.float32(0.25) * rng.integers(1, 4, n).astype(np.float32)
    hi = np.float32(0.25) * rng.integers(1, 4, n).astype(np.float32)
    rho = rng.integers(1, 40, n).astype(np.float32)
    return lo, hi, rho


def _tiles_by_kind(wl):
    """One forced tile index per kernel family (0 block, 1 warp)."""
    import paper_2001_04931_gb300 as E
    out = {}
    for tile in range(1, 64):
        try:
            prob = gpu_problem(wl, tile=tile)
        except E.EmpcError as e:
            assert e.status == E.EMPC_EINVAL
            break
        out.setdefault(prob.info().tile_kind, tile)
        prob.close()
    return out


@pytest.mark.parametrize("kw", [
    dict(dof=3, T=25, p=4, P=200, E=8),
    dict(dof=24, radius=3, dt=0.005, T=60, p=5, P=300, E=16),
    dict(dof=5, T=1, p=1, P=33, E=3),
])
@pytest.mark.parametrize("clamp,penalty", [(True, False), (False, True), (True, True)])
def test_hooked_costs_match_oracle(kw, clamp, penalty):
    wl = W.small(**kw)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    lo, hi, rho = _box(wl.n, 1)  # x0 may start outside: the hook acts after each update
    pop = np.random.default_rng(2).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    ref = M.cost_population(x0, g, pop,
                            box=O.StateBox(lo, hi, rho, clamp=clamp, penalty=penalty))
    plain = M.cost_population(x0, g, pop)
    assert (ref != plain).any()  # the box binds for some candidates
    for kind, tile in _tiles_by_kind(wl).items():
        prob = gpu_problem(wl, tile=tile)
        prob.set_state_box(lo, hi, rho, clamp=clamp, penalty=penalty)
        got = _evaluate(prob, x0, g, pop)
        assert rel_err(got, ref).max() <= COST_RTOL, (kind, float(rel_err(got, ref).max()))
        prob.close()


def test_box_that_never_binds_is_bitwise_plain():
    wl = W.small(dof=24, radius=3, dt=0.005, T=60, p=5, P=300, E=16)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(3).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    big = np.full(wl.n, 1e30, np.float32)
    for kind, tile in _tiles_by_kind(wl).items():
        prob = gpu_problem(wl, tile=tile)
        plain = _evaluate(prob, x0, g, pop)
        prob.set_state_box(-big, big, np.ones(wl.n), clamp=True, penalty=True)
        hooked = _evaluate(prob, x0, g, pop)
        np.testing.assert_array_equal(hooked.view(np.uint32), plain.view(np.uint32))
        prob.set_state_box()  # off again
        np.testing.assert_array_equal(_evaluate(prob, x0, g, pop).view(np.uint32),
                                      plain.view(np.uint32))
        prob.close()


def test_hooked_solve_selects_by_hooked_costs():
    """Breeding does not see the hook (bit-exact replay against the oracle);
    selection follows the hooked FP64 costs; switching the hook on and off
    re-captures the generation graphs."""
    import torch
    wl = W.small(dof=4, T=30, p=4, P=256, E=12)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    lo, hi, rho = _box(wl.n, 4)
    x0 = np.clip(x0, lo, hi)
    box = O.StateBox(lo, hi, rho, clamp=True, penalty=True)
    b = wl.bounds().astype(np.float32)
    prob = gpu_problem(wl, seed=9)
    prob.solve(x0, g, 1)  # a plain generation first: its graph must not be reused
    prob.reset()
    prob.set_state_box(lo, hi, rho, clamp=True, penalty=True)
    prev = None
    for gen in range(3):
        knots, best = prob.solve(x0, g, 1)
        pop = torch.empty((prob.D, prob.P), device="cuda")
        cost = torch.empty(prob.P, device="cuda")
        el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
        prob.get_state(pop, cost, el)
        torch.cuda.synchronize()
        pop, cost, el = pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()
        if prev is None:
            ref = O.breed_cold(9, gen + 1, b[:, 0], b[:, 1], wl.m, wl.p, wl.P)
        else:
            ref = O.breed_warm(9, gen + 1, prev[0], prev[1], b[:, 0], b[:, 1], wl.m, wl.p,
                               wl.sigma)
        np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
        oc = M.cost_population(x0, g, pop, box=box)
        assert rel_err(cost, oc).max() <= COST_RTOL
        check_elites(el, oc, wl.E, rtol=2 * COST_RTOL)
        assert best == cost[el[0]]
        np.testing.assert_array_equal(knots, pop[:, el[0]])
        prev = (pop, el)
    prob.close()


def test_closed_loop_with_stop_matches_oracle_loop():
    wl = W.small(dof=2, T=20, p=3, P=200, E=12)
    lo = np.full(wl.n, -0.125, np.float32)
    hi = np.full(wl.n, 0.125, np.float32)
    rho = np.full(wl.n, 16.0, np.float32)
    x0 = np.zeros(wl.n)
    g = np.r_[np.full(wl.dof, 0.5), np.zeros(wl.dof)]  # beyond the stop
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    steps, G = 20, 2
    prob = gpu_problem(wl, seed=6)
    prob.set_state_box(lo, hi, rho, clamp=True, penalty=True)
    out = prob.closed_loop(A, B, x0, g, steps, G)
    assert ((out["x"] >= lo) & (out["x"] <= hi)).all()
    assert (out["x"] == hi).any()  # the plant reached the stop
    ga = O.EMPC(oracle_model(wl), wl.P, wl.E, seed=6, sigma=wl.sigma,
                box=O.StateBox(lo, hi, rho, clamp=True, penalty=True))
    xs, us, J, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, steps, G)
    np.testing.assert_array_equal(out["u"][0], us[0])
    np.testing.assert_allclose(out["x"][1:], np.clip(out["x"][:-1] @ A.T + out["u"] @ B.T,
                                                     lo, hi), rtol=0, atol=1e-12)
    assert abs(out["actual_cost"] - J) <= 1e-3 * J
    prob.close()


def test_state_box_rejects_bad_requests():
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=2, T=10, p=2, P=64, E=4)
    n = wl.n
    prob = gpu_problem(wl)
    bad = [
        dict(lo=np.ones(n), hi=np.zeros(n), clamp=True),               # lo > hi
        dict(lo=np.full(n, np.nan), clamp=True),                       # NaN bound
        dict(lo=np.full(n, np.inf), hi=np.full(n, np.inf), clamp=True),  # lo = +inf
        dict(rho=-np.ones(n), penalty=True),                           # negative weight
        dict(rho=np.full(n, np.inf), penalty=True),                    # infinite weight
    ]
    for kw in bad:
        with pytest.raises(E.EmpcError) as ei:
            prob.set_state_box(**kw)
        assert ei.value.status == E.EMPC_EINVAL, kw
    prob.close()
    for cfg in (dict(evaluator=E.EMPC_EVAL_CONDENSED), dict(refine_steps=2)):
        prob = gpu_problem(wl, **cfg)
        with pytest.raises(E.EmpcError) as ei:
            prob.set_state_box(-np.ones(n), np.ones(n), clamp=True)
        assert ei.value.status == E.EMPC_EUNSUPPORTED
        prob.set_state_box()  # turning the hook off is always allowed
        prob.close()
