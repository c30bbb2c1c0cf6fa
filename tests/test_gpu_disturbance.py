"""The constant disturbance w_d of Eq. first_order_integration on the GPU
against the FP64 oracle, through the C ABI.

Bars as for the plain path: costs within 1e-5 relative in both FP32 kernel
families (and with the state box, which acts after w_d); the adjoint within
2e-4 of max |dJ/dU| per candidate; the condensed evaluator within 1e-5 of
the size of its terms; selection consistent with the FP64 costs; the closed
loop's plant carries w_d.  A zero w_d is no disturbance, bit for bit."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, gpu_problem, rel_err

pytestmark = pytest.mark.gpu
COST_RTOL = 1e-5
GRAD_TOL = 2e-4


def _w(n, seed=0):
    return 0.02 * np.random.default_rng([seed, 77]).standard_normal(n)


def _oracle(wl, w, A=None, B=None):
    if A is None:
        A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    return O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p, w=w)


def _dev(v):
    import torch
    return torch.tensor(np.asarray(v), dtype=torch.float32, device="cuda")


def _evaluate(prob, x0, g, pop_np):
    import torch
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    cost = torch.empty(pop.shape[1], device="cuda")
    prob.evaluate(_dev(x0), _dev(g), pop, cost)
    torch.cuda.synchronize()
    return cost.cpu().numpy()


def _tiles_by_kind(wl):
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
])
def test_costs_with_disturbance_match_oracle(kw):
    wl = W.small(**kw)
    w = _w(wl.n)
    M = _oracle(wl, w)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(2).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    ref = M.cost_population(x0, g, pop)
    for kind, tile in _tiles_by_kind(wl).items():
        prob = gpu_problem(wl, tile=tile)
        prob.set_disturbance(w)
        got = _evaluate(prob, x0, g, pop)
        assert rel_err(got, ref).max() <= COST_RTOL, (kind, float(rel_err(got, ref).max()))
        # with the state box as well: w_d first, then the hook
        lo, hi = np.full(wl.n, -0.25, np.float32), np.full(wl.n, 0.25, np.float32)
        rho = np.full(wl.n, 8.0, np.float32)
        prob.set_state_box(lo, hi, rho, clamp=True, penalty=True)
        refb = M.cost_population(x0, g, pop, box=O.StateBox(lo, hi, rho, clamp=True,
                                                            penalty=True))
        got = _evaluate(prob, x0, g, pop)
        assert rel_err(got, refb).max() <= COST_RTOL, kind
        prob.close()


def test_large_state_block_family_with_hooks():
    """n = 80 runs only in the block family (state class 128, padded rows)."""
    wl = W.small(dof=40, T=20, p=3, P=64, E=4)
    w = _w(wl.n, 9)
    M = _oracle(wl, w)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(8).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    prob = gpu_problem(wl)
    assert prob.info().tile_kind == 0
    prob.set_disturbance(w)
    lo, hi = np.full(wl.n, -0.25, np.float32), np.full(wl.n, 0.25, np.float32)
    rho = np.full(wl.n, 8.0, np.float32)
    prob.set_state_box(lo, hi, rho, clamp=True, penalty=True)
    ref = M.cost_population(x0, g, pop, box=O.StateBox(lo, hi, rho, clamp=True, penalty=True))
    got = _evaluate(prob, x0, g, pop)
    assert rel_err(got, ref).max() <= COST_RTOL
    prob.close()


def test_zero_disturbance_is_none_bitwise():
    wl = W.small(dof=4, T=30, p=4, P=96, E=8)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(3).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    prob = gpu_problem(wl)
    plain = _evaluate(prob, x0, g, pop)
    prob.set_disturbance(np.zeros(wl.n))
    np.testing.assert_array_equal(_evaluate(prob, x0, g, pop).view(np.uint32),
                                  plain.view(np.uint32))
    prob.set_disturbance(_w(wl.n))
    assert (_evaluate(prob, x0, g, pop) != plain).any()
    prob.set_disturbance(None)
    np.testing.assert_array_equal(_evaluate(prob, x0, g, pop).view(np.uint32),
                                  plain.view(np.uint32))
    prob.close()


def test_solve_with_disturbance_selects_by_oracle_costs():
    import torch
    wl = W.small(dof=3, T=30, p=4, P=256, E=12)
    w = _w(wl.n, 1)
    M = _oracle(wl, w)
    x0, g = wl.start_goal()
    prob = gpu_problem(wl, seed=4)
    prob.set_disturbance(w)
    for _ in range(3):
        knots, best = prob.solve(x0, g, 1)
        pop = torch.empty((prob.D, prob.P), device="cuda")
        cost = torch.empty(prob.P, device="cuda")
        el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
        prob.get_state(pop, cost, el)
        torch.cuda.synchronize()
        pop, cost, el = pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()
        oc = M.cost_population(x0, g, pop)
        assert rel_err(cost, oc).max() <= COST_RTOL
        check_elites(el, oc, wl.E, rtol=2 * COST_RTOL)
        assert best == cost[el[0]]
        np.testing.assert_array_equal(knots, pop[:, el[0]])
    prob.close()


def test_gradient_with_disturbance_matches_oracle():
    import torch
    wl = W.small(dof=3, T=23, p=4, P=40, E=4)
    w = _w(wl.n, 2)
    M = _oracle(wl, w)
    x0, g = wl.start_goal()
    pop_np = np.random.default_rng(5).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    prob = gpu_problem(wl)
    prob.set_disturbance(w)
    pop = torch.from_numpy(pop_np).cuda()
    grad = torch.empty_like(pop)
    cost = torch.empty(wl.P, device="cuda")
    prob.grad(_dev(x0), _dev(g), pop, grad, cost)
    torch.cuda.synchronize()
    gg, cc = grad.cpu().numpy(), cost.cpu().numpy()
    assert rel_err(cc, M.cost_population(x0, g, pop_np)).max() <= COST_RTOL
    for c in range(wl.P):
        _, gref = M.grad(x0, g, pop_np[:, c].astype(np.float64))
        assert np.abs(gg[:, c] - gref).max() <= GRAD_TOL * np.abs(gref).max(), c
    prob.close()


def test_condensed_evaluator_with_disturbance():
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=3, T=23, p=4, P=200, E=16)
    w = _w(wl.n, 3)
    M = _oracle(wl, w)
    x0, g = wl.start_goal()
    H, f, c0 = M.condensed(x0, g)
    prob = gpu_problem(wl, evaluator=E.EMPC_EVAL_CONDENSED)
    prob.set_disturbance(w)
    import torch
    prob.solve(x0, g, 1)  # the condensed terms come from one adjoint pass per solve
    pop = torch.empty((prob.D, prob.P), device="cuda")
    cost = torch.empty(prob.P, device="cuda")
    prob.get_state(pop, cost, None)
    torch.cuda.synchronize()
    U = pop.cpu().numpy().astype(np.float64)
    oc = M.cost_population(x0, g, pop.cpu().numpy())
    scale = np.abs(np.einsum("ic,ij,jc->c", U, H, U)) + np.abs(2.0 * f @ U) + abs(c0)
    assert (np.abs(cost.cpu().numpy() - oc) <= 1e-5 * scale).all()
    prob.close()


def test_closed_loop_plant_carries_disturbance():
    wl = W.small(dof=2, T=20, p=3, P=200, E=12)
    w = _w(wl.n, 4)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    x0 = np.zeros(wl.n)
    g = np.r_[np.full(wl.dof, 0.5), np.zeros(wl.dof)]
    steps, G = 20, 2
    prob = gpu_problem(wl, seed=6)
    prob.set_disturbance(w)
    out = prob.closed_loop(A, B, x0, g, steps, G)
    np.testing.assert_allclose(out["x"][1:], out["x"][:-1] @ A.T + out["u"] @ B.T + w,
                               rtol=0, atol=1e-12)
    ga = O.EMPC(_oracle(wl, w), wl.P, wl.E, seed=6, sigma=wl.sigma)
    xs, us, J, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, steps, G)
    np.testing.assert_array_equal(out["u"][0], us[0])
    assert abs(out["actual_cost"] - J) <= 1e-3 * J
    prob.close()


def test_disturbance_rejects_bad_requests():
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=2, T=10, p=2, P=64, E=4)
    prob = gpu_problem(wl)
    with pytest.raises(E.EmpcError) as ei:
        prob.set_disturbance(np.full(wl.n, np.nan))
    assert ei.value.status == E.EMPC_EINVAL
    prob.close()
    prob = gpu_problem(wl, precision=E.EMPC_BF16)
    with pytest.raises(E.EmpcError) as ei:
        prob.set_disturbance(_w(wl.n))
    assert ei.value.status == E.EMPC_EUNSUPPORTED
    prob.set_disturbance(np.zeros(wl.n))  # no disturbance is always allowed
    prob.close()
