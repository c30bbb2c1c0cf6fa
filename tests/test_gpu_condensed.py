"""Condensed quadratic-form evaluator (Sec. IV-B and IV-E) against the FP64
oracle: the tensor-core kernel (padded D up to 256) and the CUDA-core one
(wider D).

The GPU evaluates J(U) = U'HU + g'U + c0 in FP32, with H rounded from the
host's FP64 Hessian and g, c0 from one FP32 adjoint evaluation at U = 0.  Its
rounding acts on the three terms, not on their (possibly much smaller) sum,
so the bar is stated against their size: |J_gpu - J_fp64| <= 1e-5 (|U'HU| +
|g'U| + |c0|), with g = 2f and H, f, c0 the oracle's FP64 condensed form.
On these workloads the terms do not cancel much, and the error relative to
J itself is held to the rollout's bar as well: |J_gpu - J_fp64| <= 1e-5 |J|
(measured: at most about 5e-7).
Breeding is the same kernel as with the rollout, so populations match the
oracle bit for bit; the elite set must agree wherever the FP64 costs are
separated by more than the evaluator's error bound."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, gpu_problem, oracle_model, report

pytestmark = pytest.mark.gpu
TERM_RTOL = 1e-5


def _state(prob):
    import torch
    pop = torch.empty((prob.D, prob.P), device="cuda")
    cost = torch.empty(prob.P, device="cuda")
    el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
    prob.get_state(pop, cost, el)
    torch.cuda.synchronize()
    return pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()


def _lockstep(wl, generations, seed=5, sample=None):
    import paper_2001_04931_gb300 as E
    prob = gpu_problem(wl, seed=seed, evaluator=E.EMPC_EVAL_CONDENSED)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    H, f, c0 = M.condensed(x0, g)
    b = wl.bounds().astype(np.float32)
    prev = None
    bests = []
    for gen in range(generations):
        knots, best = prob.solve(x0, g, 1)
        pop, cost, el = _state(prob)
        if prev is None:
            ref = O.breed_cold(seed, gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P)
        else:
            ref = O.breed_warm(seed, gen, prev[0], prev[2], b[:, 0], b[:, 1], wl.m, wl.p,
                               wl.sigma)
        np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
        cols = np.arange(wl.P) if sample is None else np.unique(np.r_[sample, el])
        U = pop[:, cols].astype(np.float64)
        oc = M.cost_population(x0, g, pop[:, cols])
        scale = np.abs(np.einsum("ic,ij,jc->c", U, H, U)) + np.abs(2.0 * f @ U) + abs(c0)
        err = np.abs(cost[cols] - oc)
        report(f"condensed_n{wl.n}_P{wl.P}_gen{gen}", max_rel_terms=np.max(err / scale),
               max_rel_J=np.max(err / np.abs(oc)))
        assert (err <= TERM_RTOL * scale).all(), float(np.max(err / scale))
        assert (err <= TERM_RTOL * np.abs(oc)).all(), float(np.max(err / np.abs(oc)))
        if sample is None:
            check_elites(el, oc, wl.E, rtol=2.0 * float(np.max(TERM_RTOL * scale / np.abs(oc))))
        assert best == cost[el[0]]
        np.testing.assert_array_equal(knots, pop[:, el[0]])
        bests.append(best)
        prev = (pop, cost, el)
    assert all(b2 <= b1 for b1, b2 in zip(bests, bests[1:]))
    prob.close()


@pytest.mark.parametrize("kw", [
    dict(dof=3, T=23, p=4, P=200, E=16),
    dict(dof=2, T=1, p=1, P=33, E=3),
    dict(dof=5, T=40, p=40, P=70, E=6),     # D = 200: the tensor cores' widest N
    dict(dof=8, T=30, p=7, P=130, E=10),
    dict(dof=30, T=40, p=10, P=130, E=8),   # D = 300 > 256: the CUDA-core kernel
])
def test_condensed_lockstep_small(kw):
    _lockstep(W.small(**kw), 3)


def test_condensed_lockstep_c2_sampled():
    wl = W.config("c2")
    rng = np.random.default_rng(11)
    _lockstep(wl, 2, sample=rng.choice(wl.P, 256, replace=False))


def test_condensed_matches_rollout_costs_on_one_population():
    """Both evaluators on the same bred population: equal within the bar."""
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=6, radius=2, T=45, p=5, P=300, E=20)
    x0, g = wl.start_goal()
    pr = gpu_problem(wl, seed=9)
    pc = gpu_problem(wl, seed=9, evaluator=E.EMPC_EVAL_CONDENSED)
    pr.solve(x0, g, 2)
    pc.solve(x0, g, 1)
    pop_r, cost_r, el_r = _state(pr)
    # hand the rollout handle's population to the condensed one and evaluate it there
    pc.set_state(torch.from_numpy(pop_r).cuda(), torch.from_numpy(cost_r).cuda(),
                 torch.from_numpy(el_r).cuda())
    _, cost_c, _ = _state(pc)
    M = oracle_model(wl)
    H, f, c0 = M.condensed(x0, g)
    U = pop_r.astype(np.float64)
    scale = np.abs(np.einsum("ic,ij,jc->c", U, H, U)) + np.abs(2.0 * f @ U) + abs(c0)
    # set_state keeps the given costs; a one-generation solve re-evaluates the elites
    pc.solve(x0, g, 1)
    pop_c2, cost_c2, el_c2 = _state(pc)
    oc = M.cost_population(x0, g, pop_c2)
    Uc = pop_c2.astype(np.float64)
    sc = np.abs(np.einsum("ic,ij,jc->c", Uc, H, Uc)) + np.abs(2.0 * f @ Uc) + abs(c0)
    assert (np.abs(cost_c2 - oc) <= TERM_RTOL * sc).all()
    pr.close()
    pc.close()
