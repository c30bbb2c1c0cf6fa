"""BF16 tensor-core rollout (tcgen05) against the FP64 oracle.

Breeding is the same FP32 code as the CUDA-core path, so bred populations
match the oracle bit for bit.  The per-step product takes D, B_d, x and u in
BF16 (unit roundoff 2^-9 = 2e-3) with FP32 accumulation, so the cost is only
close: these tests bound the relative cost error at 3e-2 (max) and 5e-3
(median) on the small workloads below, and at 1e-3 (max) and 2e-4 (median)
over the full 200-step horizon of the 64-DoF chain (measured there: about
1.5e-4 max and 6e-5 median), and require the elite set to be drawn from the
FP64 cost order within that tolerance."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_problem, oracle_model, rel_err, report

pytestmark = pytest.mark.gpu
MAX_RTOL, MED_RTOL = 3e-2, 5e-3
C5_MAX_RTOL, C5_MED_RTOL = 1e-3, 2e-4


def _eval(prob, x0, g, pop_np):
    import torch
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    cost = torch.empty(pop.shape[1], device="cuda")
    prob.evaluate(torch.tensor(x0, dtype=torch.float32, device="cuda"),
                  torch.tensor(g, dtype=torch.float32, device="cuda"), pop, cost)
    torch.cuda.synchronize()
    return cost.cpu().numpy()


@pytest.mark.parametrize("kw", [
    dict(dof=64, radius=3, dt=0.005, T=60, p=8, P=300, E=16, q_pos=10.0, q_vel=1.0, r=1e-4),
    dict(dof=4, T=30, p=4, P=200, E=8),
    dict(dof=40, radius=3, dt=0.005, T=25, p=3, P=129, E=8),
    # one knot: a constant input
    dict(dof=6, T=17, p=1, P=130, E=8),
    # a one-step horizon: one commit, no operand written for a next step
    dict(dof=4, T=1, p=1, P=130, E=8),
    # fewer candidates than one tile: most TMEM lanes hold no candidate
    dict(dof=3, T=10, p=2, P=50, E=4),
])
def test_bf16_costs_against_oracle(kw):
    import paper_2001_04931_gb300 as E
    wl = W.small(**kw)
    prob = gpu_problem(wl, precision=E.EMPC_BF16)
    assert prob.info().tile_kind == 2
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(0).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    err = rel_err(_eval(prob, x0, g, pop), M.cost_population(x0, g, pop))
    report(f"bf16_costs_n{wl.n}_T{wl.T}", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= MAX_RTOL and np.median(err) <= MED_RTOL, (err.max(), np.median(err))
    prob.close()


def test_bf16_lockstep_breeding_bit_exact():
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=16, radius=3, dt=0.005, T=40, p=5, P=256, E=16)
    prob = gpu_problem(wl, seed=7, precision=E.EMPC_BF16)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    b = wl.bounds().astype(np.float32)
    prev = None
    for gen in range(3):
        prob.solve(x0, g, 1)
        pop = torch.empty((prob.D, prob.P), device="cuda")
        cost = torch.empty(prob.P, device="cuda")
        el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
        prob.get_state(pop, cost, el)
        torch.cuda.synchronize()
        pop, cost, el = pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()
        ref = (O.breed_cold(7, gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P) if prev is None else
               O.breed_warm(7, gen, prev[0], prev[2], b[:, 0], b[:, 1], wl.m, wl.p, wl.sigma))
        np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
        oc = M.cost_population(x0, g, pop)
        assert rel_err(cost, oc).max() <= MAX_RTOL
        # elites by the GPU's BF16 costs: every FP64 cost of an elite is within
        # the tolerance band of the E-th smallest FP64 cost
        tE = np.sort(oc)[wl.E - 1]
        assert (oc[el] <= tE * (1 + 2 * MAX_RTOL)).all()
        prev = (pop, cost, el)
    prob.close()


def _c5_workload(P):
    """The 64-DoF chain of the large workload (n = 128, m = 64, T = 200, 8
    knots, Q = diag(10 pos, 1 vel), R = 1e-4 I) at a population the oracle
    costs in seconds."""
    return W.small(dof=64, radius=3, dt=0.005, T=200, p=8, P=P, E=16, q_pos=10.0, q_vel=1.0,
                   r=1e-4)


def test_bf16_costs_c5_horizon_cold_population():
    """The full horizon of the 64-DoF workload (rounding compounds over 200
    steps): 4.5 tiles of candidates drawn uniformly in the bounds."""
    import paper_2001_04931_gb300 as E
    wl = _c5_workload(577)
    prob = gpu_problem(wl, precision=E.EMPC_BF16)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(4).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    err = rel_err(_eval(prob, x0, g, pop), M.cost_population(x0, g, pop))
    report("bf16_c5_horizon_cold", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= C5_MAX_RTOL and np.median(err) <= C5_MED_RTOL, (err.max(),
                                                                        np.median(err))
    prob.close()


def test_bf16_costs_c5_horizon_evolved_population():
    """The same workload after six BF16 generations: the population the
    search actually evaluates (near-optimal plans, smaller costs), every
    candidate against the FP64 oracle; the elites come from the FP64 order
    within the error band."""
    import torch
    import paper_2001_04931_gb300 as E
    wl = _c5_workload(512)
    prob = gpu_problem(wl, seed=2, precision=E.EMPC_BF16)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    prob.solve(x0, g, 6)
    pop = torch.empty((prob.D, prob.P), device="cuda")
    cost = torch.empty(prob.P, device="cuda")
    el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
    prob.get_state(pop, cost, el)
    torch.cuda.synchronize()
    pop, cost, el = pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()
    oc = M.cost_population(x0, g, pop)
    err = rel_err(cost, oc)
    report("bf16_c5_horizon_evolved", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= C5_MAX_RTOL and np.median(err) <= C5_MED_RTOL, (err.max(),
                                                                        np.median(err))
    tE = np.sort(oc)[wl.E - 1]
    assert (oc[el] <= tE * (1 + 2 * C5_MAX_RTOL)).all()
    prob.close()


def test_bf16_wait_runs_out_and_reports_timeout():
    """Failure detection of the tensor-core rollout without a GPU fault: the
    MMA issuer is made to stop at step 7 (host-side injection), so the other
    threads' bounded waits run out after 50 ms; the solve reports
    EMPC_ETIMEOUT, and after the injection is cleared the same handle solves
    again with costs matching the oracle (the context stayed usable)."""
    import time
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=16, radius=3, dt=0.005, T=40, p=5, P=256, E=16)
    prob = gpu_problem(wl, seed=5, precision=E.EMPC_BF16)
    x0, g = wl.start_goal()
    prob.inject_stall(7, 0.05)
    t = time.perf_counter()
    with pytest.raises(E.EmpcError) as ei:
        prob.solve(x0, g, 1)
    assert ei.value.status == E.EMPC_ETIMEOUT
    assert time.perf_counter() - t < 30.0
    prob.inject_stall(-1, 1.0)
    prob.reset()
    gen = prob.info().generation  # the counter moved on with the failed solve
    prob.solve(x0, g, 1)
    pop = torch.empty((prob.D, prob.P), device="cuda")
    cost = torch.empty(prob.P, device="cuda")
    prob.get_state(pop, cost, None)
    torch.cuda.synchronize()
    pop, cost = pop.cpu().numpy(), cost.cpu().numpy()
    b = wl.bounds().astype(np.float32)
    np.testing.assert_array_equal(
        pop.view(np.uint32),
        O.breed_cold(5, gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P).view(np.uint32))
    assert rel_err(cost, oracle_model(wl).cost_population(x0, g, pop)).max() <= MAX_RTOL
    prob.close()


def test_inject_stall_is_for_bf16_handles():
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=3, T=20, p=4, P=128, E=8)
    prob = gpu_problem(wl)
    with pytest.raises(E.EmpcError) as ei:
        prob.inject_stall(3, 0.1)
    assert ei.value.status == E.EMPC_EUNSUPPORTED
    prob.close()
    bf = gpu_problem(wl, precision=E.EMPC_BF16)
    for step, t in ((-2, 0.1), (3, 0.0), (3, 61.0)):
        with pytest.raises(E.EmpcError) as ei:
            bf.inject_stall(step, t)
        assert ei.value.status == E.EMPC_EINVAL
    bf.close()


def test_bf16_rejects_sizes_beyond_its_tile():
    """The tensor-core tile holds n <= 128 states and m <= 64 inputs: a model
    with m = 70 inputs (n = 100, within the library's FP32 limits) is refused
    at create with BF16, not truncated, and accepted with FP32."""
    import paper_2001_04931_gb300 as E
    n, m = 100, 70
    rng = np.random.default_rng(3)
    A = np.eye(n) * 0.99
    B = rng.uniform(-0.01, 0.01, (n, m))
    Q, R = np.eye(n), 1e-3 * np.eye(m)
    bounds = np.tile([-1.0, 1.0], (m, 1))
    with pytest.raises(E.EmpcError) as ei:
        E.Problem(A, B, Q, R, bounds, 10, 2, 128, elite=8, precision=E.EMPC_BF16)
    assert ei.value.status == E.EMPC_EUNSUPPORTED
    E.Problem(A, B, Q, R, bounds, 10, 2, 128, elite=8).close()
