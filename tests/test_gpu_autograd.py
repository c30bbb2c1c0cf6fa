"""The adjoint kernel behind torch autograd (rollout_cost) against the FP64
oracle.

For loss = sum_c w_c J_c the gradient with respect to candidate c's knots is
w_c dJ_c/dU_c.  Bars: the costs within 1e-5 relative of the oracle; the
gradient within 2e-4 of max |w_c dJ_c/dU_c| per candidate (the adjoint
kernel's bar); without requires_grad the costs come from the rollout kernel,
bit for bit those of empc_evaluate."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_problem, oracle_model, rel_err

pytestmark = pytest.mark.gpu
COST_RTOL = 1e-5
GRAD_TOL = 2e-4


@pytest.mark.parametrize("kw", [
    dict(dof=3, T=23, p=4, P=70, E=8),
    dict(dof=24, radius=3, dt=0.005, T=60, p=5, P=40, E=4),
])
def test_autograd_gradient_matches_oracle(kw):
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(**kw)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    rng = np.random.default_rng(3)
    pop_np = rng.uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    w_np = rng.uniform(0.5, 2.0, wl.P).astype(np.float32)
    prob = gpu_problem(wl)
    pop = torch.from_numpy(pop_np).cuda().requires_grad_()
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    J = E.rollout_cost(prob, x0d, gd, pop)
    loss = (torch.from_numpy(w_np).cuda() * J).sum()
    loss.backward()
    torch.cuda.synchronize()
    Jc = J.detach().cpu().numpy()
    assert rel_err(Jc, M.cost_population(x0, g, pop_np)).max() <= COST_RTOL
    got = pop.grad.cpu().numpy()
    for c in range(wl.P):
        _, gref = M.grad(x0, g, pop_np[:, c].astype(np.float64))
        gref = float(w_np[c]) * gref
        assert np.abs(got[:, c] - gref).max() <= GRAD_TOL * np.abs(gref).max(), c
    prob.close()


def test_no_grad_costs_are_the_rollout_costs():
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=4, T=30, p=4, P=96, E=8)
    x0, g = wl.start_goal()
    pop_np = np.random.default_rng(4).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    prob = gpu_problem(wl)
    pop = torch.from_numpy(pop_np).cuda()
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    J = E.rollout_cost(prob, x0d, gd, pop)
    ref = torch.empty(wl.P, device="cuda")
    prob.evaluate(x0d, gd, pop, ref)
    torch.cuda.synchronize()
    assert not J.requires_grad
    np.testing.assert_array_equal(J.cpu().numpy().view(np.uint32),
                                  ref.cpu().numpy().view(np.uint32))
    prob.close()


def test_gradient_refused_with_a_state_box():
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=2, T=10, p=2, P=32, E=4)
    prob = gpu_problem(wl)
    prob.set_state_box(-np.ones(wl.n), np.ones(wl.n), clamp=True)
    pop = torch.zeros((wl.m * wl.p, wl.P), device="cuda", requires_grad=True)
    z = torch.zeros(wl.n, device="cuda")
    with pytest.raises(E.EmpcError) as ei:
        E.rollout_cost(prob, z, z, pop)
    assert ei.value.status == E.EMPC_EUNSUPPORTED
    prob.close()


def test_bf16_handle_gradient_is_fp32():
    """The adjoint runs in FP32 whatever the rollout precision."""
    import torch
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=3, T=20, p=3, P=64, E=4)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop_np = np.random.default_rng(5).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    prob = gpu_problem(wl, precision=E.EMPC_BF16)
    pop = torch.from_numpy(pop_np).cuda().requires_grad_()
    J = E.rollout_cost(prob, torch.tensor(x0, dtype=torch.float32, device="cuda"),
                       torch.tensor(g, dtype=torch.float32, device="cuda"), pop)
    J.sum().backward()
    torch.cuda.synchronize()
    assert rel_err(J.detach().cpu().numpy(), M.cost_population(x0, g, pop_np)).max() <= COST_RTOL
    got = pop.grad.cpu().numpy()
    for c in range(0, wl.P, 9):
        _, gref = M.grad(x0, g, pop_np[:, c].astype(np.float64))
        assert np.abs(got[:, c] - gref).max() <= GRAD_TOL * np.abs(gref).max(), c
    prob.close()
