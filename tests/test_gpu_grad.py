"""Adjoint gradient and elite refinement on the GPU against the FP64 oracle.

Gradient bar: max |g_gpu - g_ref| <= 2e-4 max |g_ref| over a candidate's
knots (FP32 adjoint over T <= 100 steps against FP64), checked against the
oracle's adjoint, the condensed form 2HU + 2f and FP64 central differences
(h = 1e-6) on 64 candidates.  Checkpoint recomputation repeats the forward
arithmetic exactly, so the gradient is bitwise independent of the interval."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_problem, oracle_model, rel_err

pytestmark = pytest.mark.gpu
GRAD_TOL = 2e-4


def _grad_gpu(prob, wl, x0, g, pop_np):
    import torch
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    grad = torch.empty_like(pop)
    cost = torch.empty(pop.shape[1], device="cuda")
    prob.grad(torch.tensor(x0, dtype=torch.float32, device="cuda"),
              torch.tensor(g, dtype=torch.float32, device="cuda"), pop, grad, cost)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), cost.cpu().numpy()


def _check_grad(gg, gref):
    for c in range(gg.shape[1]):
        scale = np.abs(gref[:, c]).max()
        assert np.abs(gg[:, c] - gref[:, c]).max() <= GRAD_TOL * scale, c


@pytest.mark.parametrize("kw", [
    dict(dof=3, T=23, p=4, P=70, E=8),
    dict(dof=1, T=1, p=1, P=9, E=1),
    dict(dof=2, T=12, p=12, P=40, E=4),
    dict(dof=24, radius=3, dt=0.005, T=100, p=5, P=64, q_pos=10.0, q_vel=1.0, r=1e-4),
])
def test_grad_matches_oracle_adjoint(kw):
    wl = W.small(**kw)
    prob = gpu_problem(wl)
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(0).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    gg, cost = _grad_gpu(prob, wl, x0, g, pop)
    ref = np.stack([M.grad(x0, g, pop[:, c].astype(np.float64))[1] for c in range(wl.P)], 1)
    _check_grad(gg, ref)
    assert rel_err(cost, M.cost_population(x0, g, pop)).max() <= 1e-5
    prob.close()


def test_grad_matches_condensed_and_central_differences_c3():
    """The 24-DoF workload (T=100, p=5, checkpoints every 10 steps): 64
    candidates against 2HU + 2f and FP64 central differences, h = 1e-6."""
    wl = W.config("c3")
    prob = gpu_problem(wl, ckpt_every=10)
    assert prob.info().ckpt_every == 10
    M = oracle_model(wl)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(3).uniform(-1, 1, (wl.m * wl.p, 64)).astype(np.float32)
    gg, _ = _grad_gpu(prob, wl, x0, g, pop)
    H, f, _ = M.condensed(x0, g)
    U = pop.astype(np.float64)
    _check_grad(gg, 2 * H @ U + 2 * f[:, None])
    h = 1e-6
    for c in range(64):
        fd = np.zeros(wl.m * wl.p)
        for q in range(wl.m * wl.p):
            e = np.zeros_like(fd)
            e[q] = h
            fd[q] = (M.cost(x0, g, U[:, c] + e) - M.cost(x0, g, U[:, c] - e)) / (2 * h)
        scale = np.abs(fd).max()
        assert np.abs(gg[:, c] - fd).max() <= GRAD_TOL * scale
    prob.close()


def test_grad_independent_of_checkpoint_interval():
    wl = W.small(dof=4, T=37, p=5, P=50)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(4).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    outs = []
    for ce in [1, 3, 7, 37]:
        prob = gpu_problem(wl, ckpt_every=ce)
        outs.append(_grad_gpu(prob, wl, x0, g, pop))
        prob.close()
    for gg, cc in outs[1:]:
        np.testing.assert_array_equal(gg, outs[0][0])
        np.testing.assert_array_equal(cc, outs[0][1])


def test_refine_lockstep():
    """Children bit-exact from the selected elites; elite slots equal the
    oracle's refinement of the same elites within the gradient tolerance."""
    import torch
    wl = W.small(dof=3, T=30, p=4, P=128, E=8)
    M = oracle_model(wl)
    eta = M.lipschitz_step()
    prob = gpu_problem(wl, seed=5, refine_steps=3)
    assert abs(prob.info().refine_lr - eta) <= 1e-6 * eta
    x0, g = wl.start_goal()
    b = wl.bounds().astype(np.float32)
    ga = O.EMPC(M, wl.P, wl.E, seed=5, sigma=wl.sigma, refine_steps=3, refine_eta=eta)

    def state():
        pop = torch.empty((prob.D, prob.P), device="cuda")
        cost = torch.empty(prob.P, device="cuda")
        el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
        prob.get_state(pop, cost, el)
        torch.cuda.synchronize()
        return pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()

    prob.solve(x0, g, 1)
    prev = state()
    best = [prev[1][prev[2][0]]]
    for gen in range(1, 4):
        _, bc = prob.solve(x0, g, 1)
        pop, cost, el = state()
        ref = O.breed_warm(5, gen, prev[0], prev[2], b[:, 0], b[:, 1], wl.m, wl.p, wl.sigma)
        np.testing.assert_array_equal(pop[:, wl.E:].view(np.uint32), ref[:, wl.E:].view(np.uint32))
        refined = ga.refined_elites(x0, g, prev[0], prev[2])
        scale = np.abs(refined).max()
        assert np.abs(pop[:, :wl.E] - refined).max() <= 1e-4 * scale
        assert rel_err(cost, M.cost_population(x0, g, pop)).max() <= 1e-5
        best.append(bc)
        prev = (pop, cost, el)
    assert all(b2 <= b1 * (1 + 1e-6) for b1, b2 in zip(best, best[1:]))
    prob.close()
