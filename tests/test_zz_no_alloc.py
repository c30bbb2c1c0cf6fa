"""empc_evaluate_noalloc (the allocation-free cost entry point) against the
handle API's empc_evaluate, through the C ABI, on two calls in a row.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

import workloads as W
from helpers import gpu_problem, rel_err

pytestmark = pytest.mark.gpu


def _costs_both_ways(wl, seed):
    import torch
    import paper_2001_04931_gb300 as E
    prob = gpu_problem(wl)
    A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    x0, g = wl.start_goal()
    x0d = torch.tensor(x0, dtype=torch.float32, device="cuda")
    gd = torch.tensor(g, dtype=torch.float32, device="cuda")
    pop = torch.from_numpy(np.random.default_rng(seed).uniform(
        -1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)).cuda()
    ref = torch.empty(wl.P, device="cuda")
    got = torch.full((wl.P,), float("nan"), device="cuda")
    prob.evaluate(x0d, gd, pop, ref)
    torch.cuda.synchronize()
    E.evaluate_noalloc(A, B, wl.Q(), wl.R(), wl.T, wl.p, x0d, gd, pop, got)
    torch.cuda.synchronize()
    prob.close()
    return got.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_matches_handle_evaluate_two_calls():
    # first call: 5-DoF chain; second call: the 24-DoF chain (larger tables,
    # different horizon and knots), so the second rewrites what the first left
    for wl, seed in [(W.small(dof=5, T=40, p=4, P=300, E=16), 0),
                     (W.small(dof=24, radius=3, dt=0.005, T=100, p=5, P=1000, E=32), 1)]:
        got, ref = _costs_both_ways(wl, seed)
        assert np.isfinite(got).all()
        assert rel_err(got, ref).max() <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_tables():
    import paper_2001_04931_gb300 as E
    import torch
    n, m = 66, 2
    dummy = torch.zeros(8, device="cuda")
    with pytest.raises(E.EmpcError) as ei:
        E.evaluate_noalloc(np.eye(n), np.ones((n, m)), np.eye(n), np.eye(m), 10, 3, dummy,
                           dummy, torch.zeros((m * 3, 4), device="cuda"), dummy)
    assert ei.value.status == E.EMPC_EINVAL
    with pytest.raises(E.EmpcError) as ei:
        E.evaluate_noalloc(np.eye(4), np.ones((4, 2)), np.eye(4), np.eye(2), 1025, 3, dummy,
                           dummy, torch.zeros((6, 4), device="cuda"), dummy)
    assert ei.value.status == E.EMPC_EINVAL
