"""empc_evaluate_noalloc, the entry point for callers that cannot allocate
memory while they run (a real-time control loop that must not stall on
cudaMalloc, or a process whose GPU memory another allocator reserved), through
the C ABI.  Its costs are compared with the handle API's empc_evaluate, on
calls in a row, within the 1e-5 bar of every cost test, and with the FP64
oracle at the same bar.

This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_problem, rel_err

pytestmark = pytest.mark.gpu
COST_RTOL = 1e-5


def _dev(v):
    import torch
    return torch.tensor(np.asarray(v), dtype=torch.float32, device="cuda")


def _pop(m, p, P, seed):
    import torch
    return torch.from_numpy(np.random.default_rng(seed).uniform(
        -1, 1, (m * p, P)).astype(np.float32)).cuda()


def _oracle_costs(wl, A, B, Q, R, x0, g, pop):
    b = wl.bounds()
    M = O.Model(A, B, Q, R, b[:, 0], b[:, 1], wl.T, wl.p)
    return M.cost_population(x0, g, pop.cpu().numpy())


def _costs_both_ways(wl, seed, Q=None, R=None, stream=None):
    """(noalloc costs, handle-API costs, oracle costs) of one population."""
    import torch
    import paper_2001_04931_gb300 as E
    Q = wl.Q() if Q is None else Q
    R = wl.R() if R is None else R
    A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    prob = E.Problem(A, B, Q, R, wl.bounds(), wl.T, wl.p, wl.P, seed=1, elite=wl.E)
    x0, g = wl.start_goal()
    x0d, gd = _dev(x0), _dev(g)
    pop = _pop(wl.m, wl.p, wl.P, seed)
    ref = torch.empty(wl.P, device="cuda")
    got = torch.full((wl.P,), float("nan"), device="cuda")
    prob.evaluate(x0d, gd, pop, ref)
    torch.cuda.synchronize()
    if stream is None:
        E.evaluate_noalloc(A, B, Q, R, wl.T, wl.p, x0d, gd, pop, got)
    else:
        with torch.cuda.stream(stream):
            E.evaluate_noalloc(A, B, Q, R, wl.T, wl.p, x0d, gd, pop, got,
                               stream=stream.cuda_stream)
    torch.cuda.synchronize()
    prob.close()
    Ao, Bo = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    oc = _oracle_costs(wl, Ao, Bo, Q, R, np.float32(x0).astype(np.float64),
                       np.float32(g).astype(np.float64), pop)
    return got.cpu().numpy(), ref.cpu().numpy(), oc


def test_noalloc_matches_handle_evaluate_two_calls():
    # first call: 5-DoF chain; second call: the 24-DoF chain (larger tables,
    # different horizon and knots), so the second rewrites what the first left
    for wl, seed in [(W.small(dof=5, T=40, p=4, P=300, E=16), 0),
                     (W.small(dof=24, radius=3, dt=0.005, T=100, p=5, P=1000, E=32), 1)]:
        got, ref, oc = _costs_both_ways(wl, seed)
        assert np.isfinite(got).all()
        assert rel_err(got, ref).max() <= COST_RTOL
        assert rel_err(got, oc).max() <= COST_RTOL


def test_noalloc_at_its_limits():
    """n = m = p = 64 and T = 1024, the largest call the fixed array takes:
    every table at its full size."""
    wl = W.small(dof=32, T=1024, p=64, P=37, E=4, radius=2, dt=0.002)
    import paper_2001_04931_gb300 as E
    # m = 64 inputs: two actuators per mass (the chain's own B, twice)
    Ac, Bc = wl.plant.Ac, np.hstack([wl.plant.Bc, 0.5 * wl.plant.Bc])
    A, B = E.discretize_zoh(Ac, Bc, wl.dt)
    n, m = 64, 64
    assert A.shape == (n, n) and B.shape == (n, m)
    Q, R = np.eye(n), 1e-3 * np.eye(m)
    x0, g = wl.start_goal()
    x0d, gd = _dev(x0), _dev(g)
    pop = _pop(m, wl.p, wl.P, 2)
    import torch
    got = torch.full((wl.P,), float("nan"), device="cuda")
    E.evaluate_noalloc(A, B, Q, R, wl.T, wl.p, x0d, gd, pop, got)
    bounds = np.tile([-1.0, 1.0], (m, 1))
    prob = E.Problem(A, B, Q, R, bounds, wl.T, wl.p, wl.P, seed=1, elite=wl.E)
    ref = torch.empty(wl.P, device="cuda")
    prob.evaluate(x0d, gd, pop, ref)
    torch.cuda.synchronize()
    prob.close()
    Ao, Bo = O.zoh(Ac, Bc, wl.dt)
    M = O.Model(Ao, Bo, Q, R, bounds[:, 0], bounds[:, 1], wl.T, wl.p)
    oc = M.cost_population(np.float32(x0).astype(np.float64), np.float32(g).astype(np.float64),
                           pop.cpu().numpy())
    got = got.cpu().numpy()
    assert rel_err(got, ref.cpu().numpy()).max() <= COST_RTOL
    assert rel_err(got, oc).max() <= COST_RTOL


def test_noalloc_dense_weights_and_a_side_stream():
    """Dense Q and R (Q's eigenbasis rotation and the rotated start and goal
    live in the fixed array too), on a non-default stream, then a diagonal
    call on the legacy stream after it."""
    import torch
    rng = np.random.default_rng(3)
    wl = W.small(dof=6, T=50, p=5, P=200, E=16, radius=2)
    L = rng.standard_normal((wl.n, wl.n))
    Lr = rng.standard_normal((wl.m, wl.m))
    Q = L @ L.T / wl.n + 0.05 * np.eye(wl.n)
    R = 1e-2 * (Lr @ Lr.T / wl.m + 0.05 * np.eye(wl.m))
    side = torch.cuda.Stream()
    got, ref, oc = _costs_both_ways(wl, 4, Q=Q, R=R, stream=side)
    assert rel_err(got, ref).max() <= COST_RTOL
    assert rel_err(got, oc).max() <= COST_RTOL
    got, ref, oc = _costs_both_ways(W.small(dof=3, T=20, p=3, P=64, E=4), 5)
    assert rel_err(got, ref).max() <= COST_RTOL
    assert rel_err(got, oc).max() <= COST_RTOL


@pytest.mark.parametrize("n,m,T,p", [(66, 2, 10, 3), (4, 65, 10, 3), (4, 2, 1025, 3),
                                     (4, 2, 100, 65), (4, 2, 10, 11), (4, 2, 10, 0)])
def test_noalloc_rejects_sizes_beyond_its_tables(n, m, T, p):
    import paper_2001_04931_gb300 as E
    import torch
    dummy = torch.zeros(n, device="cuda")
    with pytest.raises(E.EmpcError) as ei:
        E.evaluate_noalloc(np.eye(n), np.ones((n, m)), np.eye(n), np.eye(m), T, p, dummy, dummy,
                           torch.zeros((m * max(p, 1), 4), device="cuda"),
                           torch.zeros(4, device="cuda"))
    assert ei.value.status == E.EMPC_EINVAL


def test_noalloc_rejects_bad_weights():
    """Negative weights and weights whose symmetric part is not positive
    semidefinite, as empc_create rejects them."""
    import paper_2001_04931_gb300 as E
    import torch
    n, m = 4, 2
    x = torch.zeros(n, device="cuda")
    pop = torch.zeros((m * 3, 4), device="cuda")
    cost = torch.zeros(4, device="cuda")
    for Q, R in [(-np.eye(n), np.eye(m)), (np.eye(n), -np.eye(m)),
                 (np.kron(np.eye(2), [[1.0, 2.0], [2.0, 1.0]]), np.eye(m)),
                 (np.eye(n), np.array([[1.0, 3.0], [3.0, 1.0]]))]:
        with pytest.raises(E.EmpcError) as ei:
            E.evaluate_noalloc(np.eye(n), np.ones((n, m)), Q, R, 10, 3, x, x, pop, cost)
        assert ei.value.status == E.EMPC_EINVAL


def test_noalloc_wrapper_checks_every_buffer():
    """The binding checks each array and tensor against n, m and the knots
    before the C call, which trusts them."""
    import paper_2001_04931_gb300 as E
    import torch
    n, m, p, P = 4, 2, 3, 8
    A, B, Q, R = np.eye(n), np.ones((n, m)), np.eye(n), np.eye(m)
    x = torch.zeros(n, device="cuda")
    pop = torch.zeros((m * p, P), device="cuda")
    cost = torch.zeros(P, device="cuda")
    bad = [
        dict(A=np.eye(n + 1)), dict(Q=np.eye(n - 1)), dict(R=np.eye(m + 1)),
        dict(x0=torch.zeros(n + 1, device="cuda")), dict(x_goal=torch.zeros(n)),
        dict(x0=torch.zeros(n, device="cuda", dtype=torch.float64)),
        dict(pop=torch.zeros((m * p + 1, P), device="cuda")),
        dict(pop=torch.zeros((P, m * p), device="cuda").t()),
        dict(cost=torch.zeros(P + 1, device="cuda")),
        dict(cost=torch.zeros(P, device="cuda", dtype=torch.float16)),
    ]
    for kw in bad:
        args = dict(A=A, B=B, Q=Q, R=R, x0=x, x_goal=x, pop=pop, cost=cost, **{})
        args.update(kw)
        with pytest.raises(E.EmpcError) as ei:
            E.evaluate_noalloc(args["A"], args["B"], args["Q"], args["R"], 10, p, args["x0"],
                               args["x_goal"], args["pop"], args["cost"])
        assert ei.value.status == E.EMPC_EINVAL, kw
