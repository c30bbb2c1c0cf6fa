"""Dense (non-diagonal) Q and R, the general weights of Eq. mpc_problem,
against the FP64 oracle, which takes them as they are (x'Qx and u'Ru in
full).

The library diagonalizes a non-diagonal Q on the host and runs the rollouts
in its eigenbasis, and adds a dense R through the knot-weight Gram; none of
that is shared with the oracle.  Bars as everywhere: costs within 1e-5
relative, gradients within 2e-4 of max|dJ/dU| per candidate, bred
populations bit-exact, elites checked, batched solves bit-identical to
single-problem ones."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import check_elites, gpu_problem, rel_err, report

pytestmark = pytest.mark.gpu
COST_RTOL = 1e-5


def spd(k, seed, scale=1.0, floor=0.05):
    """A random symmetric positive definite k x k matrix with entries of
    order `scale` (a Wishart draw plus a floor on the spectrum)."""
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((k, k))
    return scale * (L @ L.T / k + floor * np.eye(k))


def dense_workload(dof=5, T=40, p=4, P=300, E=16, radius=1, dt=0.01, seed=0):
    wl = W.small(dof=dof, T=T, p=p, P=P, E=E, radius=radius, dt=dt, seed=seed)
    Q = spd(wl.n, 100 + seed, 2.0)
    R = spd(wl.m, 200 + seed, 1e-2)
    return wl, Q, R


def _problem(wl, Q, R, seed=1, **cfg):
    import paper_2001_04931_gb300 as E
    A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    return E.Problem(A, B, Q, R, wl.bounds(), wl.T, wl.p, wl.P, seed=seed, elite=wl.E,
                     sigma=wl.sigma, **cfg)


def _oracle(wl, Q, R):
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    return O.Model(A, B, Q, R, b[:, 0], b[:, 1], wl.T, wl.p)


def _dev(v):
    import torch
    return torch.tensor(np.asarray(v), dtype=torch.float32, device="cuda")


def _eval(prob, x0, g, pop_np):
    import torch
    pop = torch.from_numpy(np.ascontiguousarray(pop_np, np.float32)).cuda()
    cost = torch.empty(pop.shape[1], device="cuda")
    prob.evaluate(_dev(x0), _dev(g), pop, cost)
    torch.cuda.synchronize()
    return cost.cpu().numpy()


def _state(prob):
    import torch
    pop = torch.empty((prob.D, prob.P), device="cuda")
    cost = torch.empty(prob.P, device="cuda")
    el = torch.empty(prob.E, device="cuda", dtype=torch.int32)
    prob.get_state(pop, cost, el)
    torch.cuda.synchronize()
    return pop.cpu().numpy(), cost.cpu().numpy(), el.cpu().numpy()


@pytest.mark.parametrize("kw", [
    dict(dof=5, T=40, p=4, P=300),                                   # warp family, n = 10
    dict(dof=24, radius=3, dt=0.005, T=100, p=5, P=600, E=32),       # the 24-DoF chain
    dict(dof=64, radius=3, dt=0.005, T=60, p=8, P=300, E=16),        # block family, n = 128
])
def test_dense_weights_costs(kw):
    wl, Q, R = dense_workload(**kw)
    prob = _problem(wl, Q, R)
    M = _oracle(wl, Q, R)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(3).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    err = rel_err(_eval(prob, x0, g, pop), M.cost_population(x0, g, pop))
    report(f"dense_costs_n{wl.n}", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= COST_RTOL, float(err.max())
    prob.close()


def test_dense_weights_only_symmetric_part_counts():
    """x'Qx depends on the symmetric part alone: Q + S with S skew gives the
    same costs as Q (the library takes (Q + Q')/2; the two symmetric parts
    agree to FP64 rounding, so the costs agree far inside the bar)."""
    wl, Q, R = dense_workload(dof=4, T=30, p=3, P=128)
    rng = np.random.default_rng(9)
    S = rng.standard_normal((wl.n, wl.n))
    Sr = rng.standard_normal((wl.m, wl.m))
    a = _problem(wl, Q, R)
    b = _problem(wl, Q + (S - S.T), R + 1e-2 * (Sr - Sr.T))
    x0, g = wl.start_goal()
    pop = np.random.default_rng(4).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    assert rel_err(_eval(b, x0, g, pop), _eval(a, x0, g, pop)).max() <= 1e-6
    a.close()
    b.close()


def test_dense_weights_lockstep():
    """Three lockstep generations with dense weights: breeding bit-exact
    against the oracle's draws, every cost within 1e-5, elites checked, the
    reported best equal to rank 0."""
    wl, Q, R = dense_workload(dof=6, T=45, p=5, P=384, E=24, radius=2)
    seed = 7
    prob = _problem(wl, Q, R, seed=seed)
    M = _oracle(wl, Q, R)
    x0, g = wl.start_goal()
    b = wl.bounds().astype(np.float32)
    prev = None
    for gen in range(3):
        knots, best = prob.solve(x0, g, 1)
        pop, cost, el = _state(prob)
        ref = (O.breed_cold(seed, gen, b[:, 0], b[:, 1], wl.m, wl.p, wl.P) if prev is None else
               O.breed_warm(seed, gen, prev[0], prev[2], b[:, 0], b[:, 1], wl.m, wl.p, wl.sigma))
        np.testing.assert_array_equal(pop.view(np.uint32), ref.view(np.uint32))
        oc = M.cost_population(x0, g, pop)
        assert rel_err(cost, oc).max() <= COST_RTOL
        check_elites(el, oc, wl.E)
        assert best == cost[el[0]]
        np.testing.assert_array_equal(knots, pop[:, el[0]])
        prev = (pop, cost, el)
    prob.close()


def test_dense_weights_gradient():
    """empc_grad (the adjoint kernel, FP32) with dense weights against the
    oracle's FP64 adjoint, which central differences pin."""
    import torch
    wl, Q, R = dense_workload(dof=8, T=50, p=5, P=96, radius=2)
    prob = _problem(wl, Q, R)
    M = _oracle(wl, Q, R)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(5).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    pt = torch.from_numpy(pop).cuda()
    grad = torch.empty_like(pt)
    cost = torch.empty(wl.P, device="cuda")
    prob.grad(_dev(x0), _dev(g), pt, grad, cost)
    torch.cuda.synchronize()
    grad, cost = grad.cpu().numpy(), cost.cpu().numpy()
    worst = 0.0
    for c in range(wl.P):
        J, gr = M.grad(x0, g, pop[:, c].astype(np.float64))
        assert abs(cost[c] - J) <= COST_RTOL * abs(J)
        err = np.max(np.abs(grad[:, c] - gr)) / np.max(np.abs(gr))
        worst = max(worst, err)
    report("dense_grad", max_rel=worst)
    assert worst <= 2e-4
    prob.close()


def test_dense_weights_bf16():
    """The BF16 tensor-core rollout in Q's eigenbasis with a dense R, within
    the BF16 bars against the FP64 oracle."""
    import paper_2001_04931_gb300 as E
    wl, Q, R = dense_workload(dof=40, T=60, p=6, P=257, radius=3, dt=0.005)
    prob = _problem(wl, Q, R, precision=E.EMPC_BF16)
    assert prob.info().tile_kind == 2
    M = _oracle(wl, Q, R)
    x0, g = wl.start_goal()
    pop = np.random.default_rng(6).uniform(-1, 1, (wl.m * wl.p, wl.P)).astype(np.float32)
    err = rel_err(_eval(prob, x0, g, pop), M.cost_population(x0, g, pop))
    report("dense_bf16", max_rel=err.max(), median_rel=np.median(err))
    assert err.max() <= 3e-2 and np.median(err) <= 5e-3
    prob.close()


def test_dense_weights_condensed():
    """The condensed evaluator's H built with dense weights."""
    import paper_2001_04931_gb300 as E
    wl, Q, R = dense_workload(dof=5, T=35, p=5, P=200)
    prob = _problem(wl, Q, R, evaluator=E.EMPC_EVAL_CONDENSED)
    M = _oracle(wl, Q, R)
    x0, g = wl.start_goal()
    prob.solve(x0, g, 2)
    pop, cost, _ = _state(prob)
    err = rel_err(cost, M.cost_population(x0, g, pop))
    report("dense_condensed", max_rel=err.max())
    assert err.max() <= COST_RTOL
    prob.close()


def test_dense_weights_device_targets_and_disturbance():
    """Start and goal given on the device (rotated by a kernel) and a constant
    disturbance (rotated on the host) with a dense Q: solve_device's best
    cost is the FP64 cost of its best knots, within 1e-5."""
    import torch
    wl, Q, R = dense_workload(dof=5, T=40, p=4, P=256)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    w = np.random.default_rng(8).uniform(-0.01, 0.01, wl.n)
    b = wl.bounds()
    M = O.Model(A, B, Q, R, b[:, 0], b[:, 1], wl.T, wl.p, w=w)
    prob = _problem(wl, Q, R)
    prob.set_disturbance(w)
    x0, g = wl.start_goal()
    kd = torch.empty(wl.m * wl.p, device="cuda")
    cd = torch.empty(1, device="cuda")
    prob.solve_device(_dev(x0), _dev(g), 3, kd, cd)
    torch.cuda.synchronize()
    J = M.cost(np.float32(x0).astype(np.float64), np.float32(g).astype(np.float64),
               kd.cpu().numpy().astype(np.float64))
    assert abs(cd.item() - J) <= COST_RTOL * abs(J)
    prob.close()


def test_dense_q_rejects_state_box():
    import paper_2001_04931_gb300 as E
    wl, Q, R = dense_workload(dof=3, T=20, p=3, P=64)
    prob = _problem(wl, Q, R)
    with pytest.raises(E.EmpcError) as ei:
        prob.set_state_box(-np.ones(wl.n), np.ones(wl.n), clamp=True)
    assert ei.value.status == E.EMPC_EUNSUPPORTED
    prob.close()
    # a dense R alone keeps the state box (the states are not rotated)
    prob = _problem(wl, np.diag(np.diag(Q)), R)
    prob.set_state_box(-np.ones(wl.n), np.ones(wl.n), clamp=True)
    prob.close()


def test_dense_weights_closed_loop():
    """The receding-horizon loop's actual cost (Eq. actual_cost) with dense
    weights against the oracle's FP64 loop (the same draws, so the same
    plans up to the rounding of near-equal costs)."""
    wl, Q, R = dense_workload(dof=3, T=30, p=4, P=256, E=16)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    M = O.Model(A, B, Q, R, b[:, 0], b[:, 1], wl.T, wl.p)
    prob = _problem(wl, Q, R, seed=3)
    x0, g = wl.start_goal()
    r = prob.closed_loop(A, B, x0, g, 10, 2)
    ga = O.EMPC(M, wl.P, wl.E, seed=3, sigma=wl.sigma)
    _, uo, Jo, _ = O.closed_loop(ga, A, B, Q, R, x0, g, 10, 2)
    np.testing.assert_allclose(r["u"][0], uo[0], rtol=0, atol=1e-6)
    assert abs(r["actual_cost"] - Jo) <= 1e-3 * abs(Jo)
    prob.close()


def test_dense_weights_batched_bit_identical_to_single():
    """Batched problems with dense weights (one rotated, one not, one with a
    dense R only) give bit-identical results to single-problem solves, and
    their costs match the oracle."""
    import paper_2001_04931_gb300 as E
    wls = [dense_workload(dof=d, T=T, p=p, P=P, E=E_, seed=s)
           for d, T, p, P, E_, s in [(3, 30, 4, 192, 12, 0), (6, 50, 5, 256, 16, 1),
                                     (4, 25, 3, 160, 10, 2)]]
    probs = []
    for i, (wl, Q, R) in enumerate(wls):
        if i == 2:
            Q = np.diag(np.diag(Q))
        A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
        x0, g = wl.start_goal()
        probs.append(dict(A=A, B=B, Q=Q, R=R, bounds=wl.bounds(), x0=x0, x_goal=g,
                          horizon=wl.T, knots=wl.p, pop=wl.P, elite=wl.E, seed=11 + i,
                          sigma=wl.sigma))
    bt = E.Batch(probs)
    knots, costs = bt.solve(3)
    bt.close()
    for i, pr in enumerate(probs):
        single = E.Problem(pr["A"], pr["B"], pr["Q"], pr["R"], pr["bounds"], pr["horizon"],
                           pr["knots"], pr["pop"], seed=pr["seed"], elite=pr["elite"],
                           sigma=pr["sigma"], tile=1)  # the warp family, as the batch runs
        assert single.info().tile_kind == 1
        k1, c1 = single.solve(pr["x0"], pr["x_goal"], 3)
        single.close()
        np.testing.assert_array_equal(k1, knots[i])
        assert c1 == costs[i]
        wl = wls[i][0]
        Mo = _oracle(wl, pr["Q"], pr["R"])
        J = Mo.cost(pr["x0"], pr["x_goal"], knots[i].astype(np.float64))
        assert abs(costs[i] - J) <= COST_RTOL * abs(J)
