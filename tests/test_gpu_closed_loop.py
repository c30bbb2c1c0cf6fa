"""Receding-horizon driver (empc_closed_loop) against the FP64 oracle loop.

Both loops breed with the same counter-based draws, so until FP32 and FP64
costs order two candidates differently (a near tie) they apply the same
inputs.  The bars: the first applied input identical; the actual cost the
library reports equal (1e-12) to the one recomputed from its returned
trajectory; and the two actual costs within 1e-3 of each other."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from helpers import gpu_problem, oracle_model

pytestmark = pytest.mark.gpu


def test_closed_loop_matches_oracle_loop():
    wl = W.small(dof=2, T=20, p=3, P=200, E=12)
    x0 = np.zeros(wl.n)
    g = np.r_[np.full(wl.dof, 0.5), np.zeros(wl.dof)]
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    steps, G = 25, 2
    prob = gpu_problem(wl, seed=6)
    out = prob.closed_loop(A, B, x0, g, steps, G)
    ga = O.EMPC(oracle_model(wl), wl.P, wl.E, seed=6, sigma=wl.sigma)
    xs, us, J, _ = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, steps, G)
    np.testing.assert_array_equal(out["u"][0], us[0])
    # the library's bookkeeping, recomputed from its own trajectory
    Q, R = wl.Q(), wl.R()
    Jr = sum((g - x) @ Q @ (g - x) for x in out["x"]) + sum(u @ R @ u for u in out["u"])
    assert abs(out["actual_cost"] - Jr) <= 1e-12 * Jr
    np.testing.assert_allclose(out["x"][1:], out["x"][:-1] @ A.T + out["u"] @ B.T,
                               rtol=0, atol=1e-12)
    assert abs(out["actual_cost"] - J) <= 1e-3 * J
    assert out["ms_per_step"] > 0
    prob.close()


def test_closed_loop_distance_scaled_sigma_matches_oracle():
    wl = W.small(dof=2, T=20, p=3, P=200, E=12)
    x0 = np.zeros(wl.n)
    g = np.r_[np.full(wl.dof, 0.05), np.zeros(wl.dof)]
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    steps, G = 20, 2
    prob = gpu_problem(wl, seed=7)
    out = prob.closed_loop(A, B, x0, g, steps, G, sigma_min=0.005, sigma_dref=0.5)
    ga = O.EMPC(oracle_model(wl), wl.P, wl.E, seed=7, sigma=wl.sigma)
    xs, us, J, sig = O.closed_loop(ga, A, B, wl.Q(), wl.R(), x0, g, steps, G, sigma_min=0.005,
                                   sigma_dref=0.5)
    assert sig[0] < np.float32(wl.sigma)  # the schedule is active from the first step
    np.testing.assert_array_equal(out["u"][0], us[0])
    assert abs(out["actual_cost"] - J) <= 1e-3 * J
    prob.close()


def test_closed_loop_rejects_bad_arguments():
    import paper_2001_04931_gb300 as E
    wl = W.small(dof=2, T=10, p=2, P=64, E=4)
    A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    prob = gpu_problem(wl)
    with pytest.raises(E.EmpcError) as ei:
        prob.closed_loop(A, B, np.zeros(wl.n), np.zeros(wl.n), 0, 1)
    assert ei.value.status == E.EMPC_EINVAL
    with pytest.raises(E.EmpcError) as ei:
        prob.closed_loop(np.full_like(A, np.nan), B, np.zeros(wl.n), np.zeros(wl.n), 3, 1)
    assert ei.value.status == E.EMPC_EINVAL
    with pytest.raises(E.EmpcError) as ei:
        prob.closed_loop(A, B, np.zeros(wl.n), np.zeros(wl.n), 3, 1, sigma_dref=-1.0)
    assert ei.value.status == E.EMPC_EINVAL
    with pytest.raises(E.EmpcError) as ei:
        prob.set_sigma(-0.5)
    assert ei.value.status == E.EMPC_EINVAL
    prob.close()
