"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/empc.h declares, validates arguments before
touching the device, and its own zero-order hold agrees with the oracle's."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(empc_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def E():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2001_04931_gb300 as mod
    return mod


def test_library_exports_every_declared_symbol(E):
    declared = _declared()
    assert {"empc_create", "empc_solve", "empc_destroy"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", E.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (empc_\w+)", out))
    assert declared <= exported, declared - exported
    for name in declared:
        assert hasattr(E, name)


def test_zoh_matches_oracle(E):
    for dof, radius, dt in [(2, 1, 0.01), (24, 3, 0.005), (64, 3, 0.005)]:
        plant = W.chain_plant(dof, seed=dof, radius=radius)
        Ad, Bd = E.discretize_zoh(plant.Ac, plant.Bc, dt)
        Ao, Bo = O.zoh(plant.Ac, plant.Bc, dt)
        np.testing.assert_allclose(Ad, Ao, rtol=0, atol=1e-13)
        np.testing.assert_allclose(Bd, Bo, rtol=0, atol=1e-15)


def test_zoh_rejects_bad_input(E):
    Ad, Bd = np.zeros((2, 2)), np.zeros((2, 1))
    p = lambda a: np.ascontiguousarray(a, np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    Ac = np.array([[0.0, np.nan], [0.0, 0.0]])
    assert E.empc_discretize_zoh(p(Ac), p(np.ones((2, 1))), 2, 1, 0.1, p(Ad), p(Bd)) == E.EMPC_EINVAL
    assert E.empc_discretize_zoh(None, p(np.ones((2, 1))), 2, 1, 0.1, p(Ad), p(Bd)) == E.EMPC_EINVAL
    assert E.empc_discretize_zoh(p(np.eye(2)), p(np.ones((2, 1))), 2, 1, -1.0, p(Ad), p(Bd)) == E.EMPC_EINVAL


@pytest.mark.parametrize("bad", [
    dict(knots=0), dict(knots=60), dict(horizon=0), dict(pop=0), dict(elite=600),
    # dense weights are taken, but their symmetric parts must be positive
    # semidefinite (eigenvalues 3 and -1 here)
    dict(Q=np.kron(np.eye(2), [[1.0, 2.0], [2.0, 1.0]])), dict(R=np.array([[1.0, 2.0], [2.0, 1.0]])),
    dict(Q=np.kron(np.eye(2), [[1.0, 4.0], [0.0, 1.0]])),
    dict(bounds=np.array([[1.0, -1.0], [-1.0, 1.0]])), dict(A=np.full((4, 4), np.inf)),
    dict(sigma=-1.0), dict(p_cross_256=300), dict(gate=7), dict(Q=-np.eye(4)),
    dict(evaluator=5), dict(evaluator=1, precision=1), dict(evaluator=1, refine_steps=2),
    dict(evaluator=1, A=np.eye(66), B=np.ones((66, 2)), Q=np.eye(66)),
])
def test_create_validates_before_touching_the_device(E, bad):
    base = dict(A=np.eye(4), B=np.ones((4, 2)), Q=np.eye(4), R=np.eye(2),
                bounds=np.tile([-1.0, 1.0], (2, 1)), horizon=50, knots=4, pop=512)
    cfg_keys = {"elite", "sigma", "p_cross_256", "gate", "evaluator", "precision", "refine_steps"}
    args = {**base, **{k: v for k, v in bad.items() if k not in cfg_keys}}
    cfg = E.default_config(**{k: v for k, v in bad.items() if k in cfg_keys})
    with pytest.raises(E.EmpcError) as ei:
        E.Problem(args["A"], args["B"], args["Q"], args["R"], args["bounds"], args["horizon"],
                  args["knots"], args["pop"], config=cfg)
    assert ei.value.status in (E.EMPC_EINVAL, E.EMPC_EUNSUPPORTED)


def test_null_handle_calls_fail_cleanly(E):
    assert E.empc_reset(None) == E.EMPC_EINVAL
    assert E.empc_solve(None, None, None, 1, None, None) == E.EMPC_EINVAL
    assert E.empc_set_state_box(None, None, None, None, E.EMPC_BOX_CLAMP) == E.EMPC_EINVAL
    assert E.empc_set_disturbance(None, None) == E.EMPC_EINVAL
    assert E.empc_inject_stall(None, 3, 0.1) == E.EMPC_EINVAL
    assert b"NULL" in E.empc_last_error(None)
    E.empc_destroy(None)


def test_default_config(E):
    c = E.default_config()
    assert c.sigma == pytest.approx(0.1) and c.p_cross_256 == 128 and c.p_mutate_256 == 128
    assert c.gate == E.EMPC_GATE_PER_INPUT and c.precision == E.EMPC_FP32
    assert c.evaluator == E.EMPC_EVAL_ROLLOUT


def test_batch_create_host_path_without_a_device(E):
    """empc_batch_create's host work (validation, tables, rotations, the work
    lists of every launch shape) runs before the first CUDA call: on a host
    without a GPU it must end in a clean EMPC_ECUDA, never a crash."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present; the GPU tests create batches")
    except ImportError:
        pass
    import workloads as W
    probs = []
    for wl in W.batched_problems(64, seed=3):
        A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
        x0, g = wl.start_goal()
        probs.append(dict(A=A, B=B, Q=wl.Q(), R=wl.R(), bounds=wl.bounds(), x0=x0, x_goal=g,
                          horizon=wl.T, knots=wl.p, pop=wl.P, elite=wl.E, seed=wl.seed,
                          sigma=wl.sigma))
    with pytest.raises(E.EmpcError) as ei:
        E.Batch(probs)
    assert ei.value.status == E.EMPC_ECUDA
