"""Shared test plumbing: build the same seeded problem for the oracle (its own
FP64 discretization) and for the CUDA library (the library's own ZOH)."""
import numpy as np

import oracle as O
import workloads as W


def oracle_model(wl: W.Workload, A=None, B=None):
    if A is None:
        A, B = O.zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    b = wl.bounds()
    return O.Model(A, B, wl.Q(), wl.R(), b[:, 0], b[:, 1], wl.T, wl.p)


def gpu_problem(wl: W.Workload, seed=1, A=None, B=None, **cfg):
    import paper_2001_04931_gb300 as E
    if A is None:
        A, B = E.discretize_zoh(wl.plant.Ac, wl.plant.Bc, wl.dt)
    return E.Problem(A, B, wl.Q(), wl.R(), wl.bounds(), wl.T, wl.p, wl.P, seed=seed,
                     elite=wl.E, sigma=wl.sigma, **cfg)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-30)


def check_elites(gpu_elite, orc_cost, E, rtol=2e-5):
    """The GPU's elite list must agree with the FP64 costs wherever they are
    separated by more than rtol: every candidate clearly below the E-th FP64
    cost is selected, none clearly above it is, and the ranks are ordered."""
    gpu_elite = np.asarray(gpu_elite)
    key = np.where(np.isnan(orc_cost), np.inf, orc_cost)
    order = np.lexsort((np.arange(key.size), key))
    tE = key[order[E - 1]]
    sel = set(gpu_elite.tolist())
    assert len(sel) == E
    below = np.nonzero(key < tE * (1 - rtol))[0]
    above = np.nonzero(key > tE * (1 + rtol))[0]
    assert set(below.tolist()) <= sel
    assert not (set(above.tolist()) & sel)
    c = key[gpu_elite]
    assert (c[1:] >= c[:-1] * (1 - rtol) - 1e-30).all()


def report(name, **values):
    """Append measured figures (errors, bounds) as one JSON line to the file
    named by EMPC_TEST_REPORT, when set; tests still assert their bars."""
    import json
    import os
    path = os.environ.get("EMPC_TEST_REPORT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"test": name, **{k: float(v) for k, v in values.items()}}) + "\n")
