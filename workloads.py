"""Seeded synthetic EMPC workloads: plants, weights, bounds, start and goal.

This module only draws inputs.  It holds none of the method's arithmetic (no
discretization, rollout, cost, selection or breeding) and imports neither the
oracle nor the CUDA library, so both sides can take their inputs from here.

Plant: a chain of `dof` point masses on a line, each driven by its own
actuator, mass 0 tied to a wall.  Springs (stiffness U[1, 10]) with parallel
dampers (damping U[0.1, 1]) join every pair of masses whose indices differ by
at most `radius` (radius 1: nearest neighbours; radius 3: the dense stiffness
Laplacian of the 24- and 64-DoF chains); masses are U[0.5, 2].  The state is
[positions; velocities] (n = 2 dof), the input is the actuator forces
(m = dof):  A_c = [[0, I], [-M^-1 K, -M^-1 C]],  B_c = [[0], [M^-1]].
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Plant:
    Ac: np.ndarray
    Bc: np.ndarray
    masses: np.ndarray
    K: np.ndarray
    C: np.ndarray


def chain_plant(dof: int, seed: int, radius: int = 1) -> Plant:
    rng = np.random.default_rng(seed)
    masses = rng.uniform(0.5, 2.0, size=dof)
    K = np.zeros((dof, dof))
    C = np.zeros((dof, dof))

    def couple(M, i, j, v):
        M[i, i] += v
        M[j, j] += v
        M[i, j] -= v
        M[j, i] -= v

    # wall spring and damper on mass 0
    K[0, 0] += rng.uniform(1.0, 10.0)
    C[0, 0] += rng.uniform(0.1, 1.0)
    for i in range(dof):
        for j in range(i + 1, min(dof, i + radius + 1)):
            couple(K, i, j, rng.uniform(1.0, 10.0))
            couple(C, i, j, rng.uniform(0.1, 1.0))
    Minv = np.diag(1.0 / masses)
    n = 2 * dof
    Ac = np.zeros((n, n))
    Ac[:dof, dof:] = np.eye(dof)
    Ac[dof:, :dof] = -Minv @ K
    Ac[dof:, dof:] = -Minv @ C
    Bc = np.zeros((n, dof))
    Bc[dof:, :] = Minv
    return Plant(Ac, Bc, masses, K, C)


@dataclass
class Workload:
    """One EMPC problem: plant, discretization step, weights, sizes, seeds."""
    name: str
    dof: int
    radius: int
    dt: float
    T: int
    p: int
    P: int
    E: int
    G: int
    sigma: float
    q_pos: float
    q_vel: float
    r: float
    seed: int = 0
    umax: float = 1.0
    refine_steps: int = 0
    ckpt_every: int = 0
    plant: Plant = field(init=False, repr=False)

    def __post_init__(self):
        self.plant = chain_plant(self.dof, self.seed, self.radius)

    @property
    def n(self):
        return 2 * self.dof

    @property
    def m(self):
        return self.dof

    def Q(self):
        return np.diag(np.r_[np.full(self.dof, self.q_pos), np.full(self.dof, self.q_vel)])

    def R(self):
        return self.r * np.eye(self.m)

    def bounds(self):
        """[m, 2] array of (u_min, u_max)."""
        return np.tile([-self.umax, self.umax], (self.m, 1)).astype(np.float64)

    def start_goal(self, k: int = 0):
        """x0 and x_goal, both U[-1, 1] per state component (stream k)."""
        rng = np.random.default_rng([self.seed, 7919, k])
        return rng.uniform(-1, 1, self.n), rng.uniform(-1, 1, self.n)


def config(name: str, seed: int = 0) -> Workload:
    """The five workloads, by name:

    c1  2-DoF nearest-neighbour chain, dt 0.01, T 50, 4 knots, P 512, E 32,
        20 generations, sigma 0.1, Q = I, R = 1e-3 I.
    c2  24-DoF chain, springs within distance 3, dt 0.005, T 100, 5 knots,
        P 4096, E 128, 30 generations, Q = diag(10 pos, 1 vel), R = 1e-4 I.
    c3  c2 plus 5 projected-gradient refinement steps on the elites per
        generation, state checkpoints every 10 steps in the adjoint.
    c5  64-DoF chain, springs within distance 3, dt 0.005, T 200, 8 knots,
        P 16384, E 512, 40 generations, weights as c2.
    (The batched workload is `batched_problems`.)
    """
    if name == "c1":
        return Workload("c1", dof=2, radius=1, dt=0.01, T=50, p=4, P=512, E=32, G=20,
                        sigma=0.1, q_pos=1.0, q_vel=1.0, r=1e-3, seed=seed)
    if name == "c2":
        return Workload("c2", dof=24, radius=3, dt=0.005, T=100, p=5, P=4096, E=128, G=30,
                        sigma=0.1, q_pos=10.0, q_vel=1.0, r=1e-4, seed=seed)
    if name == "c3":
        return Workload("c3", dof=24, radius=3, dt=0.005, T=100, p=5, P=4096, E=128, G=30,
                        sigma=0.1, q_pos=10.0, q_vel=1.0, r=1e-4, seed=seed,
                        refine_steps=5, ckpt_every=10)
    if name == "c5":
        return Workload("c5", dof=64, radius=3, dt=0.005, T=200, p=8, P=16384, E=512, G=40,
                        sigma=0.1, q_pos=10.0, q_vel=1.0, r=1e-4, seed=seed)
    raise KeyError(name)


def small(name: str = "s1", seed: int = 0, **kw) -> Workload:
    """Small cases the oracle finishes in seconds (parity tests)."""
    base = dict(dof=3, radius=1, dt=0.01, T=23, p=4, P=200, E=16, G=3, sigma=0.1,
                q_pos=1.0, q_vel=0.5, r=1e-3, seed=seed)
    base.update(kw)
    return Workload(name, **base)


def batched_problems(count: int = 256, seed: int = 0):
    """The batched workload: `count` independent problems with DoF uniform on
    {2..32}, horizon on {20..200}, population on {256..4096} (multiples of 32),
    3-8 knots, each with its own plant, start and goal; nearest-neighbour
    chains, dt 0.01, Q = I, R = 1e-3 I, elite P/16, sigma 0.1, 20 generations.
    """
    rng = np.random.default_rng([seed, 4242])
    out = []
    for b in range(count):
        dof = int(rng.integers(2, 33))
        T = int(rng.integers(20, 201))
        P = int(rng.integers(8, 129)) * 32
        p = int(rng.integers(3, 9))
        wl = Workload(f"b{b}", dof=dof, radius=1, dt=0.01, T=T, p=p, P=P, E=P // 16,
                      G=20, sigma=0.1, q_pos=1.0, q_vel=1.0, r=1e-3,
                      seed=int(rng.integers(0, 2**31 - 1)))
        out.append(wl)
    return out
