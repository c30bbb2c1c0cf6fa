"""EMPC oracle: plain FP64 CPU reference of one evolutionary-MPC generation.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library and never imports it; the product path never imports this.

What it computes follows Hyatt, Williams & Killpack (arXiv 2001.04931):
  * model and discretization: Sec. III-A (Eq. first_order_integration),
  * cost: Eq. mpc_problem with u_goal = 0, stage cost after each update,
  * knot parameterization: Sec. IV-C,
  * condensed quadratic form: Sec. IV-B and IV-E (parameterized S),
  * the evolutionary loop: Algorithm 1 and Sec. V (cold start, mate, mutate,
    keep the numParents best).
The heavy loops live in empc_oracle.c (plain C, FP64, compiled by build.py);
this module marshals numpy arrays and runs Algorithm 1's generation loop.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_long)
_up = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox4x32_10.argtypes = [_up, _up, _up]
        L.orc_log_f32.argtypes = [ctypes.c_float]
        L.orc_log_f32.restype = ctypes.c_float
        L.orc_sincos_octant.argtypes = [ctypes.c_uint32, _fp, _fp]
        L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _fp, _fp]
        L.orc_breed_cold.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _fp, _fp,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp]
        L.orc_breed_warm.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _fp, _ip,
                                     ctypes.c_int, _fp, _fp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _fp]
        L.orc_knot_table.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _lp]
        L.orc_knot_table.restype = ctypes.c_long
        L.orc_expand.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_cost.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_cost.restype = ctypes.c_double
        L.orc_cost_population.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _fp,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_cost_box.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                   ctypes.c_int, _dp]
        L.orc_cost_box.restype = ctypes.c_double
        L.orc_cost_population_box.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _fp,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                              ctypes.c_int, _dp]
        L.orc_condensed.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                    _dp, _dp]
        L.orc_grad.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_grad.restype = ctypes.c_double
        L.orc_refine.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_double, _dp]
        L.orc_select.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _ip]
        L.orc_expm.argtypes = [_dp, ctypes.c_int, _dp]
        L.orc_zoh.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              _dp, _dp]
        L.orc_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t):
    return a.ctypes.data_as(t)


def _opt(a):
    if a is None:
        return None, None
    a = _d(a)
    return a, _ptr(a, _dp)


# --------------------------------------------------------------------------
# Random draws (Philox4x32-10 and the Gaussian transform)
# --------------------------------------------------------------------------
def philox4x32_10(counter, key):
    """Philox4x32-10 block: four uint32 counter words, two uint32 key words."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _up), _ptr(k, _up), _ptr(out, _up))
    return out


def log_f32(u):
    return float(lib().orc_log_f32(ctypes.c_float(u)))


def sincos_2pi(r24):
    s = ctypes.c_float()
    c = ctypes.c_float()
    lib().orc_sincos_octant(ctypes.c_uint32(r24), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def box_muller(ra, rb):
    z0 = ctypes.c_float()
    z1 = ctypes.c_float()
    lib().orc_box_muller(ctypes.c_uint32(ra), ctypes.c_uint32(rb), ctypes.byref(z0),
                         ctypes.byref(z1))
    return z0.value, z1.value


# --------------------------------------------------------------------------
# Parameterization, rollout, cost
# --------------------------------------------------------------------------
def knot_table(T, p):
    """(idx1[T], num[T], den): u_k = (1 - num/den) U_idx1 + (num/den) U_idx1+1."""
    idx1 = np.zeros(T, dtype=np.int32)
    num = np.zeros(T, dtype=np.int64 if ctypes.sizeof(ctypes.c_long) == 8 else np.int32)
    den = lib().orc_knot_table(T, p, _ptr(idx1, _ip), _ptr(num, _lp))
    return idx1, num, int(den)


def expand(U, m, T, p):
    """Per-step inputs u[T, m] from knots U[m*p] (parameter q = i*p + j)."""
    U = _d(U)
    out = np.zeros((T, m))
    lib().orc_expand(_ptr(U, _dp), m, T, p, _ptr(out, _dp))
    return out


class StateBox:
    """The state-box hook (Sec. V: with every state of every step simulated,
    effects such as hard stops and non-convex state costs go into the
    simulation as plain if/else).  Per state i: bounds lo_i <= hi_i and weight
    rho_i >= 0.  After each update, d_i = max(0, lo_i - x_i, x_i - hi_i);
    `penalty` adds rho_i d_i^2 to the cost, `clamp` stops the state at the
    box.  Both act before the stage cost, which sees the stopped state."""

    def __init__(self, lo, hi, rho=None, clamp=False, penalty=False):
        self.lo = _d(lo)
        self.hi = _d(hi)
        self.rho = np.zeros_like(self.lo) if rho is None else _d(rho)
        self.mode = (1 if clamp else 0) | (2 if penalty else 0)

    def _args(self):
        return _ptr(self.lo, _dp), _ptr(self.hi, _dp), _ptr(self.rho, _dp), self.mode

    def stop(self, x):
        """The hard stop applied to a plant state (identity without clamp)."""
        return np.minimum(np.maximum(x, self.lo), self.hi) if self.mode & 1 else x


class Model:
    """Discrete model and cost weights, all FP64 (row-major)."""

    def __init__(self, A, B, Q, R, umin, umax, T, p, w=None):
        self.A = _d(A)
        self.B = _d(B)
        self.Q = _d(Q)
        self.R = _d(R)
        self.n = self.A.shape[0]
        self.m = self.B.shape[1]
        self.umin = _d(umin)
        self.umax = _d(umax)
        self.T = int(T)
        self.p = int(p)
        self.w, self._wp = _opt(w)

    def _mats(self):
        return (_ptr(self.A, _dp), _ptr(self.B, _dp), _ptr(self.Q, _dp),
                _ptr(self.R, _dp), self._wp)

    def cost(self, x0, g, U, conv=0, return_traj=False, box=None):
        """J(U) (and x_0..x_T); with a StateBox, the hooked simulation
        (conv 0 only)."""
        x0, g, U = _d(x0), _d(g), _d(U)
        traj = np.zeros((self.T + 1, self.n)) if return_traj else None
        tp = _ptr(traj, _dp) if return_traj else None
        if box is None:
            J = lib().orc_cost(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp), _ptr(U, _dp),
                               self.n, self.m, self.T, self.p, conv, tp)
        else:
            if conv != 0:
                raise ValueError("the state-box hook follows cost convention 0")
            J = lib().orc_cost_box(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp),
                                   _ptr(U, _dp), self.n, self.m, self.T, self.p,
                                   *box._args(), tp)
        return (J, traj) if return_traj else J

    def cost_population(self, x0, g, pop, conv=0, box=None):
        """FP64 costs of an SoA FP32 population pop[m*p, P]."""
        x0, g = _d(x0), _d(g)
        pop = np.ascontiguousarray(pop, dtype=np.float32)
        P = pop.shape[1]
        out = np.zeros(P)
        if box is None:
            lib().orc_cost_population(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp),
                                      _ptr(pop, _fp), self.n, self.m, self.T, self.p, P,
                                      conv, _ptr(out, _dp))
        else:
            if conv != 0:
                raise ValueError("the state-box hook follows cost convention 0")
            lib().orc_cost_population_box(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp),
                                          _ptr(pop, _fp), self.n, self.m, self.T, self.p,
                                          P, *box._args(), _ptr(out, _dp))
        return out

    def condensed(self, x0, g, return_S=False):
        """(H, f, c0[, S]) with J(U) = U'HU + 2f'U + c0."""
        x0, g = _d(x0), _d(g)
        D = self.m * self.p
        H = np.zeros((D, D))
        f = np.zeros(D)
        c0 = ctypes.c_double()
        S = np.zeros((self.T * self.n, D)) if return_S else None
        lib().orc_condensed(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp), self.n, self.m,
                            self.T, self.p, _ptr(S, _dp) if return_S else None,
                            _ptr(H, _dp), _ptr(f, _dp), ctypes.byref(c0))
        if return_S:
            return H, f, c0.value, S
        return H, f, c0.value

    def grad(self, x0, g, U):
        """(J, dJ/dU) by the FP64 adjoint recursion."""
        x0, g, U = _d(x0), _d(g), _d(U)
        gr = np.zeros(self.m * self.p)
        J = lib().orc_grad(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp), _ptr(U, _dp),
                           self.n, self.m, self.T, self.p, _ptr(gr, _dp))
        return J, gr

    def refine(self, x0, g, U, steps, eta):
        """Projected gradient: `steps` times U <- clip(U - eta dJ/dU), FP64."""
        x0, g = _d(x0), _d(g)
        U = _d(U).copy()
        lib().orc_refine(*self._mats(), _ptr(x0, _dp), _ptr(g, _dp),
                         _ptr(self.umin, _dp), _ptr(self.umax, _dp), self.n, self.m,
                         self.T, self.p, int(steps), float(eta), _ptr(U, _dp))
        return U

    def lipschitz_step(self, x0=None, g=None):
        """eta = 1/L with L = 2 lambda_max(H), the gradient's Lipschitz constant."""
        x0 = np.zeros(self.n) if x0 is None else x0
        g = np.zeros(self.n) if g is None else g
        H, _, _ = self.condensed(x0, g)
        return 1.0 / (2.0 * float(np.linalg.eigvalsh(0.5 * (H + H.T))[-1]))


# --------------------------------------------------------------------------
# Selection and breeding
# --------------------------------------------------------------------------
def select(cost, E):
    """Indices of the E lowest costs, ordered by (cost, index); NaN = +inf."""
    cost = _d(cost)
    out = np.zeros(E, dtype=np.int32)
    lib().orc_select(_ptr(cost, _dp), cost.shape[0], E, _ptr(out, _ip))
    return out


def breed_cold(seed, gen, umin, umax, m, p, P):
    umin = np.ascontiguousarray(umin, dtype=np.float32)
    umax = np.ascontiguousarray(umax, dtype=np.float32)
    pop = np.zeros((m * p, P), dtype=np.float32)
    lib().orc_breed_cold(seed, gen, _ptr(umin, _fp), _ptr(umax, _fp), m, p, P,
                         _ptr(pop, _fp))
    return pop


def breed_warm(seed, gen, old_pop, elite_idx, umin, umax, m, p, sigma, pc256=128,
               pm256=128, gate_mode=0):
    old_pop = np.ascontiguousarray(old_pop, dtype=np.float32)
    elite_idx = np.ascontiguousarray(elite_idx, dtype=np.int32)
    umin = np.ascontiguousarray(umin, dtype=np.float32)
    umax = np.ascontiguousarray(umax, dtype=np.float32)
    P = old_pop.shape[1]
    new = np.zeros_like(old_pop)
    lib().orc_breed_warm(seed, gen, _ptr(old_pop, _fp), _ptr(elite_idx, _ip),
                         elite_idx.shape[0], _ptr(umin, _fp), _ptr(umax, _fp), m, p, P,
                         float(sigma), int(pc256), int(pm256), int(gate_mode),
                         _ptr(new, _fp))
    return new


# --------------------------------------------------------------------------
# Discretization
# --------------------------------------------------------------------------
def expm(M):
    M = _d(M)
    out = np.zeros_like(M)
    lib().orc_expm(_ptr(M, _dp), M.shape[0], _ptr(out, _dp))
    return out


def zoh(Ac, Bc, dt):
    Ac, Bc = _d(Ac), _d(Bc)
    n, m = Bc.shape
    Ad = np.zeros((n, n))
    Bd = np.zeros((n, m))
    lib().orc_zoh(_ptr(Ac, _dp), _ptr(Bc, _dp), n, m, float(dt), _ptr(Ad, _dp),
                  _ptr(Bd, _dp))
    return Ad, Bd


def num_threads():
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# Algorithm 1: the generation loop
# --------------------------------------------------------------------------
class EMPC:
    """Algorithm 1 in FP64: cold start, then per generation mate + mutate from
    the elites, simulate every candidate, keep the E best (elitism, Sec. V).

    Mirrors the library's call semantics: the population persists between
    solve() calls (warm start); generation numbers count up across calls and
    key the random draws; reset() makes the next generation a cold start.
    With refine_steps > 0 the elites are refined between generations: the
    children are bred from the elites as selected, and slot e of the new
    population holds elite e after `refine_steps` projected-gradient steps
    (instead of the unchanged copy).
    """

    def __init__(self, model, P, E, seed, sigma, pc256=128, pm256=128, gate_mode=0,
                 refine_steps=0, refine_eta=0.0, box=None):
        self.model = model
        self.box = box
        self.P, self.E = int(P), int(E)
        self.seed = int(seed)
        self.sigma = float(sigma)
        self.pc256, self.pm256, self.gate_mode = pc256, pm256, gate_mode
        self.refine_steps = int(refine_steps)
        self.refine_eta = float(refine_eta)
        self.umin32 = model.umin.astype(np.float32)
        self.umax32 = model.umax.astype(np.float32)
        self.gen = 0
        self.pop = None
        self.cost = None
        self.elite = None

    def reset(self):
        self.pop = None

    def refined_elites(self, x0, g, pop=None, elite=None):
        """[m*p, E] float64: each elite after refine_steps projected steps."""
        pop = self.pop if pop is None else pop
        elite = self.elite if elite is None else elite
        M = self.model
        out = np.zeros((pop.shape[0], len(elite)))
        for r, e in enumerate(elite):
            out[:, r] = M.refine(x0, g, pop[:, e].astype(np.float64), self.refine_steps,
                                 self.refine_eta)
        return out

    def generation(self, x0, g):
        M = self.model
        if self.pop is None:
            pop = breed_cold(self.seed, self.gen, self.umin32, self.umax32, M.m, M.p,
                             self.P)
        else:
            pop = breed_warm(self.seed, self.gen, self.pop, self.elite, self.umin32,
                             self.umax32, M.m, M.p, self.sigma, self.pc256, self.pm256,
                             self.gate_mode)
            if self.refine_steps > 0:
                pop[:, :self.E] = self.refined_elites(x0, g).astype(np.float32)
        self.gen += 1
        self.pop = pop
        self.cost = M.cost_population(x0, g, pop, box=self.box)
        self.elite = select(self.cost, self.E)

    def solve(self, x0, g, generations):
        for _ in range(int(generations)):
            self.generation(x0, g)
        best = int(self.elite[0])
        return self.pop[:, best].copy(), float(self.cost[best])


def closed_loop(ga, Ad, Bd, Q, R, x0, goal, steps, generations, sigma_min=0.0, sigma_dref=0.0):
    """Receding-horizon control in FP64 (Sec. III-A: solve, apply only the
    first input, solve again from the state reached; Sec. V: the best input
    after each solve of `generations` generations).  u_k is the first knot of
    each input of the best candidate; the plant x_{k+1} = Ad x_k + Bd u_k runs
    in FP64.  With sigma_dref > 0 the mutation sigma depends on the distance
    to the goal (Sec. VII): sigma_k = max(sigma_min, sigma0 min(1, |x_k - g| /
    sigma_dref)) with sigma0 the EMPC object's (FP32) sigma and the norm
    summed in index order, rounded to FP32.  Actual cost (Eq. actual_cost):
    the stage costs (goal - x_k)' Q (goal - x_k) + u_k' R u_k over the applied
    steps plus the state term of the final state.  The model's constant
    disturbance w_d (Eq. first_order_integration), if it has one, acts on the
    plant too: x_{k+1} = Ad x_k + Bd u_k + w_d.  With the EMPC object's
    StateBox set to clamp, the plant is stopped at the same box after every
    step.  Returns (x [(steps+1), n], u [steps, m], actual cost, sigmas
    [steps])."""
    Ad, Bd, Q, R = _d(Ad), _d(Bd), _d(Q), _d(R)
    x = _d(x0).copy()
    goal = _d(goal)
    p = ga.model.p
    sigma0 = float(np.float32(ga.sigma))
    xs, us, sig, total = [x.copy()], [], [], 0.0
    for _ in range(int(steps)):
        if sigma_dref > 0.0:
            d2 = 0.0
            for v in (x - goal):
                d2 += float(v) * float(v)
            ga.sigma = float(np.float32(max(sigma_min, sigma0 * min(1.0, np.sqrt(d2) / sigma_dref))))
        sig.append(ga.sigma)
        knots, _ = ga.solve(x, goal, generations)
        u = np.asarray(knots, np.float64)[::p].copy()
        e = goal - x
        total += e @ Q @ e + u @ R @ u
        x = Ad @ x + Bd @ u
        if ga.model.w is not None:
            x = x + ga.model.w
        if ga.box is not None:
            x = ga.box.stop(x)
        xs.append(x.copy())
        us.append(u)
    ga.sigma = sigma0
    e = goal - x
    total += e @ Q @ e
    return np.array(xs), np.array(us), float(total), np.array(sig)
