"""Python binding of the EMPC C-ABI library (libempc.so, include/empc.h).

Argument marshalling only: every step of an EMPC generation (breeding, knot
expansion, rollout, cost, elite selection) runs in the library's CUDA
kernels.  The raw entry points carry the C names (empc_create, empc_solve,
...); `Problem` wraps a handle for numpy / torch callers.  PyTorch is used
only to own device memory and streams.

Importing this module raises if the compiled library is missing: there is no
CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libempc.so")

EMPC_OK, EMPC_EINVAL, EMPC_ENOMEM, EMPC_ECUDA, EMPC_ETIMEOUT = 0, 1, 2, 3, 4
EMPC_ENONFINITE, EMPC_ESTATE, EMPC_EUNSUPPORTED = 5, 6, 7
EMPC_FP32, EMPC_BF16 = 0, 1
EMPC_GATE_PER_INPUT, EMPC_GATE_PER_KNOT, EMPC_GATE_ALWAYS = 0, 1, 2
EMPC_EVAL_ROLLOUT, EMPC_EVAL_CONDENSED = 0, 1
EMPC_BOX_CLAMP, EMPC_BOX_PENALTY = 1, 2

_STATUS = {0: "EMPC_OK", 1: "EMPC_EINVAL", 2: "EMPC_ENOMEM", 3: "EMPC_ECUDA",
           4: "EMPC_ETIMEOUT", 5: "EMPC_ENONFINITE", 6: "EMPC_ESTATE",
           7: "EMPC_EUNSUPPORTED"}


class empc_config(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("elite", ctypes.c_int), ("sigma", ctypes.c_float),
                ("p_cross_256", ctypes.c_int), ("p_mutate_256", ctypes.c_int),
                ("gate", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("refine_lr", ctypes.c_float),
                ("ckpt_every", ctypes.c_int), ("tile", ctypes.c_int),
                ("evaluator", ctypes.c_int)]


class empc_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("horizon", ctypes.c_int),
                ("knots", ctypes.c_int), ("pop", ctypes.c_int), ("elite", ctypes.c_int),
                ("generation", ctypes.c_uint64), ("tile_nx", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("tile_cands", ctypes.c_int),
                ("tile_groups", ctypes.c_int), ("threads_per_cta", ctypes.c_int),
                ("smem_bytes", ctypes.c_int), ("ctas", ctypes.c_int),
                ("tuned_us", ctypes.c_float), ("refine_lr", ctypes.c_float),
                ("tile_kind", ctypes.c_int), ("ckpt_every", ctypes.c_int)]


class empc_problem_desc(ctypes.Structure):
    _fields_ = [("A", ctypes.POINTER(ctypes.c_double)), ("B", ctypes.POINTER(ctypes.c_double)),
                ("Q", ctypes.POINTER(ctypes.c_double)), ("R", ctypes.POINTER(ctypes.c_double)),
                ("bounds", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.POINTER(ctypes.c_double)),
                ("x_goal", ctypes.POINTER(ctypes.c_double)), ("n", ctypes.c_int),
                ("m", ctypes.c_int), ("horizon", ctypes.c_int), ("knots", ctypes.c_int),
                ("pop", ctypes.c_int), ("elite", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("sigma", ctypes.c_float)]


class empc_batch_info(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("total_knots", ctypes.c_int), ("ctas", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("cands_per_lane", ctypes.c_int),
                ("items_per_generation", ctypes.c_int),
                ("state_steps_per_generation", ctypes.c_double), ("tuned_us", ctypes.c_float),
                ("h2d_bytes_targets", ctypes.c_int), ("d2h_bytes_solve", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p
_h = ctypes.c_void_p
_i = ctypes.c_int

# name -> (restype, argtypes); the C declarations are in include/empc.h
_SIGNATURES = {
    "empc_config_default": (None, [ctypes.POINTER(empc_config)]),
    "empc_create": (_i, [_dp, _dp, _dp, _dp, _dp, _i, _i, _i, _i, _i,
                         ctypes.POINTER(empc_config), ctypes.POINTER(_h)]),
    "empc_solve": (_i, [_h, _dp, _dp, _i, _fp, _fp]),
    "empc_solve_device": (_i, [_h, _vp, _vp, _i, _vp, _vp]),
    "empc_evaluate": (_i, [_h, _vp, _vp, _vp, _i, _vp]),
    "empc_grad": (_i, [_h, _vp, _vp, _vp, _i, _vp, _vp]),
    "empc_get_state": (_i, [_h, _vp, _vp, _vp]),
    "empc_set_state": (_i, [_h, _vp, _vp, _vp]),
    "empc_reset": (_i, [_h]),
    "empc_set_stream": (_i, [_h, _vp]),
    "empc_get_info": (_i, [_h, ctypes.POINTER(empc_info)]),
    "empc_destroy": (None, [_h]),
    "empc_last_error": (ctypes.c_char_p, [_h]),
    "empc_discretize_zoh": (_i, [_dp, _dp, _i, _i, ctypes.c_double, _dp, _dp]),
    "empc_time_generation": (_i, [_h, _i, _fp, _fp, _fp]),
    "empc_closed_loop": (_i, [_h, _dp, _dp, _dp, _dp, _i, _i, ctypes.c_double, ctypes.c_double,
                              _dp, _dp, _dp, _dp]),
    "empc_set_sigma": (_i, [_h, ctypes.c_float]),
    "empc_set_state_box": (_i, [_h, _fp, _fp, _fp, _i]),
    "empc_set_disturbance": (_i, [_h, _dp]),
    "empc_measure_fp32_peak": (_i, [_dp]),
    "empc_evaluate_noalloc": (_i, [_dp, _dp, _dp, _dp, _i, _i, _i, _i, _vp, _vp, _vp, _i,
                                  _vp, _vp]),
    "empc_batch_create": (_i, [ctypes.POINTER(empc_problem_desc), _i,
                               ctypes.POINTER(empc_config), ctypes.POINTER(_h)]),
    "empc_batch_solve": (_i, [_h, _i, _fp, _fp]),
    "empc_batch_reset": (_i, [_h]),
    "empc_batch_set_targets": (_i, [_h, _dp, _dp]),
    "empc_batch_solve_device": (_i, [_h, _i]),
    "empc_batch_set_stream": (_i, [_h, _vp]),
    "empc_batch_get_state": (_i, [_h, _i, _vp, _vp, _vp]),
    "empc_batch_get_info": (_i, [_h, ctypes.POINTER(empc_batch_info)]),
    "empc_batch_inject_stall": (_i, [_h, _i, ctypes.c_double]),
    "empc_inject_stall": (_i, [_h, _i, ctypes.c_double]),
    "empc_batch_destroy": (None, [_h]),
    "empc_batch_last_error": (ctypes.c_char_p, [_h]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2001_04931_gb300/build.py` "
            "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


_lib = _load()
globals().update({name: getattr(_lib, name) for name in _SIGNATURES})


class EmpcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status, handle=None):
    if status != EMPC_OK:
        msg = _lib.empc_last_error(handle)
        raise EmpcError(status, msg.decode() if msg else "")
    return status


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _dev(t):
    """Device pointer of a CUDA tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def default_config(**kw):
    cfg = empc_config()
    _lib.empc_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def discretize_zoh(Ac, Bc, dt):
    """Zero-order-hold (Ad, Bd) of x' = Ac x + Bc u over dt (host, FP64)."""
    Ac, Bc = _d(Ac), _d(Bc)
    n, m = Bc.shape
    Ad, Bd = np.zeros((n, n)), np.zeros((n, m))
    check(_lib.empc_discretize_zoh(_ptr(Ac), _ptr(Bc), n, m, float(dt), _ptr(Ad), _ptr(Bd)))
    return Ad, Bd


def _noalloc_tensor(name, t, shape):
    """A contiguous float32 CUDA tensor of `shape` on the current device, or
    EmpcError(EMPC_EINVAL): the C side trusts these sizes."""
    import torch
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and
          t.is_contiguous() and tuple(t.shape) == tuple(shape) and
          t.device.index == torch.cuda.current_device())
    if not ok:
        raise EmpcError(EMPC_EINVAL, f"{name} must be a contiguous float32 CUDA tensor of shape "
                                     f"{tuple(shape)} on the current device")


def evaluate_noalloc(A, B, Q, R, horizon, knots, x0, x_goal, pop, cost, stream=None):
    """Population costs for callers that must not allocate memory while they
    run (empc_evaluate_noalloc in include/empc.h: the tables live in a fixed
    device array).  A [n, n], B [n, m], Q [n, n], R [m, m] are host arrays;
    x0 and x_goal [n], pop [m*knots, count] and cost [count] are contiguous
    float32 CUDA tensors on the current device; asynchronous on `stream` (a
    cudaStream_t as an int, or None for the legacy default stream).  Every
    shape is checked here (EmpcError EMPC_EINVAL) before the C call."""
    A, B, Q, R = _d(A), _d(B), _d(Q), _d(R)
    if B.ndim != 2:
        raise EmpcError(EMPC_EINVAL, "B must be [n, m]")
    n, m = B.shape
    for name, M, k in (("A", A, n), ("Q", Q, n), ("R", R, m)):
        if M.shape != (k, k):
            raise EmpcError(EMPC_EINVAL, f"{name} must be [{k}, {k}]")
    horizon, knots = int(horizon), int(knots)
    if knots < 1:
        raise EmpcError(EMPC_EINVAL, "knots must be >= 1")
    _noalloc_tensor("x0", x0, (n,))
    _noalloc_tensor("x_goal", x_goal, (n,))
    if getattr(pop, "ndim", 0) != 2:
        raise EmpcError(EMPC_EINVAL, "pop must be [m*knots, count]")
    count = int(pop.shape[1])
    _noalloc_tensor("pop", pop, (m * knots, count))
    _noalloc_tensor("cost", cost, (count,))
    check(_lib.empc_evaluate_noalloc(_ptr(A), _ptr(B), _ptr(Q), _ptr(R), n, m, horizon, knots,
                                     _dev(x0), _dev(x_goal), _dev(pop), count, _dev(cost),
                                     stream))


def measure_fp32_peak():
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    v = ctypes.c_double()
    check(_lib.empc_measure_fp32_peak(ctypes.byref(v)))
    return v.value


class Problem:
    """One EMPC problem on the current CUDA device (owns an empc_handle)."""

    def __init__(self, A, B, Q, R, bounds, horizon, knots, pop, config=None, **cfg):
        A, B, Q, R, bounds = _d(A), _d(B), _d(Q), _d(R), _d(bounds)
        self.n, self.m = B.shape
        self.T, self.p, self.P = int(horizon), int(knots), int(pop)
        self.D = self.m * self.p
        c = config if config is not None else default_config(**cfg)
        h = _h()
        check(_lib.empc_create(_ptr(A), _ptr(B), _ptr(Q), _ptr(R), _ptr(bounds), self.n,
                               self.m, self.T, self.p, self.P, ctypes.byref(c),
                               ctypes.byref(h)))
        self.handle = h
        self.E = self.info().elite

    def close(self):
        if getattr(self, "handle", None):
            _lib.empc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = empc_info()
        check(_lib.empc_get_info(self.handle, ctypes.byref(inf)), self.handle)
        return inf

    def solve(self, x0, x_goal, generations):
        """Host in, host out: (best_knots[m*p] float32, best_cost float)."""
        x0, g = _d(x0), _d(x_goal)
        out = np.zeros(self.D, np.float32)
        cost = ctypes.c_float()
        check(_lib.empc_solve(self.handle, _ptr(x0), _ptr(g), int(generations),
                              out.ctypes.data_as(_fp), ctypes.byref(cost)), self.handle)
        return out, cost.value

    def solve_device(self, x0, x_goal, generations, best_knots, best_cost):
        check(_lib.empc_solve_device(self.handle, _dev(x0), _dev(x_goal), int(generations),
                                     _dev(best_knots), _dev(best_cost)), self.handle)

    def evaluate(self, x0, x_goal, pop, cost):
        """Costs of pop [m*p, count] (CUDA tensors) into cost [count]."""
        check(_lib.empc_evaluate(self.handle, _dev(x0), _dev(x_goal), _dev(pop),
                                 int(pop.shape[1]), _dev(cost)), self.handle)

    def grad(self, x0, x_goal, pop, grad=None, cost=None):
        """Adjoint dJ/dU of pop [m*p, count] into grad (same shape) and cost."""
        check(_lib.empc_grad(self.handle, _dev(x0), _dev(x_goal), _dev(pop), int(pop.shape[1]),
                             _dev(grad), _dev(cost)), self.handle)

    def get_state(self, pop=None, cost=None, elite=None):
        check(_lib.empc_get_state(self.handle, _dev(pop), _dev(cost), _dev(elite)),
              self.handle)

    def set_state(self, pop, cost, elite):
        check(_lib.empc_set_state(self.handle, _dev(pop), _dev(cost), _dev(elite)),
              self.handle)

    def reset(self):
        check(_lib.empc_reset(self.handle), self.handle)

    def set_sigma(self, sigma):
        check(_lib.empc_set_sigma(self.handle, float(sigma)), self.handle)

    def set_disturbance(self, w_d=None):
        """The constant disturbance w_d [n] of x_{k+1} = A_d x_k + B_d u_k +
        w_d (None or zeros: none)."""
        if w_d is None:
            check(_lib.empc_set_disturbance(self.handle, None), self.handle)
            return
        w = _d(w_d)
        if w.shape != (self.n,):
            raise ValueError(f"w_d needs shape ({self.n},)")
        check(_lib.empc_set_disturbance(self.handle, _ptr(w)), self.handle)

    def set_state_box(self, lo=None, hi=None, rho=None, clamp=False, penalty=False):
        """The state-box hook inside every rollout: per-state bounds lo, hi
        and weight rho (None: -inf, +inf, 0); `penalty` adds rho d^2 for the
        distance d outside the box after each update, `clamp` stops the state
        at the box.  Both False turn the hook off."""
        flags = (EMPC_BOX_CLAMP if clamp else 0) | (EMPC_BOX_PENALTY if penalty else 0)
        arrs = [None if v is None else np.ascontiguousarray(v, dtype=np.float32)
                for v in (lo, hi, rho)]
        for v in arrs:
            if v is not None and v.shape != (self.n,):
                raise ValueError(f"state box arrays need shape ({self.n},)")
        ptrs = [None if v is None else v.ctypes.data_as(_fp) for v in arrs]
        check(_lib.empc_set_state_box(self.handle, *ptrs, flags), self.handle)

    def closed_loop(self, Ad, Bd, x0, x_goal, steps, generations, sigma_min=0.0,
                    sigma_dref=0.0):
        """Receding-horizon control of the plant (Ad, Bd) for `steps` steps of
        `generations` generations each (sigma_dref > 0: mutation sigma scaled
        by the distance to the goal, at least sigma_min): dict(x [(steps+1), n],
        u [steps, m], actual_cost, ms_per_step)."""
        Ad, Bd = _d(Ad), _d(Bd)
        x0, g = _d(x0), _d(x_goal)
        xt = np.zeros((int(steps) + 1, self.n))
        ut = np.zeros((int(steps), self.m))
        cost, ms = ctypes.c_double(), ctypes.c_double()
        check(_lib.empc_closed_loop(self.handle, _ptr(Ad), _ptr(Bd), _ptr(x0), _ptr(g),
                                    int(steps), int(generations), float(sigma_min),
                                    float(sigma_dref), _ptr(xt), _ptr(ut), ctypes.byref(cost),
                                    ctypes.byref(ms)), self.handle)
        return {"x": xt, "u": ut, "actual_cost": cost.value, "ms_per_step": ms.value}

    def time_generation(self, reps):
        """Average (breed_us, rollout_us, select_us) of `reps` warm generations."""
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        check(_lib.empc_time_generation(self.handle, int(reps), ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)), self.handle)
        return a.value, b.value, c.value

    def set_stream(self, stream):
        check(_lib.empc_set_stream(self.handle, stream), self.handle)

    def inject_stall(self, step, timeout_s):
        """Test hook (BF16 handles): the tensor-core rollout's MMA issuer stops
        at horizon step `step` (-1: never); its waits run out after timeout_s."""
        check(_lib.empc_inject_stall(self.handle, int(step), float(timeout_s)), self.handle)


_COST_FN = None


def _cost_function():
    """The torch.autograd.Function behind rollout_cost (built on first use so
    that importing this module does not import torch)."""
    global _COST_FN
    if _COST_FN is None:
        import torch

        class RolloutCost(torch.autograd.Function):
            @staticmethod
            def forward(ctx, pop, x0, x_goal, problem):
                cost = torch.empty(pop.shape[1], device=pop.device, dtype=torch.float32)
                if ctx.needs_input_grad[0]:
                    grad = torch.empty_like(pop)
                    problem.grad(x0, x_goal, pop, grad, cost)  # costs and dJ/dU, one launch
                    ctx.save_for_backward(grad)
                else:
                    problem.evaluate(x0, x_goal, pop, cost)
                return cost

            @staticmethod
            def backward(ctx, grad_cost):
                (grad,) = ctx.saved_tensors
                return grad * grad_cost.unsqueeze(0), None, None, None

        _COST_FN = RolloutCost
    return _COST_FN


def rollout_cost(problem, x0, x_goal, pop):
    """Differentiable population cost: J [count] (FP32) of the knot vectors
    pop [m*p, count] (contiguous CUDA float32, SoA like the population) from
    x0 and x_goal (CUDA float32 [n]).  When pop requires grad, the forward
    pass runs empc_grad, which returns the costs and the adjoint dJ/dU in one
    launch, and the backward pass scales dJ/dU by the incoming gradient of J;
    otherwise it runs empc_evaluate.  The library works on torch's current
    stream (set_stream), so the results are ordered like any torch op."""
    import torch
    problem.set_stream(torch.cuda.current_stream().cuda_stream)
    return _cost_function().apply(pop, x0, x_goal, problem)


def _bcheck(status, batch):
    if status != EMPC_OK:
        msg = _lib.empc_batch_last_error(batch)
        raise EmpcError(status, msg.decode() if msg else "")


class Batch:
    """Many independent problems solved in one persistent launch (empc_batch_*).

    `problems` is a list of dicts with keys A, B, Q, R, bounds, x0, x_goal,
    horizon, knots, pop and optionally elite, seed, sigma."""

    def __init__(self, problems, config=None, **cfg):
        self._keep = []
        descs = (empc_problem_desc * len(problems))()
        self.dims = []
        for d, pr in zip(descs, problems):
            arrs = {k: _d(pr[k]) for k in ("A", "B", "Q", "R", "bounds", "x0", "x_goal")}
            self._keep.append(arrs)
            for k, v in arrs.items():
                setattr(d, k, _ptr(v))
            n, m = arrs["B"].shape
            d.n, d.m = n, m
            d.horizon, d.knots, d.pop = int(pr["horizon"]), int(pr["knots"]), int(pr["pop"])
            d.elite = int(pr.get("elite", 0))
            d.seed = int(pr.get("seed", 0))
            d.sigma = float(pr.get("sigma", 0.0))
            self.dims.append((n, m, d.horizon, d.knots, d.pop))
        c = config if config is not None else default_config(**cfg)
        h = _h()
        _bcheck(_lib.empc_batch_create(descs, len(problems), ctypes.byref(c), ctypes.byref(h)),
                None)
        self.handle = h
        self.total_knots = sum(m * p for _, m, _, p, _ in self.dims)

    def close(self):
        if getattr(self, "handle", None):
            _lib.empc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        inf = empc_batch_info()
        _bcheck(_lib.empc_batch_get_info(self.handle, ctypes.byref(inf)), self.handle)
        return inf

    def solve(self, generations):
        """(list of best knot vectors, costs[count]) after `generations`."""
        knots = np.zeros(self.total_knots, np.float32)
        costs = np.zeros(len(self.dims), np.float32)
        _bcheck(_lib.empc_batch_solve(self.handle, int(generations), knots.ctypes.data_as(_fp),
                                      costs.ctypes.data_as(_fp)), self.handle)
        out, at = [], 0
        for _, m, _, p, _ in self.dims:
            out.append(knots[at:at + m * p].copy())
            at += m * p
        return out, costs

    def solve_device(self, generations):
        """Asynchronous solve on the batch's stream; results stay on the device."""
        _bcheck(_lib.empc_batch_solve_device(self.handle, int(generations)), self.handle)

    def set_stream(self, stream):
        _bcheck(_lib.empc_batch_set_stream(self.handle, stream), self.handle)

    def reset(self):
        _bcheck(_lib.empc_batch_reset(self.handle), self.handle)

    def set_targets(self, x0s, goals):
        """New start states and goals (one array per problem), used from the
        next generation on; the populations are kept."""
        x = np.ascontiguousarray(np.concatenate([np.ravel(v) for v in x0s]), np.float64)
        g = np.ascontiguousarray(np.concatenate([np.ravel(v) for v in goals]), np.float64)
        if x.size != sum(d[0] for d in self.dims) or g.size != x.size:
            raise ValueError("need one x0 and one goal of length n per problem")
        _bcheck(_lib.empc_batch_set_targets(self.handle, x.ctypes.data_as(_dp),
                                            g.ctypes.data_as(_dp)), self.handle)

    def get_state(self, index, pop=None, cost=None, elite=None):
        _bcheck(_lib.empc_batch_get_state(self.handle, int(index), _dev(pop), _dev(cost),
                                          _dev(elite)), self.handle)

    def inject_stall(self, problem, timeout_s):
        _bcheck(_lib.empc_batch_inject_stall(self.handle, int(problem), float(timeout_s)),
                self.handle)
