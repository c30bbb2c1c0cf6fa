/*
 * empc.h - C ABI of the GB300 evolutionary-MPC (EMPC) library.
 *
 * One generation of EMPC, after Hyatt, Williams & Killpack, "Parameterized
 * and GPU-Parallelized Real-Time Model Predictive Control for High Degree of
 * Freedom Robots" (arXiv 2001.04931), Sec. V and Algorithm 1:
 *   breed (cold start: uniform in the input bounds; warm start: two parents
 *   drawn from the elites, uniform crossover, Gaussian mutation, clip),
 *   expand the knots into per-step inputs (Sec. IV-C), roll the discrete
 *   linear model forward (Eq. first_order_integration), accumulate the
 *   quadratic cost (Eq. mpc_problem), keep the E best (elitism).
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  Host inputs are FP64 and copied at call time;
 *    the caller keeps ownership of every buffer it passes.
 *  - "dev" pointers are CUDA device pointers on the handle's device; "host"
 *    pointers are ordinary host memory.  Device-pointer calls are
 *    asynchronous on the handle's stream; host-pointer calls return after the
 *    results are in the caller's buffers.
 *  - The population is SoA FP32: parameter q = i*p + j (input i, knot j) of
 *    candidate c is pop[q*P + c].
 *  - Every call returns an empc_status; nothing throws across the ABI.  On
 *    failure empc_last_error(h) (or empc_last_error(NULL) for calls without
 *    a handle) describes the cause.
 *  - A handle is not thread-safe: one host thread at a time.
 *  - There is no CPU fallback: without a usable CUDA device, calls that need
 *    one fail with EMPC_ECUDA.
 */
#ifndef EMPC_H
#define EMPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct empc_problem_s* empc_handle;

typedef enum {
    EMPC_OK = 0,
    EMPC_EINVAL = 1,       /* bad argument (null pointer, size, bound, non-finite input) */
    EMPC_ENOMEM = 2,       /* device or pinned host allocation failed */
    EMPC_ECUDA = 3,        /* CUDA runtime error (no device, launch failure, ...) */
    EMPC_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
    EMPC_ENONFINITE = 5,   /* the best cost is +inf or NaN (unstable model or inputs) */
    EMPC_ESTATE = 6,       /* call not valid in the handle's state */
    EMPC_EUNSUPPORTED = 7  /* valid request outside what the GPU path implements */
} empc_status;

/* Arithmetic of the rollout.  FP32: FP32 CUDA-core kernels, costs within
 * 1e-5 relative of the FP64 definition.  BF16 (no counterpart in the paper):
 * the per-step product x_k D' + u_k B_d' on the tensor cores (tcgen05) with
 * BF16 operands, the state, the force and the cost accumulated in FP32; it
 * needs n <= 128 and m <= 64 and takes no refinement, disturbance or state
 * box; its costs differ from the FP64 definition by the BF16 rounding of
 * the operands (measured: 1.5e-4 relative at most on a 64-DoF chain over 200
 * steps, up to 2.6e-3 on small chains).  Its device waits are bounded in
 * time, one second unless empc_inject_stall sets another limit. */
typedef enum { EMPC_FP32 = 0, EMPC_BF16 = 1 } empc_precision;

/* How population costs are evaluated.  ROLLOUT simulates every candidate
 * over the horizon (Sec. V-A).  CONDENSED uses the parameterized small-matrix
 * form of the linear-quadratic problem (Sec. IV-B, IV-E): J(U) = U'HU + g'U +
 * c0 with H fixed at create (FP64 on the host, used in FP32) and g = dJ/dU(0),
 * c0 = J(0) from one adjoint evaluation per solve; the same costs up to
 * rounding, in 2 (m p)^2 flops per candidate instead of T (2 n^2 + 6 n).
 * CONDENSED needs FP32, n <= 64, m p <= 832 and no refinement. */
typedef enum { EMPC_EVAL_ROLLOUT = 0, EMPC_EVAL_CONDENSED = 1 } empc_evaluator;

/* Granularity of the 50% mutation decision (Sec. V gates the mutation per
 * input with probability one half; Algorithm 1 adds the noise without a gate). */
typedef enum {
    EMPC_GATE_PER_INPUT = 0, /* one decision per (child, input); all its knots move together */
    EMPC_GATE_PER_KNOT = 1,  /* one decision per (child, knot parameter) */
    EMPC_GATE_ALWAYS = 2     /* every parameter mutated (Algorithm 1 read literally) */
} empc_gate;

typedef struct {
    uint64_t seed;       /* Philox4x32-10 key (lo, hi words) */
    int elite;           /* numParents E; 0 = max(1, P/16) */
    float sigma;         /* sigma_noise of the mutation, default 0.1 */
    int p_cross_256;     /* P(take parameter from parent 2) * 256, default 128 */
    int p_mutate_256;    /* P(mutate) * 256, default 128 */
    int gate;            /* empc_gate, default EMPC_GATE_PER_INPUT */
    int precision;       /* empc_precision, default EMPC_FP32 */
    int refine_steps;    /* projected-gradient steps on the elites per generation, default 0 */
    float refine_lr;     /* step size; 0 = 1/L, L the gradient's Lipschitz constant */
    int ckpt_every;      /* adjoint checkpoint interval; 0 = ceil(sqrt(T)) */
    int tile;            /* 0 = autotune the rollout tile; k > 0 forces candidate shape k-1 */
    int evaluator;       /* empc_evaluator, default EMPC_EVAL_ROLLOUT */
} empc_config;

typedef struct {
    int n, m, horizon, knots, pop, elite;
    uint64_t generation;     /* generations run so far (keys the next draws) */
    int tile_nx, tile_rows, tile_cands, tile_groups; /* rollout tile chosen */
    int threads_per_cta, smem_bytes, ctas;
    float tuned_us;          /* autotuner's best rollout time (microseconds), 0 if forced */
    float refine_lr;         /* projected-gradient step in use */
    int tile_kind;           /* 0: block-synchronous rollout, 1: warp-synchronous */
    int ckpt_every;          /* adjoint checkpoint interval in use */
} empc_info;

/* Defaults listed in empc_config. */
void empc_config_default(empc_config* cfg);

/*
 * empc_create - build a problem on the current CUDA device.
 *   A [n*n], B [n*m]  discrete model x_{k+1} = A x_k + B u_k (Eq.
 *                     first_order_integration, w_d = 0); host FP64.
 *   Q [n*n], R [m*m]  cost weights of Eq. mpc_problem (u_goal = 0); host FP64,
 *                     dense or diagonal.  Only their symmetric parts enter the
 *                     cost; those must be positive semidefinite (else
 *                     EMPC_EINVAL).  A diagonal Q is used as it is.  A
 *                     non-diagonal Q is diagonalized on the host (Q_s = V
 *                     diag(lambda) V', FP64 Jacobi) and every rollout runs in
 *                     z = V'x, where the model is V'AV, V'B and the weight
 *                     diag(lambda): the same J for every knot vector, with no
 *                     per-step cost beyond the diagonal one.  Start states,
 *                     goals and disturbances are rotated on the way in; the
 *                     state box (empc_set_state_box), which acts on x, is then
 *                     not available.  A non-diagonal R enters the input cost
 *                     through the knot-weight Gram W: sum_ij R_ij U_i' W U_j.
 *   bounds [m*2]      (u_min, u_max) per input; knots are clipped to them.
 *   horizon T >= 1, knots p in [1, T] (Sec. IV-C), pop P >= 1, n <= 128.
 *   cfg               NULL for defaults.
 * The cost of a knot vector U is
 *   J(U) = sum_{k=0}^{T-1} (x_{k+1}-g)' Q (x_{k+1}-g) + u_k' R u_k,
 * the stage cost taken after each update as Algorithm 1 accumulates it.
 * Allocates all device memory the handle needs; *out receives the handle.
 */
empc_status empc_create(const double* A, const double* B, const double* Q, const double* R,
                        const double* bounds, int n, int m, int horizon, int knots, int pop,
                        const empc_config* cfg, empc_handle* out);

/*
 * empc_solve - run `generations` >= 1 generations of Algorithm 1 from host
 * x0 [n] and x_goal [n] (FP64).  The population persists across calls (warm
 * start, Sec. V); the first call after create or empc_reset starts cold.
 * Writes the best knot vector (host, [m*p], parameter q = i*p + j) and its
 * cost.  u* of Algorithm 1 is best_knots[i*p + 0] for each input i.
 * Host-to-device copy of x0/x_goal, the generations, and the device-to-host
 * copy of the result all happen inside the call (the EMPC solve time of the
 * simulation experiments, Sec. VI-A).  Returns EMPC_ENONFINITE if the best cost is not finite.
 */
empc_status empc_solve(empc_handle h, const double* x0, const double* x_goal,
                       int generations, float* best_knots, float* best_cost);

/*
 * empc_set_sigma - the standard deviation of the mutation noise used from
 * the next generation on (initially empc_config.sigma).  Stream-ordered on
 * the handle's stream; EMPC_EINVAL unless finite and >= 0.
 */
empc_status empc_set_sigma(empc_handle h, float sigma);

/*
 * empc_set_disturbance - the constant disturbance w_d of Eq.
 * first_order_integration, x_{k+1} = A_d x_k + B_d u_k + w_d: host FP64
 * w_d [n], rounded to FP32 for the rollouts; NULL or all zeros removes it.
 * It applies to every later solve, evaluation and gradient (and so to the
 * condensed evaluator's terms), and empc_closed_loop adds it to its plant.
 * Copies the array before returning.  EMPC_EINVAL for a non-finite entry;
 * EMPC_EUNSUPPORTED for a non-zero w_d with BF16 precision.
 */
empc_status empc_set_disturbance(empc_handle h, const double* w_d);

/*
 * empc_inject_stall - failure injection for tests of the BF16 tensor-core
 * rollout (no counterpart in the paper).  From the next launch on, its MMA
 * issuer stops at horizon step `step` (-1: never), so the other threads'
 * waits run out; every wait of that kernel is limited to timeout_s seconds
 * (one second until this is called).  A solve that hits the stall returns
 * EMPC_ETIMEOUT and the context stays usable: call again with step -1 and
 * solve (empc_reset first for a fresh population).  Synchronous.
 * EMPC_EUNSUPPORTED unless the handle's precision is EMPC_BF16; EMPC_EINVAL
 * for step < -1 or timeout_s outside (0, 60].
 */
empc_status empc_inject_stall(empc_handle h, int step, double timeout_s);

/* Flags of empc_set_state_box. */
enum { EMPC_BOX_CLAMP = 1, EMPC_BOX_PENALTY = 2 };

/*
 * empc_set_state_box - a nonlinear hook inside every rollout (Sec. V,
 * simulation and cost calculation: because each state of each step is
 * simulated, hard stops and non-convex state costs can be written into the
 * simulation as if/else).  Per state i, host FP32 arrays of n entries:
 * lo [n] (NULL: -inf), hi [n] (NULL: +inf), rho [n] (NULL: 0).  After every
 * update x_{k+1} = A_d x_k + B_d u_k (+ w_d, empc_set_disturbance), for each
 * state, in this order:
 *   d_i = max(0, lo_i - x_i, x_i - hi_i)   (distance outside the box)
 *   EMPC_BOX_PENALTY:  J += rho_i d_i^2      (soft state limit)
 *   EMPC_BOX_CLAMP:    x_i = min(max(x_i, lo_i), hi_i)   (hard stop)
 * and the stage cost then sees the stopped state, from which the next step
 * starts.  flags = 0 turns the hook off (the arrays are then ignored).  It
 * applies to every later empc_solve, empc_solve_device, empc_evaluate and
 * empc_closed_loop call; empc_closed_loop also stops its plant at the box
 * when EMPC_BOX_CLAMP is set.  Copies the arrays before returning.
 * EMPC_EINVAL unless lo_i <= hi_i, lo_i < +inf, hi_i > -inf and rho_i is
 * finite and >= 0 (NaN fails), or on unknown flag bits; EMPC_EUNSUPPORTED
 * with a non-zero flag for BF16 precision, the condensed evaluator or
 * refinement (none of them simulates the states one by one); while a box is
 * set, empc_grad returns EMPC_EUNSUPPORTED too.
 */
empc_status empc_set_state_box(empc_handle h, const float* lo, const float* hi,
                               const float* rho, int flags);

/*
 * empc_closed_loop - receding-horizon control of a plant (Sec. III-A: solve,
 * apply only the first input, solve again from the new state; Sec. V: EMPC
 * applies the best input after each solve of `generations` generations).
 * For k = 0 .. steps-1: x_k is sent to empc_solve (warm-started from the
 * previous population), u_k = u* (the first knot of each input of the best
 * candidate), and the plant advances in FP64 on the host:
 * x_{k+1} = Ad x_k + Bd u_k.  Ad [n*n] and Bd [n*m] (row-major, host FP64)
 * are the plant, which may differ from the model given to empc_create
 * (model error).  With sigma_dref > 0 the mutation noise depends on the
 * distance to the goal (Sec. VII: exploration that shrinks near the goal
 * keeps the system there): sigma_k = max(sigma_min, sigma min(1, |x_k - g| /
 * sigma_dref)), |.| the Euclidean norm summed in index order in FP64 and
 * sigma the configured one; sigma is restored afterwards.  Outputs:
 * actual_cost (Eq. actual_cost) = sum_k (x_goal - x_k)' Q (x_goal - x_k) +
 * u_k' R u_k over the applied steps plus the state term of the final state
 * x_steps; optional x_traj [(steps+1)*n], u_traj [steps*m] and the mean
 * wall time per step in ms (solve plus plant update).  A disturbance set by
 * empc_set_disturbance is added to the plant update.  With an
 * EMPC_BOX_CLAMP state box (empc_set_state_box) the plant state is stopped
 * at the box after each update.  Errors as empc_solve;
 * EMPC_ENONFINITE if the plant state diverges.
 */
empc_status empc_closed_loop(empc_handle h, const double* Ad, const double* Bd, const double* x0,
                             const double* x_goal, int steps, int generations, double sigma_min,
                             double sigma_dref, double* x_traj, double* u_traj,
                             double* actual_cost, double* ms_per_step);

/*
 * empc_solve_device - as empc_solve with device inputs and outputs:
 * dev_x0 [n], dev_goal [n] (FP32), dev_best_knots [m*p], dev_best_cost [1].
 * Asynchronous on the handle's stream; no host synchronization.
 */
empc_status empc_solve_device(empc_handle h, const float* dev_x0, const float* dev_goal,
                              int generations, float* dev_best_knots, float* dev_best_cost);

/*
 * empc_evaluate - costs of a given population (no breeding): the rollout and
 * cost of Algorithm 1 applied to dev_pop [m*p][count] (SoA with stride
 * `count`), writing dev_cost [count].  Asynchronous.
 */
empc_status empc_evaluate(empc_handle h, const float* dev_x0, const float* dev_goal,
                          const float* dev_pop, int count, float* dev_cost);

/*
 * empc_evaluate_noalloc - empc_evaluate for callers that cannot allocate
 * memory while they run (a real-time control loop where cudaMalloc/cudaFree
 * could stall the device for an unbounded time, or a process whose GPU memory
 * another allocator reserved up front).  The paper has no counterpart; it is
 * a library addition.
 *   A [n*n], B [n*m], Q [n*n], R [m*m]: host FP64, the same model and
 *     weights as empc_create (dense or diagonal; symmetric parts positive
 *     semidefinite, else EMPC_EINVAL); horizon T and knots p as there.
 *   dev_x0 [n], dev_goal [n], dev_pop [m*p][count] (SoA, stride count):
 *     device FP32 inputs; dev_cost [count]: device FP32 output.
 *   stream: a cudaStream_t (NULL = legacy default stream); asynchronous.
 * Allocates nothing, on the device or the host: the per-problem tables live
 * in one fixed device array of 24,992 floats (about 98 KiB) that every
 * device loading the library holds until the process exits; each call
 * copies in only the floats its sizes need.  Limits: n <= 64, m <= 64,
 * T <= 1024, p <= 64; larger sizes return EMPC_EINVAL (use the handle API).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture begins.  Every call shares the array,
 * so calls whose GPU work overlaps race and give wrong costs: order them on
 * one stream.  Failures leave a message for empc_last_error(NULL).
 */
empc_status empc_evaluate_noalloc(const double* A, const double* B, const double* Q,
                                  const double* R, int n, int m, int horizon, int knots,
                                  const float* dev_x0, const float* dev_goal,
                                  const float* dev_pop, int count, float* dev_cost,
                                  void* stream);

/*
 * empc_grad - adjoint gradient of the cost (the empc_create formula) with
 * respect to the knots, for dev_pop [m*p][count] (SoA, stride count):
 * dev_grad [m*p][count] (same layout) and dev_cost [count]; either output
 * may be NULL, not both.  The forward pass keeps the state every ckpt_every
 * steps and the backward pass recomputes each segment from its checkpoint,
 * so memory is O(T/ckpt_every + ckpt_every) states per candidate.  FP32
 * whatever cfg.precision is.  EMPC_EUNSUPPORTED for n > 64, while a state
 * box is set (empc_set_state_box), or when the checkpoints do not fit in
 * shared memory.  Asynchronous.  The paper's
 * optimizer is gradient-free; this is a library addition (with
 * cfg.refine_steps > 0 the elites of every generation take that many
 * projected-gradient steps U <- clip(U - eta dJ/dU) before the next one).
 */
empc_status empc_grad(empc_handle h, const float* dev_x0, const float* dev_goal,
                      const float* dev_pop, int count, float* dev_grad, float* dev_cost);

/*
 * empc_get_state - copy the current population [m*p][P], its costs [P] and
 * the elite indices [E] in rank order (best first) to device buffers; any
 * pointer may be NULL.  Asynchronous.  EMPC_ESTATE before the first solve.
 */
empc_status empc_get_state(empc_handle h, float* dev_pop, float* dev_cost, int* dev_elite);

/*
 * empc_set_state - replace the population, costs and elite indices (all
 * three device buffers required); the next generation breeds from them.
 */
empc_status empc_set_state(empc_handle h, const float* dev_pop, const float* dev_cost,
                           const int* dev_elite);

/* empc_reset - the next generation is a cold start.  The generation counter
 * keeps counting, so draws never repeat within a handle. */
empc_status empc_reset(empc_handle h);

/* empc_set_stream - run subsequent work on `stream` (a cudaStream_t); NULL
 * selects the handle's own stream. */
empc_status empc_set_stream(empc_handle h, void* stream);

empc_status empc_get_info(empc_handle h, empc_info* info);

/*
 * empc_time_generation - measurement aid (no counterpart in the paper): run
 * `reps` warm generations as plain launches on the handle's stream and
 * report the average duration of the fused crossover + mutation kernel, of
 * the rollout + cost kernel and of the elite-selection kernel, from CUDA
 * events around each launch.  The generations are real (the population
 * advances).  EMPC_ESTATE before the first solve.  Synchronizes the stream.
 */
empc_status empc_time_generation(empc_handle h, int reps, float* breed_us, float* rollout_us,
                                 float* select_us);

/*
 * empc_measure_fp32_peak - measurement aid (no counterpart in the paper):
 * FP32 fused-multiply-add throughput of the current device in TFLOP/s (2
 * flops per FMA) from a register-only kernel, best of 5 timed launches.
 */
empc_status empc_measure_fp32_peak(double* tflops);

/* empc_destroy - free the handle and its device memory (NULL is a no-op). */
void empc_destroy(empc_handle h);

/* empc_last_error - text of the last failure on h (or of the calling thread
 * for calls without a handle when h is NULL).  Owned by the library. */
const char* empc_last_error(empc_handle h);

/* ---------------------------------------------------------------------- */
/* Batched EMPC: many independent problems in one persistent launch (no    */
/* counterpart in the paper).                                              */
/* ---------------------------------------------------------------------- */
typedef struct empc_batch_s* empc_batch;

/* One problem of a batch: the empc_create arguments plus its start, goal and
 * breeding seed.  All host FP64 except seed/sigma; n <= 64.  elite 0 =
 * max(1, pop/16); sigma 0 = the batch config's sigma. */
typedef struct {
    const double* A;
    const double* B;
    const double* Q;
    const double* R;
    const double* bounds;
    const double* x0;
    const double* x_goal;
    int n, m, horizon, knots, pop, elite;
    uint64_t seed;
    float sigma;
} empc_problem_desc;

typedef struct {
    int count, total_knots;
    int ctas, warps_per_cta, cands_per_lane, items_per_generation;
    double state_steps_per_generation;  /* sum over problems of pop * horizon */
    float tuned_us;                     /* autotuned cold generation of the whole batch */
    int h2d_bytes_targets;              /* bytes one empc_batch_set_targets transfers */
    int d2h_bytes_solve;                /* bytes one empc_batch_solve reads back */
} empc_batch_info;

/*
 * empc_batch_create - upload `count` problems (copied; caller keeps
 * ownership) into one device arena and autotune the persistent launch shape
 * (warps per CTA, candidates per lane) on a cold generation.  cfg supplies
 * the shared breeding parameters (p_cross_256, p_mutate_256, gate, sigma
 * default); cfg.tile > 0 forces launch shape tile-1.  FP32, no refinement.
 * Q and R as in empc_create (dense or diagonal; a problem with a
 * non-diagonal Q runs in Q's eigenbasis, its x0 and goal rotated on the
 * host here and in empc_batch_set_targets).
 */
empc_status empc_batch_create(const empc_problem_desc* probs, int count, const empc_config* cfg,
                              empc_batch* out);

/*
 * empc_batch_solve - `generations` generations of every problem in one
 * persistent kernel launch (replayed from a cached CUDA graph).  Outputs
 * (host): best_knots, the problems' best knot vectors concatenated in order
 * ([m_i * p_i] each), and best_costs [count].  Populations persist (warm
 * start); empc_batch_reset makes the next generation cold.  Device waits are
 * bounded; if one runs out the call returns EMPC_ETIMEOUT and the next solve
 * starts cold.  EMPC_ENONFINITE if a problem's best cost is not finite.
 */
empc_status empc_batch_solve(empc_batch b, int generations, float* best_knots, float* best_costs);
/* As empc_batch_solve without the copies back: asynchronous on the batch's
 * stream (results stay on the device; read them with empc_batch_get_state).
 * A wait that runs out is reported by the next empc_batch_solve. */
empc_status empc_batch_solve_device(empc_batch b, int generations);
/* Run subsequent batch work on `stream` (a cudaStream_t); NULL selects the
 * batch's own stream. */
empc_status empc_batch_set_stream(empc_batch b, void* stream);
/*
 * empc_batch_set_targets - new start states and goals for every problem, as in
 * a receding-horizon step where each problem's x0 is the measured state
 * (Sec. III-A).  x0 and x_goal are host FP64, the problems' vectors
 * concatenated in order ([n_i] each); both are copied (rounded to FP32) to the
 * device on the batch's stream in one transfer and used from the next
 * generation on.  Populations are kept, so the next solve warm-starts from
 * the previous plan.  EMPC_EINVAL on NULL or non-finite input.
 */
empc_status empc_batch_set_targets(empc_batch b, const double* x0, const double* x_goal);
empc_status empc_batch_reset(empc_batch b);
/* Current population [m*p][pop], costs [pop] and elites [E] of problem
 * `index` into device buffers (any may be NULL); synchronous. */
empc_status empc_batch_get_state(empc_batch b, int index, float* dev_pop, float* dev_cost,
                                 int* dev_elite);
empc_status empc_batch_get_info(empc_batch b, empc_batch_info* info);
/* Failure injection for tests: problem `problem` (-1: none) never publishes
 * its selected generation, so every wait on it runs out after timeout_s
 * seconds (also the wait limit used from now on). */
empc_status empc_batch_inject_stall(empc_batch b, int problem, double timeout_s);
void empc_batch_destroy(empc_batch b);
const char* empc_batch_last_error(empc_batch b);

/*
 * empc_discretize_zoh - zero-order-hold discretization of x' = Ac x + Bc u
 * over dt (Sec. III-A, "matrix exponential"): [[Ad, Bd], [0, I]] =
 * expm([[Ac, Bc], [0, 0]] dt).  Host FP64, row-major; Ad [n*n], Bd [n*m]
 * are caller-owned outputs.  Needs no GPU.
 */
empc_status empc_discretize_zoh(const double* Ac, const double* Bc, int n, int m, double dt,
                                double* Ad, double* Bd);

#ifdef __cplusplus
}
#endif

#endif /* EMPC_H */
