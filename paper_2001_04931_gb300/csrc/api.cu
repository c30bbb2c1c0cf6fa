// Host side of the EMPC C ABI (include/empc.h): validation, model staging,
// device buffers, the per-generation launch sequence, CUDA-graph capture of a
// whole solve, and the rollout-tile autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/empc.h"
#include "empc_internal.h"
#include "host_tables.h"

using empc::KnotStep;
using empc::RolloutArgs;
using empc::TileShape;

namespace {

thread_local std::string g_thread_error;

struct GraphKey {
    int generations;
    int cold_first;
    int parity;
    bool operator<(const GraphKey& o) const {
        return std::tie(generations, cold_first, parity) <
               std::tie(o.generations, o.cold_first, o.parity);
    }
};

}  // namespace

struct empc_problem_s {
    int n = 0, m = 0, T = 0, p = 0, P = 0, E = 0, D = 0;
    empc_config cfg{};
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    // model, FP32 on device
    float *D_ = nullptr, *BT = nullptr, *qdiag = nullptr, *rdiag = nullptr, *gram = nullptr;
    float *umin = nullptr, *umax = nullptr, *x0 = nullptr, *goal = nullptr;
    float* rmat = nullptr;     // dense symmetric R [m][m] (null when R is diagonal)
    // non-diagonal Q: the rollouts run in z = Vt x (Q's eigenbasis); Vt in
    // FP64 on the host and the device, and device scratch for rotated inputs
    // of empc_evaluate / empc_grad
    bool rotated = false;
    std::vector<double> Vt_h;
    double* Vt_dev = nullptr;
    float *ev_x0 = nullptr, *ev_goal = nullptr;
    KnotStep* ktab = nullptr;
    // population state
    float* pop[2] = {nullptr, nullptr};
    float* cost = nullptr;
    int* elite_idx = nullptr;
    float* elite_cost = nullptr;
    float* best_knots = nullptr;
    float* best_cost = nullptr;
    uint32_t* gen = nullptr;
    int* status = nullptr;
    // pinned staging: x0, goal (2n) | best knots (D) | best cost | status
    float* stage = nullptr;
    int cur = 0;
    bool has_pop = false;
    uint64_t gen_host = 0;
    TileShape shape{};
    float tuned_us = 0.0f;
    // refinement (projected gradient on the elites) and the adjoint
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int ce = 1;            // checkpoint interval
    float eta = 0.0f;      // refinement step
    int grad_cands = 1, grad_wpc = 2;      // adjoint shape for whole populations (empc_grad)
    int refine_cands = 1, refine_wpc = 2;  // adjoint shape for the elites' refinement
    int grad_nx = 0;  // the adjoint kernel's state class (the warp family's, n <= 64)
    float* sigma_dev = nullptr;  // the mutation sigma the breeding kernel reads
    int* inject = nullptr;       // tensor-core rollout: [stall step, wait limit us]
    int inject_h[2] = {-1, 1000000};  // host copy being transferred to inject
    float sigma_now = 0.0f;      // host copy being transferred to sigma_dev
    // state-box hook: [3][n] lo, hi, rho on the device and its host copy
    float* box = nullptr;
    std::vector<float> box_h;
    int box_mode = 0;
    // constant disturbance w_d: [n] FP32 on the device, FP64 host copy
    float* wd_dev = nullptr;
    std::vector<double> wd_h;
    bool has_wd = false;
    // Q and R in FP64 (closed-loop actual cost)
    std::vector<double> Q_h, R_h;
    // condensed evaluator: J(U) = U'HU + g'U + c0 (H padded to Dp x Dp)
    int Dp = 0;
    float *Hc = nullptr, *gvec = nullptr, *c0 = nullptr, *zero_knots = nullptr;
    std::map<GraphKey, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

empc_status fail(empc_handle h, empc_status s, const std::string& msg) {
    if (h) h->err = msg;
    g_thread_error = msg;
    return s;
}

empc_status cuda_fail(empc_handle h, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorName(e) + " (" +
                      cudaGetErrorString(e) + ")";
    return fail(h, EMPC_ECUDA, msg);
}

#define EMPC_CUDA(h, call)                                          \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<size_t>(count, 1));
}

RolloutArgs base_args(empc_handle h) {
    RolloutArgs a{};
    a.D = h->D_;
    a.BT = h->BT;
    a.qdiag = h->qdiag;
    a.rdiag = h->rdiag;
    a.rmat = h->rmat;
    a.gram = h->gram;
    a.ktab = h->ktab;
    a.x0 = h->x0;
    a.goal = h->goal;
    a.umin = h->umin;
    a.umax = h->umax;
    a.n = h->n;
    a.m = h->m;
    a.T = h->T;
    a.p = h->p;
    a.P = h->P;
    a.E = h->E;
    a.seed = h->cfg.seed;
    a.gen = h->gen;
    a.sigma = h->cfg.sigma;
    a.sigma_dev = h->sigma_dev;
    a.box = h->box;
    a.box_mode = h->box_mode;
    a.wd = h->has_wd ? h->wd_dev : nullptr;
    a.pc256 = h->cfg.p_cross_256;
    a.pm256 = h->cfg.p_mutate_256;
    a.gate = h->cfg.gate;
    a.status = h->status;
    a.inject = h->inject;
    return a;
}

empc::GradArgs grad_args(empc_handle h) {
    empc::GradArgs g{};
    g.D = h->D_;
    g.BT = h->BT;
    g.qdiag = h->qdiag;
    g.rdiag = h->rdiag;
    g.rmat = h->rmat;
    g.gram = h->gram;
    g.ktab = h->ktab;
    g.x0 = h->x0;
    g.goal = h->goal;
    g.wd = h->has_wd ? h->wd_dev : nullptr;
    g.umin = h->umin;
    g.umax = h->umax;
    g.n = h->n;
    g.m = h->m;
    g.T = h->T;
    g.p = h->p;
    g.ce = h->ce;
    g.eta = h->eta;
    return g;
}

// Costs of the population a.pop_in into a.cost: the rollout kernel, or the
// condensed quadratic form (g and c0 of the current start and goal must have
// been computed by condensed_terms earlier on the stream).
cudaError_t evaluate_population(empc_handle h, const RolloutArgs& a, cudaStream_t st) {
    if (h->cfg.evaluator == EMPC_EVAL_CONDENSED) {
        const empc::CondArgs c{h->Hc, h->gvec, h->c0, a.pop_in, a.cost, h->D, h->Dp, h->P};
        // the P x D x D product on the tensor cores where D fits one MMA's N
        if (empc::condensed_tc_supported(h->Dp))
            return empc::launch_condensed_tc(c, h->status, st, a.pdl != 0);
        return empc::launch_condensed(c, st, a.pdl != 0);
    }
    return empc::launch_rollout(a, h->shape, st);
}

// g = dJ/dU at U = 0 and c0 = J(0) for the current start state and goal:
// one adjoint evaluation of the zero knot vector.
cudaError_t condensed_terms(empc_handle h, cudaStream_t st) {
    empc::GradArgs g = grad_args(h);
    g.x0 = h->x0;
    g.goal = h->goal;
    g.pop_in = h->zero_knots;
    g.ld_in = 1;
    g.count = 1;
    g.grad = h->gvec;
    g.ld_grad = 1;
    g.cost = h->c0;
    g.steps = 0;
    return empc::launch_grad(g, h->grad_nx, h->grad_cands, h->grad_wpc, st);
}

// One generation into pop[parity^1], then elite selection.  Cold: draw every
// candidate, then roll out and cost them.  Warm: the fused crossover +
// mutation kernel breeds the children (slots E..P-1) from the previous
// elites and copies the elites, then the rollout kernel evaluates them; with
// refinement enabled the elites themselves are refined by projected gradient
// on a second stream at the same time and written, with their costs, to
// slots 0..E-1.
cudaError_t enqueue_generation(empc_handle h, bool cold, int parity, cudaStream_t st) {
    RolloutArgs a = base_args(h);
    a.mode = cold ? empc::kCold : empc::kWarm;
    a.pop_in = h->pop[parity];
    a.pop_out = h->pop[parity ^ 1];
    a.cost = h->cost;
    a.elite_idx = h->elite_idx;
    const bool refine = !cold && h->cfg.refine_steps > 0;
    cudaError_t e = cudaSuccess;
    if (refine) {
        a.cand_begin = h->E;
        empc::GradArgs g = grad_args(h);
        g.pop_in = h->pop[parity];
        g.ld_in = h->P;
        g.index = h->elite_idx;
        g.count = h->E;
        g.cost = h->cost;
        g.pop_out = h->pop[parity ^ 1];
        g.ld_out = h->P;
        g.steps = h->cfg.refine_steps;
        if ((e = cudaEventRecord(h->ev_fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0)) != cudaSuccess) return e;
        e = empc::launch_grad(g, h->grad_nx, h->refine_cands, h->refine_wpc, h->aux_stream);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventRecord(h->ev_join, h->aux_stream)) != cudaSuccess) return e;
    }
    // Programmatic dependent launch between the generation's kernels (not
    // across the refinement fork/join).
    a.pdl = refine ? 0 : 1;
    e = empc::launch_breed(a, st);
    if (e != cudaSuccess) return e;
    a.mode = empc::kEval;  // the evaluator reads the bred population
    a.pop_in = h->pop[parity ^ 1];
    e = evaluate_population(h, a, st);
    if (e != cudaSuccess) return e;
    if (refine && (e = cudaStreamWaitEvent(st, h->ev_join, 0)) != cudaSuccess) return e;
    return empc::launch_select(h->cost, h->P, h->E, h->pop[parity ^ 1], h->D, h->elite_idx,
                               h->elite_cost, h->best_knots, h->best_cost, h->gen, h->status,
                               st, !refine);
}

// The condensed Hessian H of J = U'HU + 2f'U + c in the knots (Sec. IV-E),
// FP64, row-major D x D.  The columns of S (stacked states x_1..x_T per unit
// knot, zero x0) come from rollouts of the parameterized dynamics;
// H = S' Qbig S + sum_k Om_k' R Om_k, with the symmetric parts of Q and R
// (dense or diagonal).
std::vector<double> condensed_hessian(const double* A, const double* B, const double* Q,
                                      const double* R, int n, int m, int T, int p,
                                      const std::vector<int>& idx, const std::vector<double>& w0,
                                      const std::vector<double>& w1) {
    const int D = m * p;
    std::vector<double> S((size_t)T * n * D, 0.0), x(n), xn(n);
    for (int q = 0; q < D; ++q) {
        const int i = q / p, a = q % p;
        std::fill(x.begin(), x.end(), 0.0);
        for (int k = 0; k < T; ++k) {
            double u = 0.0;
            if (idx[k] == a) u += w0[k];
            if (p > 1 && idx[k] + 1 == a) u += w1[k];
            for (int r = 0; r < n; ++r) {
                double v = B[(size_t)r * m + i] * u;
                for (int j = 0; j < n; ++j) v += A[(size_t)r * n + j] * x[j];
                xn[r] = v;
            }
            x.swap(xn);
            for (int r = 0; r < n; ++r) S[((size_t)k * n + r) * D + q] = x[r];
        }
    }
    std::vector<double> H((size_t)D * D, 0.0), QS((size_t)n * D);
    for (int k = 0; k < T; ++k) {
        // QS = Q_s S_k, then H += S_k' QS
        const double* Sk = &S[(size_t)k * n * D];
        for (int r = 0; r < n; ++r)
            for (int a = 0; a < D; ++a) {
                double v = 0.0;
                for (int j = 0; j < n; ++j) {
                    const double q = 0.5 * (Q[(size_t)r * n + j] + Q[(size_t)j * n + r]);
                    if (q != 0.0) v += q * Sk[(size_t)j * D + a];
                }
                QS[(size_t)r * D + a] = v;
            }
        for (int r = 0; r < n; ++r) {
            const double* row = &Sk[(size_t)r * D];
            for (int a = 0; a < D; ++a) {
                if (row[a] == 0.0) continue;
                for (int b = 0; b < D; ++b) H[(size_t)a * D + b] += row[a] * QS[(size_t)r * D + b];
            }
        }
    }
    // input cost: u_k = sum_a w_ka U_a, so H[(i,a),(j,b)] += R_s,ij w_ka w_kb
    for (int k = 0; k < T; ++k)
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                const double rij = 0.5 * (R[(size_t)i * m + j] + R[(size_t)j * m + i]);
                if (rij == 0.0) continue;
                const int a = i * p + idx[k], b = j * p + idx[k];
                H[(size_t)a * D + b] += rij * w0[k] * w0[k];
                if (p > 1) {
                    H[(size_t)(a + 1) * D + (b + 1)] += rij * w1[k] * w1[k];
                    H[(size_t)a * D + (b + 1)] += rij * w0[k] * w1[k];
                    H[(size_t)(a + 1) * D + b] += rij * w1[k] * w0[k];
                }
            }
    return H;
}

// Largest eigenvalue of the condensed Hessian, for the projected-gradient
// step 1/L with L = 2 lambda_max(H).  Power iteration.
double hessian_lambda_max(const std::vector<double>& H, int D) {
    std::vector<double> v(D, 1.0), hv(D);
    double lam = 0.0;
    for (int it = 0; it < 500; ++it) {
        double nrm = 0.0;
        for (int a = 0; a < D; ++a) {
            double t = 0.0;
            for (int b = 0; b < D; ++b) t += H[(size_t)a * D + b] * v[b];
            hv[a] = t;
            nrm += t * t;
        }
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) return 0.0;
        double vn = 0.0;
        for (int a = 0; a < D; ++a) vn += v[a] * v[a];
        const double next = nrm / std::sqrt(vn);
        for (int a = 0; a < D; ++a) v[a] = hv[a] / nrm;
        if (std::fabs(next - lam) <= 1e-12 * next) {
            lam = next;
            break;
        }
        lam = next;
    }
    return lam;
}

// Row i of the rollout coordinates of a host FP64 vector: (Vt v)_i in FP64
// when the rollouts run in Q's eigenbasis, else v_i.
double rotate_row(empc_handle h, const double* v, int i) {
    if (!h->rotated) return v[i];
    double s = 0.0;
    for (int j = 0; j < h->n; ++j) s += h->Vt_h[(size_t)i * h->n + j] * v[j];
    return s;
}

// Device start and goal in the rollout coordinates: rotated into (zx, zg)
// when Q is not diagonal, else copied (or, with zx == x, used in place).
cudaError_t stage_targets(empc_handle h, const float* x, const float* g, float* zx, float* zg) {
    if (h->rotated) return empc::launch_rotate(h->Vt_dev, x, g, zx, zg, h->n, h->stream);
    cudaError_t e = cudaSuccess;
    if (zx != x) e = cudaMemcpyAsync(zx, x, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && zg != g)
        e = cudaMemcpyAsync(zg, g, sizeof(float) * h->n, cudaMemcpyDeviceToDevice, h->stream);
    return e;
}

empc_status run_generations(empc_handle h, int G) {
    const GraphKey key{G, h->has_pop ? 0 : 1, h->cur};
    auto it = h->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != h->graphs.end()) {
        exec = it->second;
    } else {
        cudaStream_t cap = h->own_stream;
        EMPC_CUDA(h, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        bool cold = !h->has_pop;
        int parity = h->cur;
        cudaError_t e = cudaSuccess;
        if (h->cfg.evaluator == EMPC_EVAL_CONDENSED) e = condensed_terms(h, cap);
        for (int g = 0; g < G && e == cudaSuccess; ++g) {
            e = enqueue_generation(h, cold, parity, cap);
            cold = false;
            parity ^= 1;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(h, e, "enqueue_generation (capture)");
        }
        if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        h->graphs[key] = exec;
    }
    EMPC_CUDA(h, cudaGraphLaunch(exec, h->stream));
    h->cur ^= (G & 1);
    h->has_pop = true;
    h->gen_host += (uint64_t)G;
    return EMPC_OK;
}

empc_status autotune(empc_handle h) {
    std::vector<TileShape> ok;
    if (h->cfg.precision == EMPC_BF16) {
        // tensor-core tile: 128 candidates, one shape
        ok.push_back(TileShape{2, 128, 1, 1, 1});
    } else {
        TileShape buf[128];
        const int ns = std::min(empc::rollout_shapes(h->n, buf, 128), 128);
        for (int i = 0; i < ns; ++i)
            if (empc::rollout_shape_supported(buf[i], h->n, h->m, h->p, h->T)) ok.push_back(buf[i]);
    }
    if (ok.empty()) return fail(h, EMPC_EUNSUPPORTED, "no rollout tile fits this problem");
    // score the rollout of a cold-drawn population of the real size
    RolloutArgs a = base_args(h);
    a.mode = empc::kCold;
    a.pop_out = h->pop[0];
    a.cost = h->cost;
    a.gen = nullptr;
    EMPC_CUDA(h, empc::launch_breed(a, h->stream));
    a.mode = empc::kEval;
    a.pop_in = h->pop[0];
    if (h->cfg.tile > 0) {
        const size_t k = (size_t)(h->cfg.tile - 1);
        if (k >= ok.size()) return fail(h, EMPC_EINVAL, "cfg.tile out of range");
        h->shape = ok[k];
        // one launch outside any capture sets the kernel's shared-memory cap
        EMPC_CUDA(h, empc::launch_rollout(a, h->shape, h->stream));
        EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
        return EMPC_OK;
    }
    cudaEvent_t e0, e1;
    EMPC_CUDA(h, cudaEventCreate(&e0));
    EMPC_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f;
    TileShape best_s = ok[0];
    for (const TileShape& s : ok) {
        if (empc::launch_rollout(a, s, h->stream) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        float t_min = 1e30f;
        bool good = true;
        for (int rep = 0; rep < 3 && good; ++rep) {
            cudaEventRecord(e0, h->stream);
            good = empc::launch_rollout(a, s, h->stream) == cudaSuccess;
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) good = false;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            t_min = std::min(t_min, ms);
        }
        // a shape whose kernel gave up a bounded wait finished early: not a candidate
        int st_word = 0;
        if (good && (cudaMemcpy(&st_word, h->status, sizeof(int), cudaMemcpyDeviceToHost) !=
                         cudaSuccess ||
                     st_word != 0)) {
            good = false;
            cudaMemset(h->status, 0, sizeof(int));
        }
        if (!good) {
            cudaGetLastError();
            continue;
        }
        if (t_min < best) {
            best = t_min;
            best_s = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
    h->shape = best_s;
    h->tuned_us = best * 1000.0f;
    return EMPC_OK;
}

// Adjoint kernel shapes (candidates per lane 1 or 2, warps per CTA 4, 2 or
// 1, within shared memory), each timed on the cold population the rollout
// autotuner drew: the gradient of the whole population (empc_grad) and, with
// refinement on, the refinement of E elites.  The per-candidate arithmetic
// does not depend on the shape.  Leaves grad_wpc = 0 when no shape fits.
empc_status autotune_grad(empc_handle h) {
    struct Shape {
        int cands, wpc;
    };
    std::vector<Shape> ok;
    for (int c : {1, 2})
        for (int wpc : {4, 2, 1})
            if (empc::grad_smem_bytes(h->grad_nx, empc::warp_nrg(h->grad_nx), c, wpc, h->n, h->m,
                                      h->p, h->T, h->ce) <= 227u * 1024u)
                ok.push_back(Shape{c, wpc});
    h->grad_wpc = h->refine_wpc = 0;
    if (ok.empty()) return EMPC_OK;
    cudaEvent_t e0, e1;
    EMPC_CUDA(h, cudaEventCreate(&e0));
    EMPC_CUDA(h, cudaEventCreate(&e1));
    auto time_shape = [&](const Shape& sh, bool refine) {
        empc::GradArgs g = grad_args(h);
        g.pop_in = h->pop[0];
        g.ld_in = h->P;
        g.cost = h->cost;
        if (refine) {  // E elites (the first E columns), written to the spare buffer
            g.count = h->E;
            g.pop_out = h->pop[1];
            g.ld_out = h->P;
            g.steps = h->cfg.refine_steps;
        } else {  // the gradient of every candidate, into the spare buffer
            g.count = h->P;
            g.grad = h->pop[1];
            g.ld_grad = h->P;
            g.steps = 0;
        }
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, h->stream);
            const cudaError_t e = empc::launch_grad(g, h->grad_nx, sh.cands, sh.wpc, h->stream);
            cudaEventRecord(e1, h->stream);
            if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                return 1e30f;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    float bg = 1e30f, br = 1e30f;
    for (const Shape& sh : ok) {
        const float tg = time_shape(sh, false);
        if (tg < bg) {
            bg = tg;
            h->grad_cands = sh.cands;
            h->grad_wpc = sh.wpc;
        }
        if (h->cfg.refine_steps > 0) {
            const float tr = time_shape(sh, true);
            if (tr < br) {
                br = tr;
                h->refine_cands = sh.cands;
                h->refine_wpc = sh.wpc;
            }
        }
    }
    if (h->cfg.refine_steps <= 0) {
        h->refine_cands = h->grad_cands;
        h->refine_wpc = h->grad_wpc;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->grad_wpc == 0 || h->refine_wpc == 0)
        return fail(h, EMPC_ECUDA, "no adjoint kernel shape ran");
    return EMPC_OK;
}

void free_handle(empc_handle h) {
    if (!h) return;
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    void* bufs[] = {h->D_, h->BT, h->qdiag, h->rdiag, h->gram, h->umin, h->umax, h->x0,
                    h->goal, h->ktab, h->pop[0], h->pop[1], h->cost, h->elite_idx,
                    h->elite_cost, h->best_knots, h->best_cost, h->gen, h->status,
                    h->Hc, h->gvec, h->c0, h->zero_knots, h->sigma_dev, h->inject, h->box,
                    h->wd_dev, h->rmat, h->Vt_dev, h->ev_x0, h->ev_goal};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->stage) cudaFreeHost(h->stage);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

// ---------------------------------------------------------------------------
// Zero-order hold by the matrix exponential: scaling and squaring with the
// diagonal [6/6] Pade approximant (Moler & Van Loan, "Nineteen dubious ways
// to compute the exponential of a matrix", method 3).
// ---------------------------------------------------------------------------
void mat_mul(const std::vector<double>& X, const std::vector<double>& Y,
             std::vector<double>& Z, int N) {
    std::vector<double> out((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < N; ++k) {
            const double x = X[(size_t)i * N + k];
            if (x == 0.0) continue;
            for (int j = 0; j < N; ++j) out[(size_t)i * N + j] += x * Y[(size_t)k * N + j];
        }
    Z.swap(out);
}

bool solve_in_place(std::vector<double> M, std::vector<double>& Bm, int N) {
    // Gaussian elimination with partial pivoting: M X = Bm, X overwrites Bm.
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int r = col + 1; r < N; ++r)
            if (std::fabs(M[(size_t)r * N + col]) > std::fabs(M[(size_t)piv * N + col])) piv = r;
        if (M[(size_t)piv * N + col] == 0.0) return false;
        if (piv != col)
            for (int j = 0; j < N; ++j) {
                std::swap(M[(size_t)piv * N + j], M[(size_t)col * N + j]);
                std::swap(Bm[(size_t)piv * N + j], Bm[(size_t)col * N + j]);
            }
        const double inv = 1.0 / M[(size_t)col * N + col];
        for (int r = 0; r < N; ++r) {
            if (r == col) continue;
            const double f = M[(size_t)r * N + col] * inv;
            if (f == 0.0) continue;
            for (int j = 0; j < N; ++j) {
                M[(size_t)r * N + j] -= f * M[(size_t)col * N + j];
                Bm[(size_t)r * N + j] -= f * Bm[(size_t)col * N + j];
            }
        }
    }
    for (int r = 0; r < N; ++r) {
        const double inv = 1.0 / M[(size_t)r * N + r];
        for (int j = 0; j < N; ++j) Bm[(size_t)r * N + j] *= inv;
    }
    return true;
}

bool expm_pade6(const std::vector<double>& A, int N, std::vector<double>& out) {
    double norm = 0.0;
    for (int i = 0; i < N; ++i) {
        double s = 0.0;
        for (int j = 0; j < N; ++j) s += std::fabs(A[(size_t)i * N + j]);
        norm = std::max(norm, s);
    }
    int sq = 0;
    if (norm > 0.5) sq = (int)std::ceil(std::log2(norm / 0.5));
    const double scale = std::ldexp(1.0, -sq);
    std::vector<double> X(A);
    for (double& v : X) v *= scale;
    // N_6(X) = sum c_k X^k, D_6(X) = sum (-1)^k c_k X^k,
    // c_k = (2q-k)! q! / ((2q)! k! (q-k)!), q = 6.
    const int q = 6;
    std::vector<double> c(q + 1);
    c[0] = 1.0;
    for (int k = 1; k <= q; ++k) c[k] = c[k - 1] * (double)(q - k + 1) / (double)(k * (2 * q - k + 1));
    std::vector<double> Np((size_t)N * N, 0.0), Dp((size_t)N * N, 0.0), Pk((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i) Pk[(size_t)i * N + i] = 1.0;
    for (int k = 0; k <= q; ++k) {
        if (k > 0) mat_mul(Pk, X, Pk, N);
        const double sgn = (k & 1) ? -1.0 : 1.0;
        for (size_t t = 0; t < Pk.size(); ++t) {
            Np[t] += c[k] * Pk[t];
            Dp[t] += sgn * c[k] * Pk[t];
        }
    }
    if (!solve_in_place(Dp, Np, N)) return false;
    for (int s = 0; s < sq; ++s) mat_mul(Np, Np, Np, N);
    out.swap(Np);
    return true;
}

}  // namespace

int empc::set_thread_error(int s, const char* msg) {
    g_thread_error = msg;
    return s;
}

extern "C" {

void empc_config_default(empc_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->seed = 0x5EEDull;
    cfg->elite = 0;
    cfg->sigma = 0.1f;
    cfg->p_cross_256 = 128;
    cfg->p_mutate_256 = 128;
    cfg->gate = EMPC_GATE_PER_INPUT;
    cfg->precision = EMPC_FP32;
    cfg->refine_steps = 0;
    cfg->refine_lr = 0.0f;
    cfg->ckpt_every = 0;
    cfg->tile = 0;
    cfg->evaluator = EMPC_EVAL_ROLLOUT;
}

empc_status empc_create(const double* A, const double* B, const double* Q, const double* R,
                        const double* bounds, int n, int m, int horizon, int knots, int pop,
                        const empc_config* cfg_in, empc_handle* out) {
    if (!out) return fail(nullptr, EMPC_EINVAL, "out is NULL");
    *out = nullptr;
    {
        std::string msg;
        const empc_status vs =
            empc::validate_problem(A, B, Q, R, bounds, n, m, horizon, knots, pop, msg);
        if (vs != EMPC_OK) return fail(nullptr, vs, msg);
    }
    empc_config cfg;
    if (cfg_in) cfg = *cfg_in; else empc_config_default(&cfg);
    if (cfg.elite == 0) cfg.elite = std::max(1, pop / 16);
    if (cfg.elite < 1 || cfg.elite > pop || cfg.elite > 2048)
        return fail(nullptr, EMPC_EINVAL, "need 1 <= elite <= min(pop, 2048)");
    if (!(cfg.sigma >= 0.0f) || !std::isfinite(cfg.sigma))
        return fail(nullptr, EMPC_EINVAL, "sigma must be finite and >= 0");
    if (cfg.p_cross_256 < 0 || cfg.p_cross_256 > 256 || cfg.p_mutate_256 < 0 ||
        cfg.p_mutate_256 > 256)
        return fail(nullptr, EMPC_EINVAL, "probabilities *256 must lie in [0, 256]");
    if (cfg.gate < 0 || cfg.gate > 2) return fail(nullptr, EMPC_EINVAL, "bad gate mode");
    if (cfg.precision != EMPC_FP32 && cfg.precision != EMPC_BF16)
        return fail(nullptr, EMPC_EINVAL, "unknown precision");
    if (cfg.precision == EMPC_BF16 && !empc::rollout_bf16_supported(n, m, horizon))
        return fail(nullptr, EMPC_EUNSUPPORTED, "BF16 tensor-core rollout needs n <= 128, m <= 64");
    if (cfg.precision == EMPC_BF16 && cfg.refine_steps > 0)
        return fail(nullptr, EMPC_EUNSUPPORTED, "refinement runs in FP32 only");
    if (cfg.refine_steps < 0 || cfg.ckpt_every < 0 || !(cfg.refine_lr >= 0.0f))
        return fail(nullptr, EMPC_EINVAL, "need refine_steps >= 0, ckpt_every >= 0, refine_lr >= 0");
    if (cfg.refine_steps > 0 && n > 64)
        return fail(nullptr, EMPC_EUNSUPPORTED, "refinement needs n <= 64");
    if (cfg.evaluator != EMPC_EVAL_ROLLOUT && cfg.evaluator != EMPC_EVAL_CONDENSED)
        return fail(nullptr, EMPC_EINVAL, "unknown evaluator");
    if (cfg.evaluator == EMPC_EVAL_CONDENSED &&
        (cfg.precision != EMPC_FP32 || n > 64 || cfg.refine_steps > 0 ||
         !empc::condensed_supported(m * knots)))
        return fail(nullptr, EMPC_EUNSUPPORTED,
                    "the condensed evaluator needs FP32, n <= 64, m*p <= 832 and no refinement");
    empc::HostTables tb;
    {
        std::string msg;
        const empc_status ts = empc::build_tables(A, B, Q, R, bounds, n, m, horizon, knots, tb, msg);
        if (ts != EMPC_OK) return fail(nullptr, ts, msg);
    }
    empc_handle h = new empc_problem_s();
    h->n = n;
    h->m = m;
    h->T = horizon;
    h->p = knots;
    h->P = pop;
    h->E = cfg.elite;
    h->D = m * knots;
    h->cfg = cfg;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
#define EMPC_TRY(call)                                 \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) {                       \
            empc_status s_ = cuda_fail(nullptr, e_, #call); \
            free_handle(h);                            \
            return s_;                                 \
        }                                              \
    } while (0)
    EMPC_TRY(cudaStreamCreate(&h->own_stream));
    h->stream = h->own_stream;
    EMPC_TRY(cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking));
    EMPC_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    EMPC_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    h->ce = cfg.ckpt_every > 0 ? std::min(cfg.ckpt_every, horizon)
                               : std::max(1, (int)std::ceil(std::sqrt((double)horizon)));

    // host-side staging of the model in FP32 (built before the device is touched)

    const std::vector<float>& Dm = tb.D;
    const std::vector<float>& BT = tb.BT;
    const std::vector<float>& qd = tb.qd;
    const std::vector<float>& rd = tb.rd;
    const std::vector<float>& lo = tb.lo;
    const std::vector<float>& hi = tb.hi;
    const std::vector<float>& gram = tb.gram;
    const std::vector<KnotStep>& ks = tb.ks;
    const std::vector<double>& w0 = tb.w0;
    const std::vector<double>& w1 = tb.w1;
    const std::vector<int>& idx = tb.idx;
    if (cfg.refine_steps > 0) {
        if (cfg.refine_lr > 0.0f) {
            h->eta = cfg.refine_lr;
        } else {
            const double lmax = hessian_lambda_max(
                condensed_hessian(A, B, Q, R, n, m, horizon, knots, idx, w0, w1), m * knots);
            h->eta = lmax > 0.0 ? (float)(1.0 / (2.0 * lmax)) : 0.0f;
        }
    }

    const size_t D = (size_t)h->D;
    EMPC_TRY(dev_alloc(&h->D_, Dm.size()));
    EMPC_TRY(dev_alloc(&h->BT, BT.size()));
    EMPC_TRY(dev_alloc(&h->qdiag, n));
    EMPC_TRY(dev_alloc(&h->rdiag, m));
    EMPC_TRY(dev_alloc(&h->gram, gram.size()));
    EMPC_TRY(dev_alloc(&h->umin, m));
    EMPC_TRY(dev_alloc(&h->umax, m));
    EMPC_TRY(dev_alloc(&h->x0, n));
    EMPC_TRY(dev_alloc(&h->goal, n));
    EMPC_TRY(dev_alloc(&h->ktab, ks.size()));
    EMPC_TRY(dev_alloc(&h->pop[0], D * pop));
    EMPC_TRY(dev_alloc(&h->pop[1], D * pop));
    EMPC_TRY(dev_alloc(&h->cost, pop));
    EMPC_TRY(dev_alloc(&h->elite_idx, h->E));
    EMPC_TRY(dev_alloc(&h->elite_cost, h->E));
    EMPC_TRY(dev_alloc(&h->best_knots, D));
    EMPC_TRY(dev_alloc(&h->best_cost, 1));
    EMPC_TRY(dev_alloc(&h->gen, 1));
    EMPC_TRY(dev_alloc(&h->status, 1));
    EMPC_TRY(dev_alloc(&h->sigma_dev, 1));
    EMPC_TRY(dev_alloc(&h->inject, 2));
    if (tb.dense_r) EMPC_TRY(dev_alloc(&h->rmat, tb.rmat.size()));
    h->rotated = tb.rotated;
    if (tb.rotated) {
        h->Vt_h = tb.Vt;
        EMPC_TRY(dev_alloc(&h->Vt_dev, tb.Vt.size()));
        EMPC_TRY(dev_alloc(&h->ev_x0, n));
        EMPC_TRY(dev_alloc(&h->ev_goal, n));
    }
    EMPC_TRY(cudaMallocHost(reinterpret_cast<void**>(&h->stage),
                            sizeof(float) * (2 * (size_t)n + D + 2)));
    cudaStream_t st = h->stream;
    EMPC_TRY(cudaMemcpyAsync(h->D_, Dm.data(), sizeof(float) * Dm.size(), cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->BT, BT.data(), sizeof(float) * BT.size(), cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->qdiag, qd.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->rdiag, rd.data(), sizeof(float) * m, cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->gram, gram.data(), sizeof(float) * gram.size(), cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->umin, lo.data(), sizeof(float) * m, cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->umax, hi.data(), sizeof(float) * m, cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->ktab, ks.data(), sizeof(KnotStep) * ks.size(), cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemsetAsync(h->x0, 0, sizeof(float) * n, st));
    EMPC_TRY(cudaMemsetAsync(h->goal, 0, sizeof(float) * n, st));
    EMPC_TRY(cudaMemsetAsync(h->gen, 0, sizeof(uint32_t), st));
    EMPC_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    EMPC_TRY(cudaMemcpyAsync(h->sigma_dev, &h->cfg.sigma, sizeof(float), cudaMemcpyHostToDevice, st));
    EMPC_TRY(cudaMemcpyAsync(h->inject, h->inject_h, sizeof(h->inject_h), cudaMemcpyHostToDevice, st));
    if (tb.dense_r)
        EMPC_TRY(cudaMemcpyAsync(h->rmat, tb.rmat.data(), sizeof(float) * tb.rmat.size(),
                                 cudaMemcpyHostToDevice, st));
    if (tb.rotated)
        EMPC_TRY(cudaMemcpyAsync(h->Vt_dev, tb.Vt.data(), sizeof(double) * tb.Vt.size(),
                                 cudaMemcpyHostToDevice, st));
    h->Q_h.assign(Q, Q + (size_t)n * n);
    h->R_h.assign(R, R + (size_t)m * m);
    if (cfg.evaluator == EMPC_EVAL_CONDENSED) {
        const std::vector<double> H =
            condensed_hessian(A, B, Q, R, n, m, horizon, knots, idx, w0, w1);
        h->Dp = empc::condensed_pad(h->D);
        std::vector<float> Hf((size_t)h->Dp * h->Dp, 0.0f);
        for (int a = 0; a < h->D; ++a)
            for (int b = 0; b < h->D; ++b)
                Hf[(size_t)a * h->Dp + b] = (float)H[(size_t)a * h->D + b];
        EMPC_TRY(dev_alloc(&h->Hc, Hf.size()));
        EMPC_TRY(dev_alloc(&h->gvec, h->Dp));
        EMPC_TRY(dev_alloc(&h->c0, 1));
        EMPC_TRY(dev_alloc(&h->zero_knots, D));
        EMPC_TRY(cudaMemcpyAsync(h->Hc, Hf.data(), sizeof(float) * Hf.size(),
                                 cudaMemcpyHostToDevice, st));
        EMPC_TRY(cudaMemsetAsync(h->gvec, 0, sizeof(float) * h->Dp, st));
        EMPC_TRY(cudaMemsetAsync(h->c0, 0, sizeof(float), st));
        EMPC_TRY(cudaMemsetAsync(h->zero_knots, 0, sizeof(float) * D, st));
    }
    EMPC_TRY(cudaStreamSynchronize(st));
#undef EMPC_TRY
    empc_status s = autotune(h);
    if (s == EMPC_OK && h->n <= 64) {
        h->grad_nx = empc::warp_class_nx(n);
        s = autotune_grad(h);
        if (s == EMPC_OK && h->grad_wpc == 0 && cfg.refine_steps > 0)
            s = fail(h, EMPC_EUNSUPPORTED, "adjoint checkpoints do not fit in shared memory");
    }
    if (s != EMPC_OK) {
        g_thread_error = h->err;
        free_handle(h);
        return s;
    }
    *out = h;
    return EMPC_OK;
}

empc_status empc_solve(empc_handle h, const double* x0, const double* x_goal, int generations,
                       float* best_knots, float* best_cost) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!x0 || !x_goal || !best_knots || !best_cost)
        return fail(h, EMPC_EINVAL, "NULL x0, x_goal or output pointer");
    if (generations < 1) return fail(h, EMPC_EINVAL, "generations must be >= 1");
    if (!empc::all_finite(x0, h->n) || !empc::all_finite(x_goal, h->n))
        return fail(h, EMPC_EINVAL, "non-finite x0 or x_goal");
    float* st_in = h->stage;
    for (int i = 0; i < h->n; ++i) {
        st_in[i] = (float)rotate_row(h, x0, i);
        st_in[h->n + i] = (float)rotate_row(h, x_goal, i);
    }
    EMPC_CUDA(h, cudaMemcpyAsync(h->x0, st_in, sizeof(float) * h->n, cudaMemcpyHostToDevice, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(h->goal, st_in + h->n, sizeof(float) * h->n, cudaMemcpyHostToDevice, h->stream));
    EMPC_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    empc_status s = run_generations(h, generations);
    if (s != EMPC_OK) return s;
    float* st_out = h->stage + 2 * h->n;
    EMPC_CUDA(h, cudaMemcpyAsync(st_out, h->best_knots, sizeof(float) * h->D, cudaMemcpyDeviceToHost, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(st_out + h->D, h->best_cost, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(st_out + h->D + 1, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
    std::memcpy(best_knots, st_out, sizeof(float) * h->D);
    *best_cost = st_out[h->D];
    int status_bits;
    std::memcpy(&status_bits, st_out + h->D + 1, sizeof(int));
    if (status_bits & 2) return fail(h, EMPC_ETIMEOUT, "a bounded device wait gave up");
    if (status_bits & 1) return fail(h, EMPC_ENONFINITE, "best cost is not finite");
    return EMPC_OK;
}

empc_status empc_set_sigma(empc_handle h, float sigma) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!(sigma >= 0.0f) || !std::isfinite(sigma)) return fail(h, EMPC_EINVAL, "need sigma >= 0");
    h->sigma_now = sigma;
    EMPC_CUDA(h, cudaMemcpyAsync(h->sigma_dev, &h->sigma_now, sizeof(float),
                                 cudaMemcpyHostToDevice, h->stream));
    return EMPC_OK;
}

empc_status empc_inject_stall(empc_handle h, int step, double timeout_s) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (h->cfg.precision != EMPC_BF16)
        return fail(h, EMPC_EUNSUPPORTED, "stall injection is for the BF16 tensor-core rollout");
    if (step < -1 || !(timeout_s > 0.0) || !(timeout_s <= 60.0))
        return fail(h, EMPC_EINVAL, "need step >= -1 and 0 < timeout_s <= 60");
    EMPC_CUDA(h, cudaStreamSynchronize(h->stream));  // inject_h is not in use by a copy
    h->inject_h[0] = step;
    h->inject_h[1] = std::max(1, (int)std::lround(timeout_s * 1e6));
    EMPC_CUDA(h, cudaMemcpyAsync(h->inject, h->inject_h, sizeof(h->inject_h),
                                 cudaMemcpyHostToDevice, h->stream));
    EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
    return EMPC_OK;
}

empc_status empc_set_state_box(empc_handle h, const float* lo, const float* hi,
                               const float* rho, int flags) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (flags & ~(EMPC_BOX_CLAMP | EMPC_BOX_PENALTY))
        return fail(h, EMPC_EINVAL, "unknown state-box flags");
    if (flags && (h->cfg.precision != EMPC_FP32 || h->cfg.evaluator != EMPC_EVAL_ROLLOUT ||
                  h->cfg.refine_steps > 0))
        return fail(h, EMPC_EUNSUPPORTED,
                    "the state-box hook needs the FP32 rollout evaluator without refinement");
    if (flags && h->rotated)
        return fail(h, EMPC_EUNSUPPORTED,
                    "the state-box hook acts on the model's states; with a non-diagonal Q the "
                    "rollouts run in Q's eigenbasis");
    const int n = h->n;
    std::vector<float> t(3 * (size_t)n);
    if (flags) {
        for (int i = 0; i < n; ++i) {
            const float l = lo ? lo[i] : -INFINITY, u = hi ? hi[i] : INFINITY;
            const float r = rho ? rho[i] : 0.0f;
            if (!(l <= u) || l == INFINITY || u == -INFINITY)
                return fail(h, EMPC_EINVAL, "state box needs lo <= hi, lo < +inf, hi > -inf");
            if (!(r >= 0.0f) || !std::isfinite(r))
                return fail(h, EMPC_EINVAL, "state box needs finite rho >= 0");
            t[i] = l;
            t[n + i] = u;
            t[2 * n + i] = r;
        }
        if (!h->box) EMPC_CUDA(h, dev_alloc(&h->box, 3 * (size_t)n));
        EMPC_CUDA(h, cudaMemcpyAsync(h->box, t.data(), sizeof(float) * t.size(),
                                     cudaMemcpyHostToDevice, h->stream));
        EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    h->box_h = t;
    if (flags != h->box_mode) {  // the captured generations carry the mode
        EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
        h->box_mode = flags;
    }
    return EMPC_OK;
}

empc_status empc_set_disturbance(empc_handle h, const double* w_d) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    const int n = h->n;
    bool nonzero = false;
    if (w_d) {
        if (!empc::all_finite(w_d, (size_t)n)) return fail(h, EMPC_EINVAL, "non-finite w_d");
        for (int i = 0; i < n; ++i) nonzero = nonzero || w_d[i] != 0.0;
    }
    if (nonzero && h->cfg.precision != EMPC_FP32)
        return fail(h, EMPC_EUNSUPPORTED, "the disturbance needs the FP32 rollout");
    if (nonzero) {
        std::vector<float> t(n);
        for (int i = 0; i < n; ++i) t[i] = (float)rotate_row(h, w_d, i);
        if (!h->wd_dev) EMPC_CUDA(h, dev_alloc(&h->wd_dev, (size_t)n));
        EMPC_CUDA(h, cudaMemcpyAsync(h->wd_dev, t.data(), sizeof(float) * n,
                                     cudaMemcpyHostToDevice, h->stream));
        EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
        h->wd_h.assign(w_d, w_d + n);
    } else {
        h->wd_h.clear();
    }
    if (nonzero != h->has_wd) {  // the captured generations carry the pointer
        EMPC_CUDA(h, cudaStreamSynchronize(h->stream));
        for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
        h->graphs.clear();
        h->has_wd = nonzero;
    }
    return EMPC_OK;
}

empc_status empc_closed_loop(empc_handle h, const double* Ad, const double* Bd, const double* x0,
                             const double* x_goal, int steps, int generations, double sigma_min,
                             double sigma_dref, double* x_traj, double* u_traj,
                             double* actual_cost, double* ms_per_step) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!Ad || !Bd || !x0 || !x_goal || !actual_cost)
        return fail(h, EMPC_EINVAL, "NULL plant, state, goal or output pointer");
    if (steps < 1 || generations < 1) return fail(h, EMPC_EINVAL, "need steps, generations >= 1");
    if (!(sigma_min >= 0.0) || !(sigma_dref >= 0.0) || !std::isfinite(sigma_min) ||
        !std::isfinite(sigma_dref))
        return fail(h, EMPC_EINVAL, "need finite sigma_min, sigma_dref >= 0");
    const int n = h->n, m = h->m, p = h->p;
    if (!empc::all_finite(Ad, (size_t)n * n) || !empc::all_finite(Bd, (size_t)n * m))
        return fail(h, EMPC_EINVAL, "non-finite plant matrices");
    std::vector<double> x(x0, x0 + n), xn(n), u(m);
    std::vector<float> knots(h->D);
    auto stage = [&](const double* xs, const double* us) {
        double J = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                J += (x_goal[i] - xs[i]) * h->Q_h[(size_t)i * n + j] * (x_goal[j] - xs[j]);
        if (us)
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < m; ++j) J += us[i] * h->R_h[(size_t)i * m + j] * us[j];
        return J;
    };
    double total = 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < steps; ++k) {
        if (x_traj) std::copy(x.begin(), x.end(), x_traj + (size_t)k * n);
        if (sigma_dref > 0.0) {
            // exploration shrinks near the goal: sigma0 min(1, |x - g| / dref), at least sigma_min
            double d2 = 0.0;
            for (int i = 0; i < n; ++i) d2 += (x[i] - x_goal[i]) * (x[i] - x_goal[i]);
            const double sg = std::max(
                sigma_min, (double)h->cfg.sigma * std::min(1.0, std::sqrt(d2) / sigma_dref));
            const empc_status s = empc_set_sigma(h, (float)sg);
            if (s != EMPC_OK) return s;
        }
        float best = 0.0f;
        const empc_status s = empc_solve(h, x.data(), x_goal, generations, knots.data(), &best);
        if (s != EMPC_OK) return s;
        for (int i = 0; i < m; ++i) u[i] = (double)knots[(size_t)i * p];  // u* = U(i, 0)
        if (u_traj) std::copy(u.begin(), u.end(), u_traj + (size_t)k * m);
        total += stage(x.data(), u.data());
        for (int r = 0; r < n; ++r) {
            double v = 0.0;
            for (int c = 0; c < n; ++c) v += Ad[(size_t)r * n + c] * x[c];
            for (int c = 0; c < m; ++c) v += Bd[(size_t)r * m + c] * u[c];
            if (h->has_wd) v += h->wd_h[r];  // the model's disturbance acts on the plant
            if (h->box_mode & EMPC_BOX_CLAMP)  // the plant meets the same hard stop
                v = std::min(std::max(v, (double)h->box_h[r]), (double)h->box_h[n + r]);
            xn[r] = v;
        }
        x.swap(xn);
        if (!empc::all_finite(x.data(), n)) return fail(h, EMPC_ENONFINITE, "plant state diverged");
    }
    const auto t1 = std::chrono::steady_clock::now();
    if (sigma_dref > 0.0) {  // back to the configured sigma
        const empc_status s = empc_set_sigma(h, h->cfg.sigma);
        if (s != EMPC_OK) return s;
    }
    if (x_traj) std::copy(x.begin(), x.end(), x_traj + (size_t)steps * n);
    total += stage(x.data(), nullptr);
    *actual_cost = total;
    if (ms_per_step)
        *ms_per_step = std::chrono::duration<double, std::milli>(t1 - t0).count() / steps;
    return EMPC_OK;
}

empc_status empc_solve_device(empc_handle h, const float* dev_x0, const float* dev_goal,
                              int generations, float* dev_best_knots, float* dev_best_cost) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!dev_x0 || !dev_goal || !dev_best_knots || !dev_best_cost)
        return fail(h, EMPC_EINVAL, "NULL device pointer");
    if (generations < 1) return fail(h, EMPC_EINVAL, "generations must be >= 1");
    EMPC_CUDA(h, stage_targets(h, dev_x0, dev_goal, h->x0, h->goal));
    empc_status s = run_generations(h, generations);
    if (s != EMPC_OK) return s;
    EMPC_CUDA(h, cudaMemcpyAsync(dev_best_knots, h->best_knots, sizeof(float) * h->D, cudaMemcpyDeviceToDevice, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(dev_best_cost, h->best_cost, sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    return EMPC_OK;
}

empc_status empc_evaluate(empc_handle h, const float* dev_x0, const float* dev_goal,
                          const float* dev_pop, int count, float* dev_cost) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!dev_x0 || !dev_goal || !dev_pop || !dev_cost)
        return fail(h, EMPC_EINVAL, "NULL device pointer");
    if (count < 0) return fail(h, EMPC_EINVAL, "count must be >= 0");
    if (count == 0) return EMPC_OK;
    RolloutArgs a = base_args(h);
    a.x0 = dev_x0;
    a.goal = dev_goal;
    if (h->rotated) {
        EMPC_CUDA(h, stage_targets(h, dev_x0, dev_goal, h->ev_x0, h->ev_goal));
        a.x0 = h->ev_x0;
        a.goal = h->ev_goal;
    }
    a.mode = empc::kEval;
    a.P = count;
    a.pop_in = dev_pop;
    a.cost = dev_cost;
    a.gen = nullptr;
    EMPC_CUDA(h, empc::launch_rollout(a, h->shape, h->stream));
    return EMPC_OK;
}

empc_status empc_grad(empc_handle h, const float* dev_x0, const float* dev_goal,
                      const float* dev_pop, int count, float* dev_grad, float* dev_cost) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!dev_x0 || !dev_goal || !dev_pop || (!dev_grad && !dev_cost))
        return fail(h, EMPC_EINVAL, "NULL device pointer");
    if (count < 0) return fail(h, EMPC_EINVAL, "count must be >= 0");
    if (h->n > 64) return fail(h, EMPC_EUNSUPPORTED, "the adjoint kernel needs n <= 64");
    if (h->box_mode)
        return fail(h, EMPC_EUNSUPPORTED, "the adjoint follows the dynamics without the state box");
    if (h->grad_wpc <= 0)
        return fail(h, EMPC_EUNSUPPORTED, "adjoint checkpoints do not fit in shared memory");
    if (count == 0) return EMPC_OK;
    empc::GradArgs g = grad_args(h);
    g.x0 = dev_x0;
    g.goal = dev_goal;
    if (h->rotated) {
        EMPC_CUDA(h, stage_targets(h, dev_x0, dev_goal, h->ev_x0, h->ev_goal));
        g.x0 = h->ev_x0;
        g.goal = h->ev_goal;
    }
    g.pop_in = dev_pop;
    g.ld_in = count;
    g.count = count;
    g.grad = dev_grad;
    g.ld_grad = count;
    g.cost = dev_cost;
    g.steps = 0;
    EMPC_CUDA(h, empc::launch_grad(g, h->grad_nx, h->grad_cands, h->grad_wpc, h->stream));
    return EMPC_OK;
}

empc_status empc_get_state(empc_handle h, float* dev_pop, float* dev_cost, int* dev_elite) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!h->has_pop) return fail(h, EMPC_ESTATE, "no population yet (solve first)");
    if (dev_pop)
        EMPC_CUDA(h, cudaMemcpyAsync(dev_pop, h->pop[h->cur], sizeof(float) * h->D * h->P,
                                     cudaMemcpyDeviceToDevice, h->stream));
    if (dev_cost)
        EMPC_CUDA(h, cudaMemcpyAsync(dev_cost, h->cost, sizeof(float) * h->P,
                                     cudaMemcpyDeviceToDevice, h->stream));
    if (dev_elite)
        EMPC_CUDA(h, cudaMemcpyAsync(dev_elite, h->elite_idx, sizeof(int) * h->E,
                                     cudaMemcpyDeviceToDevice, h->stream));
    return EMPC_OK;
}

empc_status empc_set_state(empc_handle h, const float* dev_pop, const float* dev_cost,
                           const int* dev_elite) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    if (!dev_pop || !dev_cost || !dev_elite)
        return fail(h, EMPC_EINVAL, "population, costs and elites are all required");
    EMPC_CUDA(h, cudaMemcpyAsync(h->pop[h->cur], dev_pop, sizeof(float) * h->D * h->P,
                                 cudaMemcpyDeviceToDevice, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(h->cost, dev_cost, sizeof(float) * h->P,
                                 cudaMemcpyDeviceToDevice, h->stream));
    EMPC_CUDA(h, cudaMemcpyAsync(h->elite_idx, dev_elite, sizeof(int) * h->E,
                                 cudaMemcpyDeviceToDevice, h->stream));
    h->has_pop = true;
    return EMPC_OK;
}

empc_status empc_reset(empc_handle h) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    h->has_pop = false;
    return EMPC_OK;
}

empc_status empc_set_stream(empc_handle h, void* stream) {
    if (!h) return fail(nullptr, EMPC_EINVAL, "NULL handle");
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    return EMPC_OK;
}

empc_status empc_get_info(empc_handle h, empc_info* info) {
    if (!h || !info) return fail(h, EMPC_EINVAL, "NULL handle or info");
    std::memset(info, 0, sizeof(*info));
    info->n = h->n;
    info->m = h->m;
    info->horizon = h->T;
    info->knots = h->p;
    info->pop = h->P;
    info->elite = h->E;
    info->generation = h->gen_host;
    info->tile_nx = h->shape.nx;
    info->tile_rows = h->shape.rows;
    info->tile_cands = h->shape.cands;
    info->tile_groups = h->shape.groups;
    info->tile_kind = h->shape.kind;
    info->threads_per_cta = empc::rollout_threads(h->shape, h->n);
    info->smem_bytes = (int)empc::rollout_smem_bytes(h->shape, h->n, h->m, h->p, h->T);
    const int ptile = empc::rollout_cands_per_cta(h->shape, h->n);
    info->ctas = (h->P + ptile - 1) / ptile;
    info->tuned_us = h->tuned_us;
    info->refine_lr = h->eta;
    info->ckpt_every = h->ce;
    return EMPC_OK;
}

empc_status empc_time_generation(empc_handle h, int reps, float* breed_us, float* rollout_us,
                                 float* select_us) {
    if (!h || !breed_us || !rollout_us || !select_us || reps < 1)
        return fail(h, EMPC_EINVAL, "need a handle, reps >= 1 and three outputs");
    if (!h->has_pop) return fail(h, EMPC_ESTATE, "no population yet (solve first)");
    cudaEvent_t ev[4];
    for (auto& e : ev) EMPC_CUDA(h, cudaEventCreate(&e));
    double t_breed = 0.0, t_roll = 0.0, t_sel = 0.0;
    empc_status s = EMPC_OK;
    for (int r = 0; r < reps && s == EMPC_OK; ++r) {
        RolloutArgs a = base_args(h);
        a.mode = empc::kWarm;
        a.pop_in = h->pop[h->cur];
        a.pop_out = h->pop[h->cur ^ 1];
        a.cost = h->cost;
        a.elite_idx = h->elite_idx;
        cudaError_t e = cudaEventRecord(ev[0], h->stream);
        if (e == cudaSuccess) e = empc::launch_breed(a, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
        a.mode = empc::kEval;
        a.pop_in = h->pop[h->cur ^ 1];
        if (e == cudaSuccess) e = evaluate_population(h, a, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
        if (e == cudaSuccess)
            e = empc::launch_select(h->cost, h->P, h->E, h->pop[h->cur ^ 1], h->D, h->elite_idx,
                                    h->elite_cost, h->best_knots, h->best_cost, h->gen,
                                    h->status, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
        if (e != cudaSuccess) {
            s = cuda_fail(h, e, "empc_time_generation");
            break;
        }
        float b_ms = 0, r_ms = 0, s_ms = 0;
        cudaEventElapsedTime(&b_ms, ev[0], ev[1]);
        cudaEventElapsedTime(&r_ms, ev[1], ev[2]);
        cudaEventElapsedTime(&s_ms, ev[2], ev[3]);
        t_breed += b_ms;
        t_roll += r_ms;
        t_sel += s_ms;
        h->cur ^= 1;
        h->gen_host += 1;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (s != EMPC_OK) return s;
    *breed_us = (float)(1000.0 * t_breed / reps);
    *rollout_us = (float)(1000.0 * t_roll / reps);
    *select_us = (float)(1000.0 * t_sel / reps);
    return EMPC_OK;
}

void empc_destroy(empc_handle h) { free_handle(h); }

const char* empc_last_error(empc_handle h) {
    return h ? h->err.c_str() : g_thread_error.c_str();
}

empc_status empc_discretize_zoh(const double* Ac, const double* Bc, int n, int m, double dt,
                                double* Ad, double* Bd) {
    if (!Ac || !Bc || !Ad || !Bd) return fail(nullptr, EMPC_EINVAL, "NULL pointer");
    if (n < 1 || m < 0 || !std::isfinite(dt) || dt < 0.0)
        return fail(nullptr, EMPC_EINVAL, "need n >= 1, m >= 0, finite dt >= 0");
    if (!empc::all_finite(Ac, (size_t)n * n) || !empc::all_finite(Bc, (size_t)n * m))
        return fail(nullptr, EMPC_EINVAL, "non-finite Ac or Bc");
    const int N = n + m;
    std::vector<double> M((size_t)N * N, 0.0), E;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) M[(size_t)i * N + j] = Ac[(size_t)i * n + j] * dt;
        for (int j = 0; j < m; ++j) M[(size_t)i * N + n + j] = Bc[(size_t)i * m + j] * dt;
    }
    if (!expm_pade6(M, N, E)) return fail(nullptr, EMPC_EINVAL, "singular Pade denominator");
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) Ad[(size_t)i * n + j] = E[(size_t)i * N + j];
        for (int j = 0; j < m; ++j) Bd[(size_t)i * m + j] = E[(size_t)i * N + n + j];
    }
    return EMPC_OK;
}

}  // extern "C"
