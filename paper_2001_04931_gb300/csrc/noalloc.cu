// empc_evaluate_noalloc: population costs without any device allocation.
//
// Who needs it: callers that must not allocate GPU memory while they run,
// for example a real-time control loop that re-solves MPC every few
// milliseconds (cudaMalloc / cudaFree can synchronize the device and take an
// unbounded time), or a host process whose GPU memory is reserved up front
// by another framework's caching allocator.  The handle API (empc_create)
// allocates its tables once per problem; this entry point instead keeps the
// per-problem tables the cost kernel reads (D = A - I, B transposed, the Q
// and R diagonals, the knot table and the input-cost Gram weights) in one
// file-scope device array of fixed size, and allocates nothing.
//
// Every call rewrites the part of the array it uses before its kernel reads
// it, so nothing carries over between calls.  All calls in the process share
// the array: two calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and give wrong costs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/empc.h"
#include "empc_internal.h"

namespace {

// Size limits of the shared table array (see include/empc.h).
constexpr int kMaxN = 64;
constexpr int kMaxM = 64;
constexpr int kMaxT = 1024;
constexpr int kMaxKnots = 64;

// Float offsets of each table inside the array.
constexpr int kOffD = 0;                             // [n][n]
constexpr int kOffBT = kOffD + kMaxN * kMaxN;        // [m][n]
constexpr int kOffQ = kOffBT + kMaxM * kMaxN;        // [n]
constexpr int kOffR = kOffQ + kMaxN;                 // [m]
constexpr int kOffGram = kOffR + kMaxM;              // [2 p]
constexpr int kOffKnots = kOffGram + 2 * kMaxKnots;  // KnotStep[T] (4 floats each)
constexpr int kScratchFloats = kOffKnots + 4 * kMaxT;

// The fixed scratch: 12,544 floats (49 KiB) on every device that loads the
// library, held until the process exits.
static __device__ __align__(256) float g_eval_tables[kScratchFloats];

// Host staging for one call, and the per-device address of g_eval_tables.
std::mutex g_mutex;
float g_host_tables[kScratchFloats];
constexpr int kMaxDevices = 64;
float* g_dev_tables[kMaxDevices] = {nullptr};

}  // namespace

extern "C" empc_status empc_evaluate_noalloc(const double* A, const double* B, const double* Q,
                                             const double* R, int n, int m, int horizon,
                                             int knots, const float* dev_x0,
                                             const float* dev_goal, const float* dev_pop,
                                             int count, float* dev_cost, void* stream) {
    using empc::set_thread_error;
    if (!A || !B || !Q || !R || !dev_x0 || !dev_goal || !dev_pop || !dev_cost)
        return (empc_status)set_thread_error(EMPC_EINVAL, "empc_evaluate_noalloc: NULL pointer");
    if (n < 1 || n > kMaxN || m < 1 || m > kMaxM || horizon < 1 || horizon > kMaxT ||
        knots < 1 || knots > horizon || knots > kMaxKnots || count < 0)
        return (empc_status)set_thread_error(
            EMPC_EINVAL,
            "empc_evaluate_noalloc: sizes beyond its fixed tables (n <= 64, m <= 64, "
            "horizon <= 1024, knots <= 64, 1 <= knots <= horizon); use empc_create");
    for (size_t i = 0; i < (size_t)n * n; ++i)
        if (!std::isfinite(A[i]) || !std::isfinite(Q[i]))
            return (empc_status)set_thread_error(EMPC_EINVAL, "non-finite A or Q");
    for (size_t i = 0; i < (size_t)n * m; ++i)
        if (!std::isfinite(B[i])) return (empc_status)set_thread_error(EMPC_EINVAL, "non-finite B");
    for (size_t i = 0; i < (size_t)m * m; ++i)
        if (!std::isfinite(R[i])) return (empc_status)set_thread_error(EMPC_EINVAL, "non-finite R");
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j && Q[(size_t)i * n + j] != 0.0)
                return (empc_status)set_thread_error(EMPC_EUNSUPPORTED, "Q must be diagonal");
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            if (i != j && R[(size_t)i * m + j] != 0.0)
                return (empc_status)set_thread_error(EMPC_EUNSUPPORTED, "R must be diagonal");
    if (count == 0) return EMPC_OK;

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return (empc_status)set_thread_error(EMPC_ECUDA, "empc_evaluate_noalloc: no CUDA device");
    // First call on a device: look up the array's device address with that
    // device current (the host-side symbol is only a stand-in).
    if (!g_dev_tables[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_eval_tables) != cudaSuccess)
            return (empc_status)set_thread_error(EMPC_ECUDA, "cudaGetSymbolAddress failed");
        g_dev_tables[dev] = static_cast<float*>(p);
    }
    float* dt = g_dev_tables[dev];

    // Host-side tables, the same construction as empc_create's.
    float* h = g_host_tables;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j)
            h[kOffD + i * n + j] = (float)(A[(size_t)i * n + j] - (i == j ? 1.0 : 0.0));
        h[kOffQ + i] = (float)Q[(size_t)i * n + i];
        for (int j = 0; j < m; ++j) h[kOffBT + j * n + i] = (float)B[(size_t)i * m + j];
    }
    for (int i = 0; i < m; ++i) h[kOffR + i] = (float)R[(size_t)i * m + i];
    double wd[kMaxKnots] = {0.0}, wo[kMaxKnots] = {0.0};
    empc::KnotStep* ks = reinterpret_cast<empc::KnotStep*>(h + kOffKnots);
    const long den = horizon > 1 ? horizon - 1 : 1;
    for (int k = 0; k < horizon; ++k) {
        long a = 0, num = 0;
        if (knots > 1 && horizon > 1) {
            a = (long)k * (knots - 1) / den;
            if (a > knots - 2) a = knots - 2;
            num = (long)k * (knots - 1) - a * den;
        }
        const double w1 = (double)num / (double)den, w0 = (double)(den - num) / (double)den;
        ks[k].idx1 = (int)a;
        ks[k].w0 = (float)w0;
        ks[k].w1 = (float)w1;
        ks[k].pad = 0;
        wd[a] += w0 * w0;
        if (knots > 1) {
            wd[a + 1] += w1 * w1;
            wo[a] += w0 * w1;
        }
    }
    for (int j = 0; j < knots; ++j) {
        h[kOffGram + j] = (float)wd[j];
        h[kOffGram + knots + j] = (float)wo[j];
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Pageable source: the copy has been staged when the call returns, so the
    // host tables may be rewritten by the next call.
    if (cudaMemcpyAsync(dt, h, sizeof(float) * kScratchFloats, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return (empc_status)set_thread_error(EMPC_ECUDA, "table copy failed");

    empc::RolloutArgs a{};
    a.D = dt + kOffD;
    a.BT = dt + kOffBT;
    a.qdiag = dt + kOffQ;
    a.rdiag = dt + kOffR;
    a.gram = dt + kOffGram;
    a.ktab = reinterpret_cast<const empc::KnotStep*>(dt + kOffKnots);
    a.x0 = dev_x0;
    a.goal = dev_goal;
    a.n = n;
    a.m = m;
    a.T = horizon;
    a.p = knots;
    a.P = count;
    a.mode = empc::kEval;
    a.pop_in = dev_pop;
    a.cost = dev_cost;
    a.gen = nullptr;
    // Default tile: warp-synchronous, 2 candidates per thread, 4 warps per CTA.
    empc::TileShape shapes[64];
    const int ns = empc::rollout_shapes(n, shapes, 64);
    for (int i = 0; i < ns && i < 64; ++i) {
        const empc::TileShape& s = shapes[i];
        if (s.kind == 1 && s.cands == 2 && s.groups == 4 &&
            empc::rollout_shape_supported(s, n, m, knots, horizon))
            return empc::launch_rollout(a, s, st) == cudaSuccess ? EMPC_OK : EMPC_ECUDA;
    }
    for (int i = 0; i < ns && i < 64; ++i)
        if (empc::rollout_shape_supported(shapes[i], n, m, knots, horizon))
            return empc::launch_rollout(a, shapes[i], st) == cudaSuccess ? EMPC_OK : EMPC_ECUDA;
    return EMPC_EUNSUPPORTED;
}
