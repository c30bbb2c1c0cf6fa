// empc_evaluate_noalloc: population costs without any device allocation.
//
// Who needs it: callers that must not allocate GPU memory while they run,
// for example a real-time control loop that re-solves MPC every few
// milliseconds (cudaMalloc / cudaFree can synchronize the device and take an
// unbounded time), or a host process whose GPU memory is reserved up front
// by another framework's caching allocator.  The handle API (empc_create)
// allocates its tables once per problem; this entry point instead keeps the
// per-problem tables the cost kernel reads (D = A - I, B transposed, the Q
// and R weights, the knot table and the input-cost Gram weights, and for a
// non-diagonal Q the rotation into its eigenbasis with the rotated start and
// goal) in one file-scope device array of fixed size, and allocates nothing,
// neither on the device nor on the host.
//
// Every call writes the part of the array it uses before its kernels read
// it (one copy of exactly the floats the call's sizes need), so nothing
// carries over between calls.  All calls in the process share the array: two
// calls whose work overlaps on the GPU (different streams, or different host
// threads without ordering) race on it and give wrong costs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/empc.h"
#include "empc_internal.h"
#include "host_tables.h"

namespace {

// Size limits of the shared table array (include/empc.h).  The rollout's
// shared memory grows with n, m, p and T, and its largest case, n = m = p =
// 64 and T = 1024, fits the one-warp tile of the warp-synchronous family
// (about 117 KB), so every size within the limits has a tile.
constexpr int kMaxN = 64;
constexpr int kMaxM = 64;
constexpr int kMaxT = 1024;
constexpr int kMaxKnots = 64;

// Floats of the array: D, BT, the Q and R weights, the Gram, the knot table
// (4 floats a step), a dense R, the FP64 rotation (2 floats per entry), the
// rotated start and goal, and alignment padding.
constexpr int kScratchFloats = kMaxN * kMaxN + kMaxM * kMaxN + kMaxN + kMaxM + 2 * kMaxKnots +
                               4 * kMaxT + kMaxM * kMaxM + 2 * kMaxN * kMaxN + 2 * kMaxN + 32;

// The fixed scratch: 24,992 floats (about 98 KiB) on every device that loads
// the library, held until the process exits.
static __device__ __align__(256) float g_eval_tables[kScratchFloats];

// Host staging of one call (guarded by g_mutex): the packed tables, then
// FP64 knot weights, knot indices and the table builder's scratch.
std::mutex g_mutex;
alignas(16) float g_host_tables[kScratchFloats];
double g_w0[kMaxT], g_w1[kMaxT];
int g_idx[kMaxT];
double g_work[3 * kMaxN * kMaxN + kMaxM * kMaxM + 2 * kMaxKnots];
constexpr int kMaxDevices = 64;
float* g_dev_tables[kMaxDevices] = {nullptr};

empc_status reject(empc_status s, const char* msg) {
    return (empc_status)empc::set_thread_error(s, msg);
}

// Float offsets of one call's tables inside the array (16-byte aligned
// where a vector type or a double is read).
struct Layout {
    int D, BT, qd, rd, gram, ks, rmat, Vt, zx, zg, used;
    Layout(int n, int m, int T, int p, bool dense_r, bool rotated) {
        auto up4 = [](int v) { return (v + 3) / 4 * 4; };
        D = 0;
        BT = up4(D + n * n);
        qd = up4(BT + m * n);
        rd = up4(qd + n);
        gram = up4(rd + m);
        ks = up4(gram + 2 * p);
        rmat = up4(ks + 4 * T);
        Vt = up4(rmat + (dense_r ? m * m : 0));
        zx = up4(Vt + (rotated ? 2 * n * n : 0));
        zg = up4(zx + (rotated ? n : 0));
        used = zg + (rotated ? n : 0);
    }
};
static_assert(kScratchFloats == 24992, "the size stated in include/empc.h");

}  // namespace

extern "C" empc_status empc_evaluate_noalloc(const double* A, const double* B, const double* Q,
                                             const double* R, int n, int m, int horizon,
                                             int knots, const float* dev_x0,
                                             const float* dev_goal, const float* dev_pop,
                                             int count, float* dev_cost, void* stream) {
    if (!A || !B || !Q || !R || !dev_x0 || !dev_goal || !dev_pop || !dev_cost)
        return reject(EMPC_EINVAL, "empc_evaluate_noalloc: NULL pointer");
    if (n < 1 || n > kMaxN || m < 1 || m > kMaxM || horizon < 1 || horizon > kMaxT ||
        knots < 1 || knots > horizon || knots > kMaxKnots || count < 0)
        return reject(EMPC_EINVAL,
                      "empc_evaluate_noalloc: sizes beyond its fixed tables (n <= 64, m <= 64, "
                      "horizon <= 1024, knots <= 64, 1 <= knots <= horizon, count >= 0); use "
                      "empc_create");
    if (!empc::all_finite(A, (size_t)n * n) || !empc::all_finite(B, (size_t)n * m) ||
        !empc::all_finite(Q, (size_t)n * n) || !empc::all_finite(R, (size_t)m * m))
        return reject(EMPC_EINVAL, "empc_evaluate_noalloc: non-finite model or weight");
    for (int i = 0; i < n; ++i)
        if (Q[(size_t)i * n + i] < 0.0) return reject(EMPC_EINVAL, "Q must be >= 0");
    for (int i = 0; i < m; ++i)
        if (R[(size_t)i * m + i] < 0.0) return reject(EMPC_EINVAL, "R must be >= 0");
    if (count == 0) return EMPC_OK;

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return reject(EMPC_ECUDA, "empc_evaluate_noalloc: no CUDA device");
    // First call on a device: look up the array's device address with that
    // device current (the host-side symbol is only a stand-in).
    if (!g_dev_tables[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_eval_tables);
        if (e != cudaSuccess) return reject(EMPC_ECUDA, cudaGetErrorString(e));
        g_dev_tables[dev] = static_cast<float*>(p);
    }
    float* dt = g_dev_tables[dev];

    // The tables, built by the same code as empc_create's, written straight
    // into the host staging array at this call's offsets.
    const bool dense_r = empc::has_off_diagonal(R, m);
    const bool rotated = empc::has_off_diagonal(Q, n);
    const Layout L(n, m, horizon, knots, dense_r, rotated);
    float* h = g_host_tables;
    const empc::TableOut o{h + L.D,
                           h + L.BT,
                           h + L.qd,
                           h + L.rd,
                           nullptr,
                           nullptr,
                           h + L.gram,
                           reinterpret_cast<empc::KnotStep*>(h + L.ks),
                           h + L.rmat,
                           reinterpret_cast<double*>(h + L.Vt),
                           g_w0,
                           g_w1,
                           g_idx,
                           g_work};
    bool rot = false, dr = false;
    const char* msg = "";
    const empc_status ts = empc::fill_tables(A, B, Q, R, nullptr, n, m, horizon, knots, o, &rot,
                                             &dr, &msg);
    if (ts != EMPC_OK) return reject(ts, msg);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Pageable source: the copy has been staged when the call returns, so the
    // host tables may be rewritten by the next call.
    cudaError_t e = cudaMemcpyAsync(dt, h, sizeof(float) * L.used, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return reject(EMPC_ECUDA, cudaGetErrorString(e));

    empc::RolloutArgs a{};
    a.D = dt + L.D;
    a.BT = dt + L.BT;
    a.qdiag = dt + L.qd;
    a.rdiag = dt + L.rd;
    a.rmat = dense_r ? dt + L.rmat : nullptr;
    a.gram = dt + L.gram;
    a.ktab = reinterpret_cast<const empc::KnotStep*>(dt + L.ks);
    a.x0 = dev_x0;
    a.goal = dev_goal;
    if (rotated) {  // start and goal into Q's eigenbasis, inside the array
        e = empc::launch_rotate(reinterpret_cast<const double*>(dt + L.Vt), dev_x0, dev_goal,
                                dt + L.zx, dt + L.zg, n, st);
        if (e != cudaSuccess) return reject(EMPC_ECUDA, cudaGetErrorString(e));
        a.x0 = dt + L.zx;
        a.goal = dt + L.zg;
    }
    a.n = n;
    a.m = m;
    a.T = horizon;
    a.p = knots;
    a.P = count;
    a.mode = empc::kEval;
    a.pop_in = dev_pop;
    a.cost = dev_cost;
    a.gen = nullptr;
    // Tile: warp-synchronous, 2 candidates per thread, 4 warps per CTA when it
    // fits, else the first shape that fits.
    empc::TileShape shapes[64];
    const int ns = std::min(empc::rollout_shapes(n, shapes, 64), 64);
    int pick = -1;
    for (int i = 0; i < ns && pick < 0; ++i)
        if (shapes[i].kind == 1 && shapes[i].cands == 2 && shapes[i].groups == 4 &&
            empc::rollout_shape_supported(shapes[i], n, m, knots, horizon))
            pick = i;
    for (int i = 0; i < ns && pick < 0; ++i)
        if (empc::rollout_shape_supported(shapes[i], n, m, knots, horizon)) pick = i;
    if (pick < 0) return reject(EMPC_EUNSUPPORTED, "empc_evaluate_noalloc: no rollout tile fits");
    e = empc::launch_rollout(a, shapes[pick], st);
    if (e != cudaSuccess) return reject(EMPC_ECUDA, cudaGetErrorString(e));
    return EMPC_OK;
}
