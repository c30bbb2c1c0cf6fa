// Fused breed + knot expansion + rollout + cost, warp-synchronous family:
// the single-problem kernel (one warp tile per warp, rollout_warp.cuh) and its
// launch and shape queries.
#include <cuda_runtime.h>

#include "rollout_warp.cuh"

namespace empc {

// Row groups per candidate group for each compiled state dimension.
int warp_nrg(int nx) {
    switch (nx) {
        case 4: return 2;
        case 8: return 4;
        case 16: return 8;
        case 24: return 8;
        case 32: return 16;
        case 40: return 16;
        case 48: return 16;
        case 56: return 32;
        case 64: return 32;
        default: return 0;
    }
}

namespace {

template <int NX, int C>
__global__ void rollout_warp_kernel(const RolloutArgs a) {
    constexpr int NRG = nrg_of(NX);
    constexpr int XR = NRG * ((NX + NRG - 1) / NRG);
    constexpr int CPW = (32 / NRG) * C;
    extern __shared__ __align__(16) float smem[];
    const int m = a.m, T = a.T;
    const int warp = threadIdx.x >> 5;
    constexpr int DS = NX + 2;  // D row stride: 8-byte pairs, rows spread over the banks
    float* BTs = smem;
    KnotStep* ks = reinterpret_cast<KnotStep*>(smem + round_up(m * XR, 4));
    float* Ds = smem + round_up(m * XR, 4) + 4 * T;
    float* Bx = Ds + round_up(a.n * DS, 4);
    float* X0 = Bx + round_up(4 * XR, 4);
    float* W = X0 + round_up(XR, 4) + warp * warp_slice_floats<NX, C>(m * a.p);
    const int c0 = a.cand_begin + (blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
    pdl_launch_dependents();
    // the model tables, staged with batched loads (they do not depend on the
    // previous kernel, so under programmatic dependent launch this overlaps it)
    const int tid = threadIdx.x, nthr = blockDim.x;
    batched_fill(BTs, m * XR, tid, nthr, [&](int i) {
        const int row = i % XR, col = i / XR;
        return row < a.n ? a.BT[col * a.n + row] : 0.0f;
    });
    batched_fill(reinterpret_cast<float*>(ks), 4 * T, tid, nthr,
                 [&](int i) { return reinterpret_cast<const float*>(a.ktab)[i]; });
    batched_fill(Ds, a.n * DS, tid, nthr, [&](int i) {
        const int r = i / DS, k = i - r * DS;
        return k < a.n ? a.D[r * a.n + k] : 0.0f;
    });
    batched_fill(X0, XR, tid, nthr, [&](int i) { return i < a.n ? a.x0[i] : 0.0f; });
    const bool hooks = has_hooks(a);
    if (hooks) stage_box(a, Bx, XR, tid, nthr);
    __syncthreads();
    if (c0 >= a.P) return;  // no block barrier follows
    warp_tile<NX, C>(a, c0, W, BTs, ks, Ds, DS, hooks ? Bx : nullptr, X0);
}

template <int NX, int C>
cudaError_t launch_shape(const RolloutArgs& a, int wpc, cudaStream_t st) {
    constexpr int NRG = nrg_of(NX);
    constexpr int CPW = (32 / NRG) * C;
    TileShape s{1, NX, (NX + NRG - 1) / NRG, C, wpc};
    const size_t smem = rollout_smem_bytes(s, a.n, a.m, a.p, a.T);
    auto kern = rollout_warp_kernel<NX, C>;
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    const int per_cta = wpc * CPW;
    const int grid = (a.P - a.cand_begin + per_cta - 1) / per_cta;
    if (grid <= 0) return cudaSuccess;
    return launch_kernel(kern, dim3(grid), dim3(32 * wpc), smem, st, a.pdl != 0, a);
}

template <int NX, int C>
int max_threads_of() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, rollout_warp_kernel<NX, C>) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

#define EMPC_WARP_NX_CASES(X) X(4) X(8) X(16) X(24) X(32) X(40) X(48) X(56) X(64)

}  // namespace

cudaError_t launch_rollout_warp(const RolloutArgs& a, const TileShape& s, cudaStream_t st) {
#define EMPC_CASE(NXV)                                                       \
    if (s.nx == NXV) {                                                       \
        if (s.cands == 1) return launch_shape<NXV, 1>(a, s.groups, st);      \
        if (s.cands == 2) return launch_shape<NXV, 2>(a, s.groups, st);      \
        if (s.cands == 4) return launch_shape<NXV, 4>(a, s.groups, st);      \
    }
    EMPC_WARP_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return cudaErrorInvalidConfiguration;
}

int warp_max_threads(const TileShape& s) {
#define EMPC_CASE(NXV)                                              \
    if (s.nx == NXV) {                                              \
        if (s.cands == 1) return max_threads_of<NXV, 1>();          \
        if (s.cands == 2) return max_threads_of<NXV, 2>();          \
        if (s.cands == 4) return max_threads_of<NXV, 4>();          \
    }
    EMPC_WARP_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return 0;
}

}  // namespace empc
