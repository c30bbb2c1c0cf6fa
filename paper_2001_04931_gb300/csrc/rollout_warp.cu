// Fused breed + knot expansion + rollout + cost, warp-synchronous family.
//
// Each warp owns whole candidates for the whole horizon: lane (cgl, rg) keeps
// rows rg*R .. rg*R+R-1 of D = A_d - I in registers and updates them for C
// candidates of candidate group cgl (32/NRG groups per warp).  The warp's
// state tile lives in its own slice of shared memory and a step needs only a
// warp barrier, so warps never wait for one another.  The horizon loop, knot
// forces and breeding are shared with the block family (rollout_common.cuh);
// the per-candidate cost is reduced over the NRG lanes of its group by a
// butterfly in a fixed order.
#include <cuda_runtime.h>

#include "rollout_common.cuh"

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

template <int NX, int NRG, int C>
__global__ void rollout_warp_kernel(const RolloutArgs a) {
    constexpr int R = (NX + NRG - 1) / NRG;
    constexpr int XR = NRG * R;
    constexpr int CGW = 32 / NRG;
    constexpr int CPW = CGW * C;
    constexpr int XS = (CPW + 3) / 4 * 4;
    extern __shared__ __align__(16) float smem[];
    const int m = a.m, p = a.p, T = a.T;
    const int D = m * p;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = lane % NRG, cgl = lane / NRG;
    const int per_warp = round_up(2 * XR * XS + D * XS + 2 * XS, 4);
    float* BTs = smem;
    KnotStep* ks = reinterpret_cast<KnotStep*>(smem + round_up(m * XR, 4));
    float* W = smem + round_up(m * XR, 4) + 4 * T + warp * per_warp;
    float* X = W;
    float* Us = W + 2 * XR * XS;
    int* par = reinterpret_cast<int*>(Us + D * XS);
    const int c0 = (blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
    const uint32_t gen = a.gen ? *a.gen : 0u;

    for (int i = threadIdx.x; i < m * XR; i += blockDim.x) {
        const int row = i % XR, col = i / XR;
        BTs[i] = row < a.n ? a.BT[col * a.n + row] : 0.0f;
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) ks[k] = a.ktab[k];
    __syncthreads();
    if (c0 >= a.P) return;  // no block barrier follows

    for (int i = lane; i < 2 * XR * XS; i += 32) {
        const int k = (i / XS) % XR;
        X[i] = (i < XR * XS && k < a.n) ? a.x0[k] : 0.0f;
    }
    fill_knots<true>(a, Us, XS, par, c0, CPW, gen, lane, 32);  // ends with a warp barrier

    float d[R][NX], qd[R], gl[R], xo[R][C], jsum[C];
    load_rows<NX, R, C>(a, rg * R, d, qd, gl, xo);
    horizon_loop<NX, R, C, true>(a, d, X, XR, XS, BTs, XR, Us, ks, rg * R, cgl * C, xo, qd, gl,
                                 jsum);

    // each lane adds the input cost of inputs rg, rg + NRG, ...; then a
    // butterfly over the group's NRG lanes
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float J = jsum[c] + input_cost_part(a, Us, XS, cgl * C + c, rg, NRG);
#pragma unroll
        for (int off = NRG / 2; off > 0; off >>= 1) J += __shfl_xor_sync(0xffffffffu, J, off);
        const int cand = c0 + cgl * C + c;
        if (rg == 0 && cand < a.P) a.cost[cand] = finite_or_inf(J);
    }
}

template <int NX, int C>
cudaError_t launch_shape(const RolloutArgs& a, int wpc, cudaStream_t st) {
    constexpr int NRG = NX == 4 ? 2 : NX == 8 ? 4 : NX <= 24 ? 8 : NX <= 48 ? 16 : 32;
    constexpr int CPW = (32 / NRG) * C;
    TileShape s{1, NX, (NX + NRG - 1) / NRG, C, wpc};
    const size_t smem = rollout_smem_bytes(s, a.n, a.m, a.p, a.T);
    auto kern = rollout_warp_kernel<NX, NRG, C>;
    static int smem_cap = 48 * 1024;
    if ((int)smem > smem_cap) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        smem_cap = (int)smem;
    }
    const int per_cta = wpc * CPW;
    const int grid = (a.P + per_cta - 1) / per_cta;
    kern<<<grid, 32 * wpc, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NX, int C>
int max_threads_of() {
    constexpr int NRG = NX == 4 ? 2 : NX == 8 ? 4 : NX <= 24 ? 8 : NX <= 48 ? 16 : 32;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, rollout_warp_kernel<NX, NRG, C>) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

#define EMPC_WARP_NX_CASES(X) X(4) X(8) X(16) X(24) X(32) X(40) X(48) X(56) X(64)

}  // namespace

cudaError_t launch_rollout_warp(const RolloutArgs& a, const TileShape& s, cudaStream_t st) {
#define EMPC_CASE(NXV)                                                   \
    if (s.nx == NXV) {                                                   \
        if (s.cands == 1) return launch_shape<NXV, 1>(a, s.groups, st);  \
        if (s.cands == 2) return launch_shape<NXV, 2>(a, s.groups, st);  \
        if (s.cands == 4) return launch_shape<NXV, 4>(a, s.groups, st);  \
    }
    EMPC_WARP_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return cudaErrorInvalidConfiguration;
}

int warp_max_threads(const TileShape& s) {
#define EMPC_CASE(NXV)                                        \
    if (s.nx == NXV) {                                        \
        if (s.cands == 1) return max_threads_of<NXV, 1>();    \
        if (s.cands == 2) return max_threads_of<NXV, 2>();    \
        if (s.cands == 4) return max_threads_of<NXV, 4>();    \
    }
    EMPC_WARP_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return 0;
}

}  // namespace empc
