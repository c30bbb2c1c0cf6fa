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

// Row groups per candidate group (warp_nrg as a compile-time function).
__host__ __device__ constexpr int nrg_of(int nx) {
    return nx == 4 ? 2 : nx == 8 ? 4 : nx <= 24 ? 8 : nx <= 48 ? 16 : 32;
}

// The horizon loop of rollout_common.cuh's horizon_loop on the
// pair-interleaved state tile, with paired FMAs and four partial sums per
// output (state_product_pairs).
template <int NX, int R, int C>
__device__ __forceinline__ void horizon_loop_pairs(const RolloutArgs& a,
                                                   const float2 (&d2)[R][NX / 2], float* X,
                                                   int xrows, int xs, const float* BTs, int ldb,
                                                   const float* Us, const KnotStep* ks,
                                                   int row0, int col0, float (&xo)[R][C],
                                                   const float (&qd)[R], const float (&gl)[R],
                                                   float (&jsum)[C]) {
    float bua[R][C], bub[R][C];
    int seg = -1;
    float jtot[C], jblk[C];
#pragma unroll
    for (int c = 0; c < C; ++c) jtot[c] = jblk[c] = 0.0f;
    int buf = 0;
    for (int k = 0; k < a.T; ++k) {
        const KnotStep st = ks[k];
        if (st.idx1 != seg) {
            if (st.idx1 == seg + 1 && seg >= 0) {
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < C; ++c) bua[r][c] = bub[r][c];
            } else {
                knot_force<R, C>(BTs, ldb, Us, xs, a.m, a.p, st.idx1, row0, col0, bua);
            }
            if (st.idx1 + 1 < a.p) {
                knot_force<R, C>(BTs, ldb, Us, xs, a.m, a.p, st.idx1 + 1, row0, col0, bub);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < C; ++c) bub[r][c] = 0.0f;
            }
            seg = st.idx1;
        }
        float2 accA[R][C], accB[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                accA[r][c] = make_float2(fmaf(st.w1, bub[r][c], st.w0 * bua[r][c]), 0.0f);
                accB[r][c] = make_float2(0.0f, 0.0f);
            }
        state_product_pairs<NX, R, C>(d2, X + buf * xrows * xs + 2 * col0, xs, accA, accB);
        float* Xn = X + (buf ^ 1) * xrows * xs;
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float sum = (accA[r][c].x + accB[r][c].x) + (accA[r][c].y + accB[r][c].y);
                const float xn = xo[r][c] + sum;
                xo[r][c] = xn;
                const float e = xn - gl[r];
                jblk[c] = fmaf(qd[r] * e, e, jblk[c]);
                Xn[pair_index(row0 + r, col0 + c, xs)] = xn;
            }
        }
        if ((k & 15) == 15) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                jtot[c] += jblk[c];
                jblk[c] = 0.0f;
            }
        }
        __syncwarp();
        buf ^= 1;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) jsum[c] = jtot[c] + jblk[c];
}

template <int NX, int C>
__global__ void rollout_warp_kernel(const RolloutArgs a) {
    constexpr int NRG = nrg_of(NX);
    constexpr int R = (NX + NRG - 1) / NRG;
    constexpr int XR = NRG * R;
    constexpr int CGW = 32 / NRG;
    constexpr int CPW = CGW * C;
    constexpr int XS = (CPW + 3) / 4 * 4;
    constexpr int KP = NX / 2;
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
    const int c0 = a.cand_begin + (blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
    pdl_launch_dependents();

    for (int i = threadIdx.x; i < m * XR; i += blockDim.x) {
        const int row = i % XR, col = i / XR;
        BTs[i] = row < a.n ? a.BT[col * a.n + row] : 0.0f;
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) ks[k] = a.ktab[k];
    __syncthreads();
    if (c0 >= a.P) return;  // no block barrier follows

    for (int i = lane; i < 2 * XR * XS; i += 32) {  // pair-interleaved rows
        const int j = i % (XR * XS);
        const int k = 2 * (j / (2 * XS)) + (j & 1);
        X[i] = (i < XR * XS && k < a.n) ? a.x0[k] : 0.0f;
    }
    float qd[R], gl[R], xo[R][C], jsum[C];
    float2 d2[R][KP];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = rg * R + r;
        const bool ok = row < a.n;
#pragma unroll
        for (int kp = 0; kp < KP; ++kp) {
            const int k = 2 * kp;
            d2[r][kp] = make_float2((ok && k < a.n) ? a.D[row * a.n + k] : 0.0f,
                                    (ok && k + 1 < a.n) ? a.D[row * a.n + k + 1] : 0.0f);
        }
        qd[r] = ok ? a.qdiag[row] : 0.0f;
        gl[r] = ok ? a.goal[row] : 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) xo[r][c] = ok ? a.x0[row] : 0.0f;
    }
    // everything above reads only the model; the population, the elites and
    // the generation counter come from the previous kernels
    pdl_wait_primary();
    const uint32_t gen = a.gen ? *a.gen : 0u;
    fill_knots<true>(a, Us, XS, par, c0, CPW, gen, lane, 32);  // ends with a warp barrier
    horizon_loop_pairs<NX, R, C>(a, d2, X, XR, XS, BTs, XR, Us, ks, rg * R, cgl * C, xo, qd, gl,
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
    constexpr int NRG = nrg_of(NX);
    constexpr int CPW = (32 / NRG) * C;
    TileShape s{1, NX, (NX + NRG - 1) / NRG, C, wpc};
    const size_t smem = rollout_smem_bytes(s, a.n, a.m, a.p, a.T);
    auto kern = rollout_warp_kernel<NX, C>;
    static int smem_cap = 48 * 1024;
    if ((int)smem > smem_cap) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        smem_cap = (int)smem;
    }
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
