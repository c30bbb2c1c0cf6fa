// Population costs from the condensed quadratic form of the parameterized
// problem (Sec. IV-B, IV-E): for linear dynamics and a quadratic cost the
// whole rollout collapses, per candidate U (the m*p knots), to
//   J(U) = U' H U + g' U + c0,
// with H the Hessian of the cost in the knots (fixed by the model, the
// weights and the knot table), g = dJ/dU at U = 0 and c0 = J(0) (both fixed
// by the start state and the goal).  Evaluating a population is one dense
// product Y = H U over the knots, then J_c = sum_i U_ic (Y_ic + g_i) + c0:
// 2 D^2 + 2 D flops per candidate (D = m p) instead of the rollout's
// T (2 n^2 + 6 n).  The rollout remains the general evaluator (it also
// admits non-quadratic costs and in-rollout effects); this one is exact only
// for the linear-quadratic problem.
//
// Tiling: a CTA owns a tile of candidates; their knots (all D rows) sit in
// shared memory, and the threads form a TI x TC grid with an MI x MC register
// tile of Y for a 64-row block at a time.  H streams through shared memory in
// 32-row slabs, the next slab loaded into registers while the current one is
// used; H is symmetric, so rows of H read along the block are the needed
// column slice.  The partial costs of the TI threads sharing candidates are
// summed in a fixed order.
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

constexpr int kJC = 32;  // rows of H staged per slab

template <int TI, int TC, int MI, int MC>
__global__ void __launch_bounds__(TI * TC) condensed_kernel(const CondArgs a) {
    constexpr int NT = TI * TC;   // threads
    constexpr int NCT = TC * MC;  // candidates per CTA
    constexpr int IB = TI * MI;   // rows of Y (= columns of the H slab) per block
    constexpr int SLAB4 = kJC * IB / 4;              // float4s per slab
    constexpr int PER = (SLAB4 + NT - 1) / NT;       // float4s per thread
    static_assert(IB == 64 && MC == 4 && MI % 2 == 0 && SLAB4 % NT == 0, "tile");
    extern __shared__ __align__(16) float smem[];
    const int Dp = a.Dp;
    float* Us = smem;                  // [Dp][NCT]
    float* Hs = smem + Dp * NCT;       // [kJC][IB]
    float* red = Hs + kJC * IB;        // [TI][NCT]
    const int tid = threadIdx.x;
    const int ti = tid / TC, tc = tid % TC;
    const int c0 = blockIdx.x * NCT;
    pdl_launch_dependents();
    pdl_wait_primary();  // the knots come from the breeding kernel
    for (int idx = tid; idx < Dp * NCT; idx += NT) {
        const int j = idx / NCT, c = idx % NCT;
        Us[idx] = (j < a.D && c0 + c < a.P) ? __ldcg(a.pop + (size_t)j * a.P + c0 + c) : 0.0f;
    }
    float jp[MC];
#pragma unroll
    for (int c = 0; c < MC; ++c) jp[c] = 0.0f;
    const int nslab = Dp / kJC;
    // the H slab [jb, jb + kJC) x [ib, ib + IB): H is symmetric, so these rows
    // of H read along the i-block are the needed column slice
    auto fetch = [&](int ib, int s, float4 (&pre)[PER]) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int f = tid + r * NT;
            const int row = f / (IB / 4), col4 = f % (IB / 4);
            pre[r] = __ldg(reinterpret_cast<const float4*>(a.H + (size_t)(s * kJC + row) * Dp +
                                                           ib + col4 * 4));
        }
    };
    for (int ib = 0; ib < Dp; ib += IB) {
        float y[MI][MC];
#pragma unroll
        for (int i = 0; i < MI; ++i)
#pragma unroll
            for (int c = 0; c < MC; ++c) y[i][c] = 0.0f;
        float4 pre[PER];
        fetch(ib, 0, pre);
        for (int s = 0; s < nslab; ++s) {
            __syncthreads();  // the previous slab has been consumed
#pragma unroll
            for (int r = 0; r < PER; ++r) reinterpret_cast<float4*>(Hs)[tid + r * NT] = pre[r];
            __syncthreads();
            if (s + 1 < nslab) fetch(ib, s + 1, pre);  // in flight during the products
#pragma unroll 8
            for (int jj = 0; jj < kJC; ++jj) {
                float hv[MI];
#pragma unroll
                for (int i = 0; i < MI; i += 2) {
                    const float2 t = *reinterpret_cast<const float2*>(Hs + jj * IB + ti * MI + i);
                    hv[i] = t.x;
                    hv[i + 1] = t.y;
                }
                const float4 u =
                    *reinterpret_cast<const float4*>(Us + (s * kJC + jj) * NCT + tc * MC);
                const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int i = 0; i < MI; ++i)
#pragma unroll
                    for (int c = 0; c < MC; ++c) y[i][c] = fmaf(hv[i], uv[c], y[i][c]);
            }
        }
#pragma unroll
        for (int i = 0; i < MI; ++i) {
            const int row = ib + ti * MI + i;
            const float gi = a.g[row];
            const float4 u = *reinterpret_cast<const float4*>(Us + row * NCT + tc * MC);
            const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int c = 0; c < MC; ++c) jp[c] = fmaf(uv[c], y[i][c] + gi, jp[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < MC; ++c) red[ti * NCT + tc * MC + c] = jp[c];
    __syncthreads();
    for (int c = tid; c < NCT; c += NT) {
        float J = *a.c0;
        for (int t = 0; t < TI; ++t) J += red[t * NCT + c];
        if (c0 + c < a.P) a.cost[c0 + c] = finite_or_inf(J);
    }
}

template <int TI, int TC, int MI, int MC>
cudaError_t launch_tile(const CondArgs& a, cudaStream_t st, bool pdl) {
    constexpr int NCT = TC * MC;
    const size_t smem = sizeof(float) * ((size_t)a.Dp * NCT + kJC * TI * MI + TI * NCT);
    auto kern = condensed_kernel<TI, TC, MI, MC>;
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    const int grid = (a.P + NCT - 1) / NCT;
    return launch_kernel(kern, dim3(grid), dim3(TI * TC), smem, st, pdl, a);
}

}  // namespace

int condensed_pad(int D) { return (D + 63) / 64 * 64; }

bool condensed_supported(int D) {
    // knots of 64 candidates, an H slab and the reduction rows in shared memory
    return D >= 1 && sizeof(float) * ((size_t)condensed_pad(D) * 64 + kJC * 64 + 16 * 64) <=
                         227u * 1024u;
}

cudaError_t launch_condensed(const CondArgs& a, cudaStream_t st, bool pdl) {
    if (!condensed_supported(a.D) || a.Dp != condensed_pad(a.D)) return cudaErrorInvalidValue;
    if (a.P <= 0) return cudaSuccess;
    // 64 candidates per CTA when that still fills the GPU, else 32
    if ((a.P + 63) / 64 >= 152) return launch_tile<16, 16, 4, 4>(a, st, pdl);
    return launch_tile<32, 8, 2, 4>(a, st, pdl);
}

}  // namespace empc
