// Warp-synchronous rollout of one warp's candidates (shared by the
// single-problem kernel in rollout_warp.cu and the batched persistent kernel
// in batched.cu).
//
// Each warp owns whole candidates for the whole horizon: lane (cgl, rg) keeps
// rows rg*R .. rg*R+R-1 of D = A_d - I in registers (as pairs of adjacent
// columns) and updates them for C candidates of candidate group cgl (32/NRG
// groups per warp).  The warp's state tile lives in its own slice of shared
// memory, pair-interleaved so one vector load returns rows (k, k+1) of
// consecutive candidates, and a step needs only a warp barrier.  The sum over
// k runs as two partial sums with paired FMAs (fma.rn.f32x2).  The
// per-candidate cost is reduced over the NRG lanes of its group by a
// butterfly in a fixed order.
#pragma once
#include "rollout_common.cuh"

namespace empc {

// Row groups per candidate group (warp_nrg as a compile-time function).
__host__ __device__ constexpr int nrg_of(int nx) {
    return nx == 4 ? 2 : nx == 8 ? 4 : nx <= 24 ? 8 : nx <= 48 ? 16 : 32;
}

// The horizon loop of rollout_common.cuh's horizon_loop on the
// pair-interleaved state tile, with paired FMAs and two partial sums per
// output (state_product_pairs).  BOX compiles in the hooks staged at bx
// (stage_box): the disturbance w_d, then the state box.
template <int NX, int R, int C, bool BOX>
__device__ __forceinline__ void horizon_loop_pairs(const RolloutArgs& a,
                                                   const float2 (&d2)[R][NX / 2], float* X,
                                                   int xrows, int xs, const float* BTs, int ldb,
                                                   const float* Us, const KnotStep* ks,
                                                   int row0, int col0, float (&xo)[R][C],
                                                   const float (&qd)[R], const float (&gl)[R],
                                                   float (&jsum)[C], const float* bx) {
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
        float2 acc[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c)
                acc[r][c] = make_float2(fmaf(st.w1, bub[r][c], st.w0 * bua[r][c]), 0.0f);
        state_product_pairs<NX, R, C>(d2, X + buf * xrows * xs + 2 * col0, xs, acc);
        float* Xn = X + (buf ^ 1) * xrows * xs;
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float sum = acc[r][c].x + acc[r][c].y;
                float xn = xo[r][c] + sum;
                if constexpr (BOX) {
                    xn = xn + bx[3 * xrows + row0 + r];  // w_d
                    xn = box_hook(bx, xrows, row0 + r, a.box_mode, xn, jblk[c]);
                }
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

// Shared-memory floats of one warp's slice for a problem with D = m p knots.
template <int NX, int C>
__host__ __device__ constexpr int warp_slice_floats(int D) {
    return round_up(2 * nrg_of(NX) * ((NX + nrg_of(NX) - 1) / nrg_of(NX)) *
                            ((((32 / nrg_of(NX)) * C) + 3) / 4 * 4) +
                        (D + 2) * ((((32 / nrg_of(NX)) * C) + 3) / 4 * 4),
                    4);
}

// One warp breeds (or loads) and rolls out candidates c0 .. c0+CPW-1 of
// problem `a` and writes their costs.  W is the warp's shared-memory slice;
// BTs ([m][XR], rows past n zero) and ks (knot table) are staged by the CTA,
// and so is D when Ds is given ([n][ds] with ds >= NX, columns past n zero;
// otherwise the rows are read from global memory).  bx, if given, holds the
// hooks staged as [4][XR] (stage_box) and selects the hooked loop.
// Reads the population, the elites and the generation counter only after
// pdl_wait_primary(); COHERENT reads them through L2 (persistent kernels).
template <int NX, int C, bool COHERENT = false>
__device__ __forceinline__ void warp_tile(const RolloutArgs& a, int c0, float* W,
                                          const float* BTs, const KnotStep* ks,
                                          const float* Ds = nullptr, int ds = 0,
                                          const float* bx = nullptr,
                                          const float* x0s = nullptr) {
    constexpr int NRG = nrg_of(NX);
    constexpr int R = (NX + NRG - 1) / NRG;
    constexpr int XR = NRG * R;
    constexpr int CGW = 32 / NRG;
    constexpr int CPW = CGW * C;
    constexpr int XS = (CPW + 3) / 4 * 4;
    constexpr int KP = NX / 2;
    const int D = a.m * a.p;
    const int lane = threadIdx.x & 31;
    const int rg = lane % NRG, cgl = lane / NRG;
    float* X = W;
    float* Us = W + 2 * XR * XS;
    int* par = reinterpret_cast<int*>(Us + D * XS);

    // pair-interleaved rows; x0 from the CTA's staged copy when given
    for (int i = lane; i < 2 * XR * XS; i += 32) {
        const int j = i % (XR * XS);
        const int k = 2 * (j / (2 * XS)) + (j & 1);
        X[i] = (i < XR * XS && k < a.n) ? (x0s ? x0s[k] : a.x0[k]) : 0.0f;
    }
    float qd[R], gl[R], xo[R][C], jsum[C];
    float2 d2[R][KP];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = rg * R + r;
        const bool ok = row < a.n;
        if (Ds) {
#pragma unroll
            for (int kp = 0; kp < KP; ++kp)
                d2[r][kp] = ok ? *reinterpret_cast<const float2*>(Ds + row * ds + 2 * kp)
                               : make_float2(0.0f, 0.0f);
        } else {
#pragma unroll
            for (int kp = 0; kp < KP; ++kp) {
                const int k = 2 * kp;
                d2[r][kp] = make_float2((ok && k < a.n) ? a.D[row * a.n + k] : 0.0f,
                                        (ok && k + 1 < a.n) ? a.D[row * a.n + k + 1] : 0.0f);
            }
        }
        qd[r] = ok ? a.qdiag[row] : 0.0f;
        gl[r] = ok ? a.goal[row] : 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) xo[r][c] = ok ? a.x0[row] : 0.0f;
    }
    // everything above reads only the model; the population, the elites and
    // the generation counter come from the previous kernels
    pdl_wait_primary();
    const uint32_t gen = a.gen ? *(volatile const uint32_t*)a.gen : 0u;
    fill_knots<true, COHERENT>(a, Us, XS, par, c0, CPW, gen, lane, 32);  // ends with a warp barrier
    if (bx)
        horizon_loop_pairs<NX, R, C, true>(a, d2, X, XR, XS, BTs, XR, Us, ks, rg * R, cgl * C,
                                           xo, qd, gl, jsum, bx);
    else
        horizon_loop_pairs<NX, R, C, false>(a, d2, X, XR, XS, BTs, XR, Us, ks, rg * R, cgl * C,
                                            xo, qd, gl, jsum, bx);

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

}  // namespace empc
