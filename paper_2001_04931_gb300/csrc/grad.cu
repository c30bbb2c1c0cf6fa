// Adjoint gradient of the EMPC cost with respect to the knots, with state
// checkpointing, and projected-gradient refinement of the elites.  (No
// counterpart in the paper, whose optimizer is gradient-free.)
//
// For J(U) = sum_{k=0}^{T-1} (x_{k+1}-g)' Q (x_{k+1}-g) + u_k' R u_k and
// x_{k+1} = x_k + D x_k + B u_k (D = A_d - I), the adjoint is
//   lambda_T = 2 Q e_T,  lambda_k = lambda_{k+1} + D' lambda_{k+1} + 2 Q e_k,
//   dJ/du_k = B' lambda_{k+1} + 2 R u_k,        e_k = x_k - g,
// and with u_k = w0_k U_idx1(k) + w1_k U_idx1(k)+1 (Sec. IV-C)
//   dJ/dU(i, a) = (B' Lambda_a)_i + 2 r_i sum_b W_ab U(i, b),
//   Lambda_a    = sum_k w_{k a} lambda_{k+1}      (W: Gram of the weights).
//
// Layout follows the warp-synchronous rollout: lane (cgl, rg) owns rows
// rg*R .. rg*R+R-1 of C candidates.  The forward pass stores x every `ce`
// steps (checkpoints, O(T/ce) state vectors).  The backward pass walks the
// segments in reverse: it recomputes the segment's states from its checkpoint
// (D rows in registers), then swaps D' rows into the same registers and runs
// the adjoint recursion through the segment (O(ce) state vectors), so shared
// memory holds O(T/ce + ce) states per candidate instead of O(T).
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

template <int NX, int NRG>
struct GradGeom {
    static constexpr int R = (NX + NRG - 1) / NRG;
    static constexpr int XR = NRG * R;
    static constexpr int CGW = 32 / NRG;
};

// Per-warp shared-memory slice (floats).
struct GradWarpLayout {
    int x, lam, ck, sb, us, lamacc, g, total;
    __host__ __device__ GradWarpLayout(int xr, int xs, int nseg, int ce, int D, int p) {
        x = 0;                              // X[2][xr][xs]
        lam = x + 2 * xr * xs;              // L[2][xr][xs]
        ck = lam + 2 * xr * xs;             // CK[nseg + 1][xr][xs]
        sb = ck + (nseg + 1) * xr * xs;     // SB[ce][xr][xs]
        us = sb + ce * xr * xs;             // U[D][xs]
        lamacc = us + D * xs;               // LAM[p][xr][xs]
        g = lamacc + p * xr * xs;           // G[D][xs]
        total = round_up(g + D * xs, 4);
    }
};

template <int NX, int R>
__device__ __forceinline__ void load_d_rows(const float* Ds, int row0, float (&d)[R][NX]) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NX; ++k) d[r][k] = Ds[(row0 + r) * (NX + 1) + k];
}

template <int NX, int R>
__device__ __forceinline__ void load_d_cols(const float* Ds, int row0, float (&d)[R][NX]) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < NX; ++k) d[r][k] = Ds[k * (NX + 1) + row0 + r];
}

// Knot-force pair for step k: refresh bua/bub when the knot segment changes.
template <int R, int C>
__device__ __forceinline__ void knot_pair(const GradArgs& a, const float* BTs, int ldb,
                                          const float* Us, int xs, int row0, int col0,
                                          const KnotStep& st, int& seg, float (&bua)[R][C],
                                          float (&bub)[R][C]) {
    if (st.idx1 == seg) return;
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

// One forward step from state tile Xin to Xout (own rows): x + D x + B u_k,
// then + w_d (wdr: this thread's rows of the disturbance, zero without one).
template <int NX, int R, int C>
__device__ __forceinline__ void fwd_step(const float (&d)[R][NX], const float* Xin,
                                         float* Xout, int xs, int row0, int col0,
                                         const KnotStep& st, const float (&bua)[R][C],
                                         const float (&bub)[R][C], const float (&wdr)[R],
                                         float (&xo)[R][C]) {
    float acc[R][C];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = fmaf(st.w1, bub[r][c], st.w0 * bua[r][c]);
    state_product<NX, R, C>(d, Xin + col0, xs, acc);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float xn[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            xn[c] = (xo[r][c] + acc[r][c]) + wdr[r];
            xo[r][c] = xn[c];
        }
        store_vec<C>(Xout + (row0 + r) * xs + col0, xn);
    }
}

template <int NX, int NRG, int C>
__global__ void grad_warp_kernel(const GradArgs a) {
    using Gm = GradGeom<NX, NRG>;
    constexpr int R = Gm::R, XR = Gm::XR, CPW = Gm::CGW * C;
    constexpr int XS = (CPW + 3) / 4 * 4;
    extern __shared__ __align__(16) float smem[];
    const int m = a.m, p = a.p, T = a.T, n = a.n;
    const int D = m * p;
    const int ce = a.ce;
    const int nseg = (T + ce - 1) / ce;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = lane % NRG, cgl = lane / NRG;
    const int row0 = rg * R, col0 = cgl * C;

    float* BTs = smem;                                   // [m][XR]
    float* Ds = BTs + round_up(m * XR, 4);               // [NX][NX+1]
    KnotStep* ks = reinterpret_cast<KnotStep*>(Ds + round_up(NX * (NX + 1), 4));
    const GradWarpLayout WL(XR, XS, nseg, ce, D, p);
    float* W = reinterpret_cast<float*>(ks + T) + warp * WL.total;
    float* X = W + WL.x;
    float* Lm = W + WL.lam;
    float* CK = W + WL.ck;
    float* SB = W + WL.sb;
    float* Us = W + WL.us;
    float* LA = W + WL.lamacc;
    float* G = W + WL.g;
    const int c0 = (blockIdx.x * (blockDim.x >> 5) + warp) * CPW;

    for (int i = threadIdx.x; i < m * XR; i += blockDim.x) {
        const int row = i % XR, col = i / XR;
        BTs[i] = row < n ? a.BT[col * n + row] : 0.0f;
    }
    for (int i = threadIdx.x; i < NX * (NX + 1); i += blockDim.x) {
        const int r = i / (NX + 1), k = i % (NX + 1);
        Ds[i] = (r < n && k < n) ? a.D[r * n + k] : 0.0f;
    }
    for (int k = threadIdx.x; k < T; k += blockDim.x) ks[k] = a.ktab[k];
    __syncthreads();
    if (c0 >= a.count) return;  // no block barrier follows

    // knots of this warp's candidates
    for (int i = lane; i < D * CPW; i += 32) {
        const int q = i / CPW, t = i % CPW;
        const int c = c0 + t;
        float v = 0.0f;
        if (c < a.count) {
            const int col = a.index ? a.index[c] : c;
            v = a.pop_in[(size_t)q * a.ld_in + col];
        }
        Us[q * XS + t] = v;
    }
    __syncwarp();

    float qd[R], gl[R], x0r[R], wdr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = row0 + r;
        wdr[r] = (row < n && a.wd) ? a.wd[row] : 0.0f;
        qd[r] = row < n ? a.qdiag[row] : 0.0f;
        gl[r] = row < n ? a.goal[row] : 0.0f;
        x0r[r] = row < n ? a.x0[row] : 0.0f;
    }
    float d[R][NX];
    const int passes = a.steps > 0 ? a.steps + 1 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        const bool last = pass == passes - 1;
        const bool need_grad = !(a.steps > 0 && last);
        // ---------------- forward: states, checkpoints, cost
        load_d_rows<NX, R>(Ds, row0, d);
        float xo[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                xo[r][c] = x0r[r];
                X[(row0 + r) * XS + col0 + c] = x0r[r];
                CK[(row0 + r) * XS + col0 + c] = x0r[r];
            }
        for (int i = lane; i < 2 * XR * XS; i += 32) {  // rows past n stay zero
            const int row = (i / XS) % XR;
            if (row >= n) X[i] = 0.0f;
        }
        __syncwarp();
        float bua[R][C], bub[R][C], jtot[C], jblk[C];
        int seg = -1;
#pragma unroll
        for (int c = 0; c < C; ++c) jtot[c] = jblk[c] = 0.0f;
        int buf = 0;
        for (int k = 0; k < T; ++k) {
            const KnotStep st = ks[k];
            knot_pair<R, C>(a, BTs, XR, Us, XS, row0, col0, st, seg, bua, bub);
            fwd_step<NX, R, C>(d, X + buf * XR * XS, X + (buf ^ 1) * XR * XS, XS, row0, col0,
                               st, bua, bub, wdr, xo);
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float e = xo[r][c] - gl[r];
                    jblk[c] = fmaf(qd[r] * e, e, jblk[c]);
                }
            if ((k & 15) == 15) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    jtot[c] += jblk[c];
                    jblk[c] = 0.0f;
                }
            }
            if ((k + 1) % ce == 0 && k + 1 < T) {
                float* ckp = CK + ((k + 1) / ce) * XR * XS;
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < C; ++c) ckp[(row0 + r) * XS + col0 + c] = xo[r][c];
            }
            __syncwarp();
            buf ^= 1;
        }
        // cost: butterfly over the group's lanes, as the rollout kernels do
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float J = jtot[c] + jblk[c] + input_cost_part(a, Us, XS, col0 + c, rg, NRG);
#pragma unroll
            for (int off = NRG / 2; off > 0; off >>= 1) J += __shfl_xor_sync(0xffffffffu, J, off);
            const int cand = c0 + col0 + c;
            if (rg == 0 && cand < a.count && last && a.cost)
                a.cost[cand] = finite_or_inf(J);
        }
        if (!need_grad) break;

        // ---------------- backward: lambda_T = 2 Q e_T
        float lam[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                lam[r][c] = 2.0f * qd[r] * (xo[r][c] - gl[r]);
                Lm[(row0 + r) * XS + col0 + c] = lam[r][c];
            }
        for (int i = lane; i < 2 * XR * XS; i += 32) {
            const int row = (i / XS) % XR;
            if (row >= n) Lm[i] = 0.0f;
        }
        for (int i = lane; i < p * XR * XS; i += 32) LA[i] = 0.0f;
        __syncwarp();
        int lb = 0;
        float la_lo[R][C], la_hi[R][C];
        int aseg = -1;
        for (int s = nseg - 1; s >= 0; --s) {
            const int k0 = s * ce, k1 = min(T, k0 + ce);
            // recompute x_{k0+1} .. x_{k1} from checkpoint s into SB
            load_d_rows<NX, R>(Ds, row0, d);
            float xr[R][C];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < C; ++c) xr[r][c] = CK[s * XR * XS + (row0 + r) * XS + col0 + c];
            for (int i = lane; i < (k1 - k0) * XR * XS; i += 32) {
                const int row = (i / XS) % XR;
                if (row >= n) SB[i] = 0.0f;
            }
            int rseg = -1;
            for (int k = k0; k < k1; ++k) {
                const KnotStep st = ks[k];
                knot_pair<R, C>(a, BTs, XR, Us, XS, row0, col0, st, rseg, bua, bub);
                const float* xin = (k == k0) ? CK + s * XR * XS : SB + (k - k0 - 1) * XR * XS;
                fwd_step<NX, R, C>(d, xin, SB + (k - k0) * XR * XS, XS, row0, col0, st, bua, bub, wdr, xr);
                __syncwarp();
            }
            // adjoint through the segment with D' rows
            load_d_cols<NX, R>(Ds, row0, d);
            for (int k = k1 - 1; k >= k0; --k) {
                const KnotStep st = ks[k];
                if (st.idx1 != aseg) {  // flush the knot accumulators of the previous segment
                    if (aseg >= 0) {
#pragma unroll
                        for (int r = 0; r < R; ++r)
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                LA[(aseg * XR + row0 + r) * XS + col0 + c] += la_lo[r][c];
                                if (aseg + 1 < p)
                                    LA[((aseg + 1) * XR + row0 + r) * XS + col0 + c] += la_hi[r][c];
                            }
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < C; ++c) la_lo[r][c] = la_hi[r][c] = 0.0f;
                    aseg = st.idx1;
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        la_lo[r][c] = fmaf(st.w0, lam[r][c], la_lo[r][c]);
                        la_hi[r][c] = fmaf(st.w1, lam[r][c], la_hi[r][c]);
                    }
                if (k >= 1) {
                    float acc[R][C];
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int c = 0; c < C; ++c) acc[r][c] = 0.0f;
                    state_product<NX, R, C>(d, Lm + lb * XR * XS + col0, XS, acc);
                    const float* xk = (k == k0) ? CK + s * XR * XS : SB + (k - k0 - 1) * XR * XS;
                    float* Ln = Lm + (lb ^ 1) * XR * XS;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        float ln[C];
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            const float e = xk[(row0 + r) * XS + col0 + c] - gl[r];
                            ln[c] = lam[r][c] + acc[r][c] + 2.0f * qd[r] * e;
                            lam[r][c] = ln[c];
                        }
                        store_vec<C>(Ln + (row0 + r) * XS + col0, ln);
                    }
                    __syncwarp();
                    lb ^= 1;
                }
            }
        }
        if (aseg >= 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    LA[(aseg * XR + row0 + r) * XS + col0 + c] += la_lo[r][c];
                    if (aseg + 1 < p) LA[((aseg + 1) * XR + row0 + r) * XS + col0 + c] += la_hi[r][c];
                }
        }
        __syncwarp();
        // dJ/dU(i, a) = sum_r B(r, i) Lambda_a(r) + 2 sum_j R_ij sum_b W_ab U(j, b)
        // (diagonal R: 2 r_i sum_b W_ab U(i, b))
        auto wu_of = [&](int j, int aa, int t) {
            const int q = j * p + aa;
            float wu = a.gram[aa] * Us[q * XS + t];
            if (aa > 0) wu = fmaf(a.gram[p + aa - 1], Us[(q - 1) * XS + t], wu);
            if (aa + 1 < p) wu = fmaf(a.gram[p + aa], Us[(q + 1) * XS + t], wu);
            return wu;
        };
        for (int it = lane; it < D * CPW; it += 32) {
            const int q = it / CPW, t = it % CPW;
            const int i = q / p, aa = q % p;
            float gsum = 0.0f;
            for (int r = 0; r < n; ++r) gsum = fmaf(BTs[i * XR + r], LA[(aa * XR + r) * XS + t], gsum);
            float ru;
            if (a.rmat) {
                ru = 0.0f;
                for (int j = 0; j < m; ++j) ru = fmaf(a.rmat[i * m + j], wu_of(j, aa, t), ru);
            } else {
                ru = a.rdiag[i] * wu_of(i, aa, t);
            }
            G[q * XS + t] = fmaf(2.0f, ru, gsum);
        }
        __syncwarp();
        if (a.steps == 0) {
            for (int it = lane; it < D * CPW; it += 32) {
                const int q = it / CPW, t = it % CPW;
                if (c0 + t < a.count && a.grad) a.grad[(size_t)q * a.ld_grad + c0 + t] = G[q * XS + t];
            }
        } else {  // projected gradient step, U <- clip(U - eta g)
            for (int it = lane; it < D * CPW; it += 32) {
                const int q = it / CPW, t = it % CPW;
                const int i = q / p;
                Us[q * XS + t] = clamp_to(fmaf(-a.eta, G[q * XS + t], Us[q * XS + t]), a.umin[i],
                                          a.umax[i]);
            }
        }
        __syncwarp();
    }
    if (a.steps > 0 && a.pop_out) {
        for (int it = lane; it < D * CPW; it += 32) {
            const int q = it / CPW, t = it % CPW;
            if (c0 + t < a.count) a.pop_out[(size_t)q * a.ld_out + c0 + t] = Us[q * XS + t];
        }
    }
}

template <int NX, int C>
cudaError_t launch_grad_shape(const GradArgs& a, int wpc, cudaStream_t st) {
    constexpr int NRG = NX == 4 ? 2 : NX == 8 ? 4 : NX <= 24 ? 8 : NX <= 48 ? 16 : 32;
    const size_t smem = grad_smem_bytes(NX, NRG, C, wpc, a.n, a.m, a.p, a.T, a.ce);
    auto kern = grad_warp_kernel<NX, NRG, C>;
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    constexpr int CPW = (32 / NRG) * C;
    const int per_cta = wpc * CPW;
    const int grid = (a.count + per_cta - 1) / per_cta;
    kern<<<grid, 32 * wpc, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t grad_smem_bytes(int nx, int nrg, int cands, int wpc, int n, int m, int p, int T, int ce) {
    (void)n;
    const int R = (nx + nrg - 1) / nrg, xr = nrg * R;
    const int cpw = (32 / nrg) * cands, xs = round_up(cpw, 4);
    const int nseg = (T + ce - 1) / ce;
    const GradWarpLayout WL(xr, xs, nseg, ce, m * p, p);
    const int head = round_up(m * xr, 4) + round_up(nx * (nx + 1), 4) + 4 * T;
    return sizeof(float) * (size_t)(head + wpc * WL.total);
}

cudaError_t launch_grad(const GradArgs& a, int nx, int cands, int wpc, cudaStream_t st) {
#define EMPC_CASE(NXV)                                                          \
    if (nx == NXV) {                                                            \
        if (cands == 1) return launch_grad_shape<NXV, 1>(a, wpc, st);           \
        if (cands == 2) return launch_grad_shape<NXV, 2>(a, wpc, st);           \
    }
    EMPC_CASE(4) EMPC_CASE(8) EMPC_CASE(16) EMPC_CASE(24) EMPC_CASE(32) EMPC_CASE(40)
    EMPC_CASE(48) EMPC_CASE(56) EMPC_CASE(64)
#undef EMPC_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace empc
