// Device helpers shared by the two fused breed + rollout + cost kernels.
//
// Both kernels evaluate, per candidate, Algorithm 1's simulation and stage
// cost over the horizon (Sec. V), in the parameterized form of Sec. IV-C:
//
//   x_{k+1} = x_k + D x_k + w0_k BU_idx1(k) + w1_k BU_idx1(k)+1,  D = A_d - I,
//
// with BU_j = B_d U_j the force of knot j, formed once per knot segment.
// The delta form keeps FP32 rounding relative to the increment.
#pragma once
#include <cuda_runtime.h>

#include "draws.cuh"
#include "empc_internal.h"

namespace empc {

template <int C>
__device__ __forceinline__ void load_vec(const float* p, float (&v)[C]) {
    if constexpr (C == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (C == 2) {
        const float2 t = *reinterpret_cast<const float2*>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = *p;
    }
}

template <int C>
__device__ __forceinline__ void store_vec(float* p, const float (&v)[C]) {
    if constexpr (C == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (C == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

__host__ __device__ __forceinline__ int round_up(int v, int to) { return (v + to - 1) / to * to; }

// Programmatic dependent launch: let the next kernel in the stream start its
// CTAs (they run their prologue, then wait), and wait here until the previous
// kernel has completed and its writes are visible.  Both are no-ops for a
// kernel launched without the programmatic-serialization attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_primary() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// out[r][c] = sum_i B_d[row0 + r][i] U[i*p + a][col0 + c]  (knot force B_d U_a).
// BTs holds B_d transposed with leading dimension ldb (rows beyond n zero).
template <int R, int C>
__device__ __forceinline__ void knot_force(const float* BTs, int ldb, const float* Us, int xs,
                                           int m, int p, int a, int row0, int col0,
                                           float (&out)[R][C]) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) out[r][c] = 0.0f;
    for (int i = 0; i < m; ++i) {
        float u[C];
        load_vec<C>(Us + (i * p + a) * xs + col0, u);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float b = BTs[i * ldb + row0 + r];
#pragma unroll
            for (int c = 0; c < C; ++c) out[r][c] = fmaf(b, u[c], out[r][c]);
        }
    }
}

// Paired FP32 fused multiply-add (sm_100 and later): two independent IEEE
// round-to-nearest FMAs in one instruction, through the CUDA intrinsic so the
// compiler keeps the operands in register pairs.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Pair-interleaved state tile: row k of column col lives at
// ((k / 2) * xs + col) * 2 + (k & 1), so one vector load returns rows
// (k, k+1) for consecutive columns.
__host__ __device__ __forceinline__ int pair_index(int k, int col, int xs) {
    return ((k >> 1) * xs + col) * 2 + (k & 1);
}

// acc[r][c] += sum_k d[r][k] X[k][c] as four partial sums in two paired
// accumulators: k pairs alternate between acc and a second set, and within a
// pair .x takes the even k and .y the odd k, one paired FMA per (row,
// candidate, k pair).  2 R C independent paired chains of half the depth
// (measured 4% faster than one set at the 24-DoF chain); the order is
// fixed, the same for every candidate.
template <int NX, int R, int C>
__device__ __forceinline__ void state_product_pairs(const float2 (&d2)[R][NX / 2],
                                                    const float* Xp, int xs,
                                                    float2 (&acc)[R][C]) {
    float2 acc2[R][C];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc2[r][c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kp = 0; kp < NX / 2; ++kp) {
        float2 xv[C];
        const float* src = Xp + kp * xs * 2;
        if constexpr (C == 1) {
            xv[0] = *reinterpret_cast<const float2*>(src);
        } else {
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                const float4 t = *reinterpret_cast<const float4*>(src + 2 * c);
                xv[c] = make_float2(t.x, t.y);
                xv[c + 1] = make_float2(t.z, t.w);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (kp & 1) acc2[r][c] = fma2(d2[r][kp], xv[c], acc2[r][c]);
                else acc[r][c] = fma2(d2[r][kp], xv[c], acc[r][c]);
            }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = __fadd2_rn(acc[r][c], acc2[r][c]);
}

// acc[r][c] += sum_k d[r][k] X[k][c]: two interleaved partial sums (even and
// odd k) double the independent FMA chains; the split is part of the fixed
// summation order, identical for every candidate.
template <int NX, int R, int C>
__device__ __forceinline__ void state_product(const float (&d)[R][NX], const float* Xb, int xs,
                                              float (&acc)[R][C]) {
    float odd[R][C];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) odd[r][c] = 0.0f;
#pragma unroll
    for (int k = 0; k < NX; ++k) {
        float xv[C];
        load_vec<C>(Xb + k * xs, xv);
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (k & 1) odd[r][c] = fmaf(d[r][k], xv[c], odd[r][c]);
                else acc[r][c] = fmaf(d[r][k], xv[c], acc[r][c]);
            }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] += odd[r][c];
}

// Population loads.  The population is written by the kernel launched just
// before (or by other CTAs of a persistent kernel), which may still be running
// when this one starts (programmatic dependent launch): every read goes
// through L2 with a coherent load, never the read-only path, whose contents
// the compiler may assume fixed for the whole kernel.
template <bool COHERENT>
__device__ __forceinline__ float pop_load(const float* p) {
    return __ldcg(p);
}

// The mutation's standard deviation: per solve from device memory when the
// host sets it (distance-dependent exploration), else the fixed one.
__device__ __forceinline__ float noise_sigma(const RolloutArgs& a) {
    return a.sigma_dev ? __ldcg(a.sigma_dev) : a.sigma;
}

// Parents of child c as population columns (s1, s2); s2 < 0 marks an elite
// slot (c < E) copied unchanged from column s1.  Warm start only.
template <bool COHERENT>
__device__ __forceinline__ void parents_of(const RolloutArgs& a, int c, uint32_t gen, int& s1,
                                           int& s2) {
    s1 = 0;
    s2 = -1;
    if (c >= a.P) return;
    if (c < a.E) {
        s1 = COHERENT ? __ldcg(a.elite_idx + c) : a.elite_idx[c];
    } else {
        const Words4 o = draw(a.seed, (uint32_t)c, gen, kDrawParents, 0u);
        const int* ei = a.elite_idx;
        s1 = COHERENT ? __ldcg(ei + parent_rank(o.w[0], a.E)) : ei[parent_rank(o.w[0], a.E)];
        s2 = COHERENT ? __ldcg(ei + parent_rank(o.w[1], a.E)) : ei[parent_rank(o.w[1], a.E)];
    }
}

// Knots q0 .. q0+3 (q0 = 4 quad) of candidate c < P: loaded (eval), drawn
// (cold), or mated and mutated from parent columns s1, s2 (warm), as
// Algorithm 1's cold / warm branches specify.
template <bool COHERENT>
__device__ __forceinline__ void breed_quad(const RolloutArgs& a, int c, int quad, uint32_t gen,
                                           int s1, int s2, float (&v)[4]) {
    const int D = a.m * a.p;
    const int q0 = quad * 4;
#pragma unroll
    for (int w = 0; w < 4; ++w) v[w] = 0.0f;
    if (a.mode == kEval) {
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (q0 + w < D) v[w] = pop_load<COHERENT>(a.pop_in + (size_t)(q0 + w) * a.P + c);
    } else if (a.mode == kCold) {
        const Words4 o = draw(a.seed, (uint32_t)c, gen, kDrawInit, (uint32_t)quad);
        int i = q0 / a.p, j = q0 - i * a.p;  // input and knot of q0, advanced below
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int q = q0 + w;
            if (q < D) {
                const float lo = a.umin[i], hi = a.umax[i];
                v[w] = clamp_to(__fmaf_rn(__fsub_rn(hi, lo), unit_closed_open(o.w[w]), lo), lo, hi);
            }
            if (++j == a.p) {
                j = 0;
                ++i;
            }
        }
    } else if (s2 < 0) {
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (q0 + w < D) v[w] = pop_load<COHERENT>(a.pop_in + (size_t)(q0 + w) * a.P + s1);
    } else {
        const uint32_t cross =
            draw(a.seed, (uint32_t)c, gen, kDrawCross, (uint32_t)(quad >> 2)).w[quad & 3];
        // issue the parent-knot gathers before the remaining draws
        float mate[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int q = q0 + w;
            const uint32_t cb = (cross >> (8 * w)) & 0xFFu;
            mate[w] = q < D ? pop_load<COHERENT>(a.pop_in + (size_t)q * a.P +
                                                 (cb < (uint32_t)a.pc256 ? s2 : s1))
                            : 0.0f;
        }
        Words4 gw;
        uint32_t gate_blk = 0xFFFFFFFFu;
        float z[4];
        bool have_z = false;
        const float sg = noise_sigma(a);  // one read of the (device) sigma per quad
        int i = q0 / a.p, j = q0 - i * a.p;  // input and knot of q0, advanced below
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int q = q0 + w;
            if (q < D) {
                bool mut = true;
                if (a.gate != 2) {
                    const uint32_t gb = (a.gate == 0) ? (uint32_t)i : (uint32_t)q;
                    if ((gb >> 4) != gate_blk) {
                        gate_blk = gb >> 4;
                        gw = draw(a.seed, (uint32_t)c, gen, kDrawGate, gate_blk);
                    }
                    mut = ((gw.w[(gb >> 2) & 3u] >> (8u * (gb & 3u))) & 0xFFu) <
                          (uint32_t)a.pm256;
                }
                float val = mate[w];
                if (mut) {
                    if (!have_z) {
                        const Words4 nz =
                            draw(a.seed, (uint32_t)c, gen, kDrawNoise, (uint32_t)quad);
                        gauss_pair(nz.w[0], nz.w[1], &z[0], &z[1]);
                        gauss_pair(nz.w[2], nz.w[3], &z[2], &z[3]);
                        have_z = true;
                    }
                    val = __fmaf_rn(sg, z[w], mate[w]);
                }
                v[w] = clamp_to(val, a.umin[i], a.umax[i]);
            }
            if (++j == a.p) {
                j = 0;
                ++i;
            }
        }
    }
}

// Knots q0 .. q0+15 (q0 = 16 hex) of warm child c >= E, mated from parent
// columns s1, s2 and mutated: the same draws and arithmetic as four
// breed_quad calls, with each Philox block computed once (one crossover
// block covers 16 knots, one gate block 16 gate bytes).  Knots are produced
// a quad at a time and handed to emit(q, value).
template <bool COHERENT, class Emit>
__device__ __forceinline__ void breed_hex_warm(const RolloutArgs& a, int c, int hex,
                                               uint32_t gen, int s1, int s2, Emit&& emit) {
    const int D = a.m * a.p;
    const Words4 cr = draw(a.seed, (uint32_t)c, gen, kDrawCross, (uint32_t)hex);
    Words4 gw;
    uint32_t gate_blk = 0xFFFFFFFFu;
#pragma unroll
    for (int qd = 0; qd < 4; ++qd) {
        const int q0 = hex * 16 + qd * 4;
        if (q0 >= D) break;
        float mate[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int q = q0 + w;
            const uint32_t cb = (cr.w[qd] >> (8 * w)) & 0xFFu;
            mate[w] = q < D ? pop_load<COHERENT>(a.pop_in + (size_t)q * a.P +
                                                 (cb < (uint32_t)a.pc256 ? s2 : s1))
                            : 0.0f;
        }
        float z[4];
        bool have_z = false;
        const float sg = noise_sigma(a);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int q = q0 + w;
            if (q >= D) continue;
            const int i = q / a.p;
            bool mut = true;
            if (a.gate != 2) {
                const uint32_t gb = (a.gate == 0) ? (uint32_t)i : (uint32_t)q;
                if ((gb >> 4) != gate_blk) {
                    gate_blk = gb >> 4;
                    gw = draw(a.seed, (uint32_t)c, gen, kDrawGate, gate_blk);
                }
                mut = ((gw.w[(gb >> 2) & 3u] >> (8u * (gb & 3u))) & 0xFFu) < (uint32_t)a.pm256;
            }
            float val = mate[w];
            if (mut) {
                if (!have_z) {
                    const Words4 nz =
                        draw(a.seed, (uint32_t)c, gen, kDrawNoise, (uint32_t)(q0 >> 2));
                    gauss_pair(nz.w[0], nz.w[1], &z[0], &z[1]);
                    gauss_pair(nz.w[2], nz.w[3], &z[2], &z[3]);
                    have_z = true;
                }
                val = __fmaf_rn(sg, z[w], mate[w]);
            }
            emit(q, clamp_to(val, a.umin[i], a.umax[i]));
        }
    }
}

// dst[i] = src_of(i) for i in [0, count) over `nthr` threads (index tid): each
// thread issues its loads in batches of 8 before any of the stores, so one
// global-memory latency covers a batch instead of each element.
template <class F>
__device__ __forceinline__ void batched_fill(float* dst, int count, int tid, int nthr,
                                             F&& src_of) {
    for (int base = tid; base < count; base += 8 * nthr) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * nthr;
            v[u] = i < count ? src_of(i) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * nthr;
            if (i < count) dst[i] = v[u];
        }
    }
}

// Breed (cold / warm, Algorithm 1) or load (eval) the knots of candidates
// c0 .. c0+count-1 into Us[q][t] (leading dimension xs; skipped when Us is
// null); bred knots also go to pop_out.  Work is spread over `nthr` threads
// with index `tid`; WARP selects warp- or block-level synchronization.
template <bool WARP, bool COHERENT = false>
__device__ void fill_knots(const RolloutArgs& a, float* Us, int xs, int* par, int c0,
                           int count, uint32_t gen, int tid, int nthr) {
    const int D = a.m * a.p;
    const int nquad = (D + 3) >> 2;
    if (a.mode == kWarm) {
        for (int t = tid; t < count; t += nthr) {
            int s1, s2;
            parents_of<COHERENT>(a, c0 + t, gen, s1, s2);
            par[2 * t] = s1;
            par[2 * t + 1] = s2;
        }
        if (WARP) __syncwarp(); else __syncthreads();
    }
    if (a.mode == kWarm) {
        // children in 16-knot items (shared draws), elites copied
        const int nhex = (D + 15) >> 4;
        for (int it = tid; it < nhex * count; it += nthr) {
            const int t = it % count;
            const int hex = it / count;
            const int c = c0 + t;
            const int s1 = par[2 * t], s2 = par[2 * t + 1];
            auto emit = [&](int q, float v) {
                if (Us) Us[q * xs + t] = v;
                if (c < a.P) a.pop_out[(size_t)q * a.P + c] = v;
            };
            if (c >= a.P || s2 < 0) {
                for (int w = 0; w < 16; ++w) {
                    const int q = hex * 16 + w;
                    if (q < D) emit(q, c < a.P ? pop_load<COHERENT>(a.pop_in + (size_t)q * a.P + s1)
                                               : 0.0f);
                }
            } else {
                breed_hex_warm<COHERENT>(a, c, hex, gen, s1, s2, emit);
            }
        }
    } else if (a.mode == kEval) {
        // evaluation: a plain copy of the knots, loads batched (the population
        // was written by the previous kernel: coherent loads through L2)
        if (Us)
            batched_fill(Us, D * xs, tid, nthr, [&](int i) {
                const int q = i / xs, t = i - q * xs;
                const int c = c0 + t;
                return (t < count && c < a.P) ? __ldcg(a.pop_in + (size_t)q * a.P + c) : 0.0f;
            });
    } else {
        for (int it = tid; it < nquad * count; it += nthr) {
            const int t = it % count;
            const int quad = it / count;
            const int c = c0 + t;
            float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (c < a.P) breed_quad<COHERENT>(a, c, quad, gen, 0, -1, v);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int q = quad * 4 + w;
                if (q < D) {
                    if (Us) Us[q * xs + t] = v[w];
                    if (a.mode != kEval && c < a.P) a.pop_out[(size_t)q * a.P + c] = v[w];
                }
            }
        }
    }
    if (WARP) __syncwarp(); else __syncthreads();
}

// Input cost sum_k u_k' R u_k of one candidate restricted to inputs
// i0, i0 + istep, ..., in closed form through the tridiagonal Gram matrix of
// the knot weights (W_aa = gram[a], W_a,a+1 = gram[p + a]):
// sum_k u_k' R u_k = sum_ij R_ij U_i' W U_j.  Diagonal R: r_i U_i' W U_i.
// Dense R (a.rmat): row i contributes U_i' W y_i with y_i,a = (R U_a)_i, U_a
// the inputs' knot a.
template <class Args>
__device__ __forceinline__ float input_cost_part(const Args& a, const float* Us, int xs,
                                                 int col, int i0, int istep) {
    const int p = a.p;
    float Ju = 0.0f;
    if (a.rmat) {
        for (int i = i0; i < a.m; i += istep) {
            float s = 0.0f, y_prev = 0.0f, u_prev = 0.0f;
            for (int j = 0; j < p; ++j) {
                float y = 0.0f;
                for (int l = 0; l < a.m; ++l)
                    y = fmaf(a.rmat[i * a.m + l], Us[(l * p + j) * xs + col], y);
                const float u = Us[(i * p + j) * xs + col];
                s = fmaf(a.gram[j] * u, y, s);
                if (j > 0) s = fmaf(a.gram[p + j - 1], fmaf(u_prev, y, u * y_prev), s);
                y_prev = y;
                u_prev = u;
            }
            Ju += s;
        }
        return Ju;
    }
    for (int i = i0; i < a.m; i += istep) {
        float s = 0.0f;
        for (int j = 0; j < p; ++j) {
            const float u = Us[(i * p + j) * xs + col];
            s = fmaf(a.gram[j] * u, u, s);
            if (j + 1 < p) s = fmaf(2.0f * a.gram[p + j] * u, Us[(i * p + j + 1) * xs + col], s);
        }
        Ju = fmaf(a.rdiag[i], s, Ju);
    }
    return Ju;
}

// The state-box hook for one state (Sec. V: with every state of every step
// simulated, hard stops and non-convex state costs go into the simulation as
// plain if/else).  bx is [3][ld] (lo, hi, rho; rows past n hold -inf, +inf,
// 0).  With mode bit 1 adds rho d^2 to j, d = max(0, lo - x, x - hi) the
// distance outside the box; with mode bit 0 returns x stopped at the box.
__device__ __forceinline__ float box_hook(const float* bx, int ld, int row, int mode, float x,
                                          float& j) {
    const float lo = bx[row], hi = bx[ld + row];
    if (mode & 2) {
        const float d = fmaxf(fmaxf(lo - x, x - hi), 0.0f);
        j = fmaf(bx[2 * ld + row] * d, d, j);
    }
    return (mode & 1) ? fminf(fmaxf(x, lo), hi) : x;
}

// Whether a rollout runs the hooked copy of its horizon loop: a state box
// or a constant disturbance.
__device__ __forceinline__ bool has_hooks(const RolloutArgs& a) {
    return a.box_mode != 0 || a.wd != nullptr;
}

// Stage the hooks of rows 0 .. ld-1 into shared memory as [4][ld]: lo, hi,
// rho of the state box (a box that never binds without one, and on padding
// rows) and the disturbance w_d (zero without one).
__device__ __forceinline__ void stage_box(const RolloutArgs& a, float* bx, int ld, int t,
                                          int nt) {
    for (int i = t; i < 4 * ld; i += nt) {
        const int which = i / ld, row = i - which * ld;
        float v = which == 0 ? -INFINITY : which == 1 ? INFINITY : 0.0f;
        if (row < a.n) {
            if (which < 3 && a.box_mode) v = a.box[which * a.n + row];
            if (which == 3 && a.wd) v = a.wd[row];
        }
        bx[i] = v;
    }
}

__device__ __forceinline__ float finite_or_inf(float v) {
    return (v == v) ? v : __int_as_float(0x7f800000);
}

}  // namespace empc

namespace empc {

// The horizon loop for one thread: rows row0 .. row0+R-1 of C candidates
// (columns col0 .. col0+C-1 of the state tile X[2][xrows][xs]).  D rows are
// in registers; BU pairs are refreshed at knot-segment changes; the stage
// cost is accumulated in 16-step blocks.  One barrier (warp or block) per
// step separates the double-buffered state reads from the writes.  BOX
// compiles in the hooks staged at bx (stage_box): the disturbance w_d, then
// the state box.
template <int NX, int R, int C, bool WARP, bool BOX = false>
__device__ __forceinline__ void horizon_loop(const RolloutArgs& a, const float (&d)[R][NX],
                                             float* X, int xrows, int xs, const float* BTs,
                                             int ldb, const float* Us, const KnotStep* ks,
                                             int row0, int col0, float (&xo)[R][C],
                                             const float (&qd)[R], const float (&gl)[R],
                                             float (&jsum)[C], const float* bx = nullptr) {
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
        float acc[R][C];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < C; ++c) acc[r][c] = fmaf(st.w1, bub[r][c], st.w0 * bua[r][c]);
        state_product<NX, R, C>(d, X + buf * xrows * xs + col0, xs, acc);
        float* Xn = X + (buf ^ 1) * xrows * xs + col0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float xn[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                xn[c] = xo[r][c] + acc[r][c];
                if constexpr (BOX) {
                    xn[c] = xn[c] + bx[3 * xrows + row0 + r];  // w_d
                    xn[c] = box_hook(bx, xrows, row0 + r, a.box_mode, xn[c], jblk[c]);
                }
                xo[r][c] = xn[c];
                const float e = xn[c] - gl[r];
                jblk[c] = fmaf(qd[r] * e, e, jblk[c]);
            }
            store_vec<C>(Xn + (row0 + r) * xs, xn);
        }
        if ((k & 15) == 15) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                jtot[c] += jblk[c];
                jblk[c] = 0.0f;
            }
        }
        if (WARP) __syncwarp(); else __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) jsum[c] = jtot[c] + jblk[c];
}

// Load this thread's D rows, Q diagonal, goal and initial state.
template <int NX, int R, int C>
__device__ __forceinline__ void load_rows(const RolloutArgs& a, int row0, float (&d)[R][NX],
                                          float (&qd)[R], float (&gl)[R], float (&xo)[R][C]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = row0 + r;
        const bool ok = row < a.n;
#pragma unroll
        for (int k = 0; k < NX; ++k) d[r][k] = (ok && k < a.n) ? a.D[row * a.n + k] : 0.0f;
        qd[r] = ok ? a.qdiag[row] : 0.0f;
        gl[r] = ok ? a.goal[row] : 0.0f;
#pragma unroll
        for (int c = 0; c < C; ++c) xo[r][c] = ok ? a.x0[row] : 0.0f;
    }
}

}  // namespace empc
