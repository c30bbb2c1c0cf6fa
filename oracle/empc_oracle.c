/*
 * EMPC oracle: a plain, slow, obviously correct CPU restatement of the
 * evolutionary MPC generation described in Hyatt, Williams & Killpack,
 * "Parameterized and GPU-Parallelized Real-Time Model Predictive Control for
 * High Degree of Freedom Robots" (arXiv 2001.04931).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the product path never links or calls it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Precision: every step of the method's arithmetic (discretization, knot
 * expansion, rollout, cost, condensed quadratic form, adjoint gradient,
 * projected-gradient refinement) is FP64.  The genome (knot values) is FP32
 * by the interface, so breeding (Philox draws, Gaussian transform, crossover,
 * mutation, clipping) is specified in FP32 with an explicit operation order;
 * this file is compiled with -ffp-contract=off so that every fused
 * multiply-add below is exactly the fmaf() written.
 *
 * Functions and the passage each follows:
 *   orc_philox4x32_10      Philox4x32-10 counter-based generator (Salmon et
 *                          al., SC'11); draws of Alg. 1 (cold start, parents,
 *                          noise).
 *   orc_log_f32, orc_sincos_octant, orc_box_muller
 *                          Gaussian transform for the N(0, sigma) mutation
 *                          noise (Sec. V, Alg. 1 Noise draw).
 *   orc_zoh                discretization of the continuous model (Sec. III-A,
 *                          "matrix exponential").
 *   orc_knot_table         piecewise-linear knot parameterization (Sec. IV-C,
 *                          Delta T, idx1, idx2, c).
 *   orc_cost               forward simulation x_{k+1} = A_d x_k + B_d u_k + w_d
 *                          (Eq. first_order_integration) and the quadratic
 *                          cost (Eq. mpc_problem).
 *   orc_condensed          parameterized small-matrix formulation
 *                          J = U'HU + 2f'U + c (Sec. IV-B and IV-E).
 *   orc_grad               adjoint gradient dJ/dU (no counterpart in the paper).
 *   orc_cost_box           orc_cost (conv 0) with the state-box hook of Sec. V:
 *                          hinge penalty and/or hard stop per state.
 *   orc_select             parent selection: the lowest-cost candidates (Alg. 1
 *                          parent line, Sec. V parent selection).
 *   orc_breed_cold/_warm   cold start and mate + mutate (Alg. 1, Sec. V).
 *   orc_refine             projected-gradient refinement of the elites (no
 *                          counterpart in the paper).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11.  Four 32-bit counter words, two key words, ten   */
/* rounds.  Each round multiplies words 0 and 2 by the two Philox constants, */
/* and the high halves are xored with the other words and the round key.     */
/* The key is bumped by the two Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                  uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for a (candidate, generation, purpose, block) counter. */
static void draw_block(uint64_t seed, uint32_t cand, uint32_t gen, uint32_t purpose,
                       uint32_t block, uint32_t out[4]) {
    uint32_t ctr[4] = {cand, gen, purpose, block};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

enum { PURPOSE_INIT = 0, PURPOSE_PARENTS = 1, PURPOSE_CROSS = 2, PURPOSE_GATE = 3,
       PURPOSE_NOISE = 4 };

/* Uniform in [0, 1): the top 24 bits of a word times 2^-24 (exact in FP32). */
static float u01(uint32_t r) { return (float)(r >> 8) * 0x1p-24f; }
/* Uniform in (0, 1]: (top 24 bits + 1) times 2^-24 (exact in FP32). */
static float u01_open0(uint32_t r) { return (float)((r >> 8) + 1u) * 0x1p-24f; }

/* ------------------------------------------------------------------------ */
/* Natural log in FP32 for u in (0, 1] (always a normal number here).        */
/* u = 2^e * f with f in [sqrt(1/2), sqrt(2)]; ln f = 2 atanh(s),            */
/* s = (f - 1)/(f + 1), by the series atanh(s) = s + s^3/3 + s^5/5 + ...     */
/* truncated after s^11/11 (|s| <= 0.1716, next term < 1e-11).               */
/* Horner form with explicit fmaf in a fixed order.                          */
/* ------------------------------------------------------------------------ */
ORC_EXPORT float orc_log_f32(float u) {
    uint32_t bits;
    memcpy(&bits, &u, 4);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    uint32_t fbits = (bits & 0x007FFFFFu) | 0x3F800000u;
    float f;
    memcpy(&f, &fbits, 4);
    if (f > 1.41421356f) { /* fold into [sqrt(1/2), sqrt(2)] exactly */
        f = f * 0.5f;
        e += 1;
    }
    float s = (f - 1.0f) / (f + 1.0f);
    float s2 = s * s;
    float poly = 1.0f / 11.0f;
    poly = fmaf(poly, s2, 1.0f / 9.0f);
    poly = fmaf(poly, s2, 1.0f / 7.0f);
    poly = fmaf(poly, s2, 1.0f / 5.0f);
    poly = fmaf(poly, s2, 1.0f / 3.0f);
    float t = s2 * poly;
    float two_s = 2.0f * s;
    float lnf = fmaf(two_s, t, two_s);
    return fmaf((float)e, 0.693147180559945309f, lnf);
}

/* sin and cos of phi in [0, pi/4] by their Taylor series, truncated after  */
/* phi^9/9! and phi^10/10! (truncation < 2e-9).  Horner in phi^2.           */
static void sincos_small(float phi, float* s, float* c) {
    float p2 = phi * phi;
    float ps = 1.0f / 362880.0f;
    ps = fmaf(ps, p2, -1.0f / 5040.0f);
    ps = fmaf(ps, p2, 1.0f / 120.0f);
    ps = fmaf(ps, p2, -1.0f / 6.0f);
    float p3 = p2 * phi;
    *s = fmaf(p3, ps, phi);
    float pc = -1.0f / 3628800.0f;
    pc = fmaf(pc, p2, 1.0f / 40320.0f);
    pc = fmaf(pc, p2, -1.0f / 720.0f);
    pc = fmaf(pc, p2, 1.0f / 24.0f);
    pc = fmaf(pc, p2, -0.5f);
    *c = fmaf(p2, pc, 1.0f);
}

/* sin and cos of 2*pi*t for t = r24 * 2^-24 (r24 < 2^24).                   */
/* Exact octant reduction: octant o = r24 >> 21, fraction fr = low 21 bits   */
/* times 2^-21.  Even o: angle = (o/2) pi/2 + fr pi/4.  Odd o: angle =        */
/* ((o+1)/2) pi/2 - (1 - fr) pi/4.  Quadrant rotations are sign/swap only.   */
ORC_EXPORT void orc_sincos_octant(uint32_t r24, float* sin_out, float* cos_out) {
    uint32_t o = (r24 >> 21) & 7u;
    float fr = (float)(r24 & 0x1FFFFFu) * 0x1p-21f;
    int neg = 0;
    uint32_t quad;
    if (o & 1u) {
        fr = 1.0f - fr; /* exact: fr is a multiple of 2^-21 in [0, 1) */
        neg = 1;
        quad = ((o + 1u) >> 1) & 3u;
    } else {
        quad = (o >> 1) & 3u;
    }
    float phi = fr * 0.785398163397448310f;
    float s, c;
    sincos_small(phi, &s, &c);
    if (neg) s = -s; /* sin(-phi) = -sin(phi) */
    float so, co;
    switch (quad) {
        case 0: so = s;  co = c;  break;
        case 1: so = c;  co = -s; break;
        case 2: so = -s; co = -c; break;
        default: so = -c; co = s; break;
    }
    *sin_out = so;
    *cos_out = co;
}

/* Box-Muller: (z0, z1) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2),        */
/* u1 in (0, 1] from word ra, u2 in [0, 1) from word rb.                     */
ORC_EXPORT void orc_box_muller(uint32_t ra, uint32_t rb, float* z0, float* z1) {
    float u1 = u01_open0(ra);
    float l = orc_log_f32(u1);
    float rad = sqrtf(-2.0f * l);
    float s, c;
    orc_sincos_octant(rb >> 8, &s, &c);
    *z0 = rad * c;
    *z1 = rad * s;
}

/* Byte b (0..) of a decision stream, one Philox block per 16 bytes. */
static uint32_t stream_byte(uint64_t seed, uint32_t cand, uint32_t gen, uint32_t purpose,
                            uint32_t b) {
    uint32_t out[4];
    draw_block(seed, cand, gen, purpose, b >> 4, out);
    uint32_t word = out[(b >> 2) & 3u];
    return (word >> (8u * (b & 3u))) & 0xFFu;
}

/* Standard normal for parameter q of candidate cand (pair q/2, block q/4). */
static float noise_normal(uint64_t seed, uint32_t cand, uint32_t gen, uint32_t q) {
    uint32_t out[4];
    uint32_t pair = q >> 1;
    draw_block(seed, cand, gen, PURPOSE_NOISE, pair >> 1, out);
    uint32_t w = (pair & 1u) * 2u;
    float z0, z1;
    orc_box_muller(out[w], out[w + 1], &z0, &z1);
    return (q & 1u) ? z1 : z0;
}

static float clipf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

/* Cold start, Alg. 1 first branch: U(i) ~ Uniform(u_min(i), u_max(i)).      */
/* pop is SoA: parameter q = i*p + j of candidate c at pop[q*P + c].         */
ORC_EXPORT void orc_breed_cold(uint64_t seed, uint32_t gen, const float* umin,
                               const float* umax, int m, int p, int P, float* pop) {
    for (int c = 0; c < P; ++c) {
        for (int q = 0; q < m * p; ++q) {
            uint32_t out[4];
            draw_block(seed, (uint32_t)c, gen, PURPOSE_INIT, (uint32_t)q >> 2, out);
            int i = q / p;
            float width = umax[i] - umin[i];
            float v = fmaf(width, u01(out[q & 3]), umin[i]);
            pop[(size_t)q * P + c] = clipf(v, umin[i], umax[i]);
        }
    }
}

/* Warm start, Alg. 1 second branch, with elitism (Sec. V parent selection):  */
/*  - slots 0..E-1 carry the elites unchanged, in rank order;                 */
/*  - child c >= E draws parents P1, P2 uniformly from the E elites           */
/*    (multiply-shift of a 32-bit word), takes each parameter from P2 with    */
/*    probability pc256/256 (else P1), then each input (gate_mode 0), each    */
/*    parameter (gate_mode 1) or everything (gate_mode 2) is mutated with      */
/*    probability pm256/256 by adding sigma * N(0,1); finally clip to bounds. */
ORC_EXPORT void orc_breed_warm(uint64_t seed, uint32_t gen, const float* old_pop,
                               const int* elite_idx, int E, const float* umin,
                               const float* umax, int m, int p, int P, float sigma,
                               int pc256, int pm256, int gate_mode, float* new_pop) {
    int D = m * p;
    for (int c = 0; c < P; ++c) {
        if (c < E) {
            for (int q = 0; q < D; ++q)
                new_pop[(size_t)q * P + c] = old_pop[(size_t)q * P + elite_idx[c]];
            continue;
        }
        uint32_t par[4];
        draw_block(seed, (uint32_t)c, gen, PURPOSE_PARENTS, 0u, par);
        int p1 = (int)(((uint64_t)par[0] * (uint64_t)E) >> 32);
        int p2 = (int)(((uint64_t)par[1] * (uint64_t)E) >> 32);
        int s1 = elite_idx[p1], s2 = elite_idx[p2];
        for (int q = 0; q < D; ++q) {
            int i = q / p;
            uint32_t cross = stream_byte(seed, (uint32_t)c, gen, PURPOSE_CROSS, (uint32_t)q);
            float mate = (cross < (uint32_t)pc256) ? old_pop[(size_t)q * P + s2]
                                                   : old_pop[(size_t)q * P + s1];
            int mutate;
            if (gate_mode == 2) {
                mutate = 1;
            } else {
                uint32_t gb = (gate_mode == 0) ? (uint32_t)i : (uint32_t)q;
                mutate = stream_byte(seed, (uint32_t)c, gen, PURPOSE_GATE, gb) < (uint32_t)pm256;
            }
            float v = mate;
            if (mutate) v = fmaf(sigma, noise_normal(seed, (uint32_t)c, gen, (uint32_t)q), mate);
            new_pop[(size_t)q * P + c] = clipf(v, umin[i], umax[i]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Knot table, Sec. IV-C: Delta T = (T-1)/(p-1), idx1 = floor(k / Delta T),  */
/* idx2 = idx1 + 1, c = (k - idx1 Delta T)/Delta T.  In exact integers:      */
/* idx1 = min(floor(k (p-1) / (T-1)), p-2), c = num/(T-1) with               */
/* num = k (p-1) - idx1 (T-1).  At k = T-1 this gives idx1 = p-2, c = 1,     */
/* i.e. u = U_{p-1}, the same input as idx1 = p-1, c = 0 without indexing    */
/* past the last knot.  p = 1 (constant input) and T = 1 give idx1 = 0,      */
/* c = 0.  Returns the denominator.                                          */
/* ------------------------------------------------------------------------ */
ORC_EXPORT long orc_knot_table(int T, int p, int* idx1, long* num) {
    long den = (T > 1) ? (long)(T - 1) : 1L;
    for (int k = 0; k < T; ++k) {
        if (p <= 1 || T <= 1) {
            idx1[k] = 0;
            num[k] = 0;
            continue;
        }
        long a = (long)k * (long)(p - 1) / den;
        if (a > p - 2) a = p - 2;
        idx1[k] = (int)a;
        num[k] = (long)k * (long)(p - 1) - a * den;
    }
    return den;
}

/* u_k(i) = (1 - c_k) U(i, idx1) + c_k U(i, idx2) for all k, FP64.  U is     */
/* [m][p] (parameter q = i*p + j).  uexp is [T][m].                          */
static void expand_inputs(const double* U, int m, int T, int p, double* uexp) {
    int* idx1 = (int*)malloc(sizeof(int) * (size_t)T);
    long* num = (long*)malloc(sizeof(long) * (size_t)T);
    long den = orc_knot_table(T, p, idx1, num);
    for (int k = 0; k < T; ++k) {
        double c = (double)num[k] / (double)den;
        for (int i = 0; i < m; ++i) {
            double a = U[i * p + idx1[k]];
            double b = (p > 1) ? U[i * p + idx1[k] + 1] : 0.0;
            uexp[k * m + i] = (1.0 - c) * a + c * b;
        }
    }
    free(idx1);
    free(num);
}

ORC_EXPORT void orc_expand(const double* U, int m, int T, int p, double* uexp) {
    expand_inputs(U, m, T, p, uexp);
}

static double quad_form(const double* M, const double* v, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += M[i * n + j] * v[j];
        s += v[i] * r;
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Forward simulation and cost of one knot vector, FP64.                     */
/* Dynamics: x_{k+1} = A_d x_k + B_d u_k + w_d (Eq. first_order_integration). */
/* Cost (Eq. mpc_problem with u_goal = 0):                                   */
/*   conv 0 (default): J = sum_{k=0}^{T-1} (x_{k+1}-g)'Q(x_{k+1}-g)          */
/*                              + u_k' R u_k                                 */
/*     i.e. the stage cost taken after each update, as Alg. 1 accumulates it */
/*     (states x_1..x_T, matching the stacked states of the small-matrix     */
/*     formulation Eq. small_matrix_sz_v); no separate terminal term.        */
/*   conv 1: the sum of Eq. mpc_problem read literally, states x_0..x_{T-1}. */
/* w may be NULL (zero disturbance).  traj, if given, receives x_0..x_T.     */
/* ------------------------------------------------------------------------ */
ORC_EXPORT double orc_cost(const double* A, const double* B, const double* Q,
                           const double* R, const double* w, const double* x0,
                           const double* g, const double* U, int n, int m, int T, int p,
                           int conv, double* traj) {
    double* uexp = (double*)malloc(sizeof(double) * (size_t)T * (size_t)m);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n);
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    expand_inputs(U, m, T, p, uexp);
    memcpy(x, x0, sizeof(double) * (size_t)n);
    if (traj) memcpy(traj, x0, sizeof(double) * (size_t)n);
    double J = 0.0;
    for (int k = 0; k < T; ++k) {
        const double* u = uexp + (size_t)k * m;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += A[i * n + j] * x[j];
            for (int j = 0; j < m; ++j) s += B[i * m + j] * u[j];
            if (w) s += w[i];
            xn[i] = s;
        }
        const double* xs = (conv == 0) ? xn : x;
        for (int i = 0; i < n; ++i) e[i] = xs[i] - g[i];
        J += quad_form(Q, e, n) + quad_form(R, u, m);
        memcpy(x, xn, sizeof(double) * (size_t)n);
        if (traj) memcpy(traj + (size_t)(k + 1) * n, x, sizeof(double) * (size_t)n);
    }
    free(uexp);
    free(x);
    free(xn);
    free(e);
    return J;
}

/* Costs of a whole SoA population (pop[q*P + c], FP32 knots), one candidate */
/* after another (each candidate is one simulation of Alg. 1).               */
ORC_EXPORT void orc_cost_population(const double* A, const double* B, const double* Q,
                                    const double* R, const double* w, const double* x0,
                                    const double* g, const float* pop, int n, int m, int T,
                                    int p, int P, int conv, double* cost) {
    int D = m * p;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < P; ++c) {
        double* U = (double*)malloc(sizeof(double) * (size_t)D);
        for (int q = 0; q < D; ++q) U[q] = (double)pop[(size_t)q * P + c];
        cost[c] = orc_cost(A, B, Q, R, w, x0, g, U, n, m, T, p, conv, NULL);
        free(U);
    }
}

/* ------------------------------------------------------------------------ */
/* Forward simulation with the state-box hook, FP64.                         */
/* Sec. V (simulation and cost calculation) notes that because every state  */
/* of every step is computed explicitly, nonlinear effects such as contact  */
/* or hard stops, and non-convex costs, can be put into the simulation as   */
/* plain if/else.  This is one such hook, per state i with bounds           */
/* lo_i <= hi_i and weight rho_i >= 0.  After each update                   */
/*   x_{k+1} = A_d x_k + B_d u_k + w_d                                      */
/* and for every state i, in this order:                                    */
/*   d_i = max(0, lo_i - x_i, x_i - hi_i)   distance outside the box        */
/*   mode bit 1 (value 2): J += rho_i d_i^2  (hinge penalty, soft limit)     */
/*   mode bit 0 (value 1): x_i = min(max(x_i, lo_i), hi_i)  (hard stop)      */
/* then the stage cost of the (stopped) state and u_k' R u_k as orc_cost    */
/* conv 0.  The stopped state is the one the next step starts from.  With   */
/* mode 0 this is orc_cost conv 0.  traj, if given, receives x_0..x_T.      */
/* ------------------------------------------------------------------------ */
ORC_EXPORT double orc_cost_box(const double* A, const double* B, const double* Q,
                               const double* R, const double* w, const double* x0,
                               const double* g, const double* U, int n, int m, int T, int p,
                               const double* lo, const double* hi, const double* rho, int mode,
                               double* traj) {
    double* uexp = (double*)malloc(sizeof(double) * (size_t)T * (size_t)m);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* xn = (double*)malloc(sizeof(double) * (size_t)n);
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    expand_inputs(U, m, T, p, uexp);
    memcpy(x, x0, sizeof(double) * (size_t)n);
    if (traj) memcpy(traj, x0, sizeof(double) * (size_t)n);
    double J = 0.0;
    for (int k = 0; k < T; ++k) {
        const double* u = uexp + (size_t)k * m;
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += A[i * n + j] * x[j];
            for (int j = 0; j < m; ++j) s += B[i * m + j] * u[j];
            if (w) s += w[i];
            xn[i] = s;
        }
        double pen = 0.0;
        for (int i = 0; i < n; ++i) {
            double d = 0.0;
            if (xn[i] < lo[i]) d = lo[i] - xn[i];
            if (xn[i] > hi[i]) d = xn[i] - hi[i];
            if (mode & 2) pen += rho[i] * d * d;
            if (mode & 1) {
                if (xn[i] < lo[i]) xn[i] = lo[i];
                if (xn[i] > hi[i]) xn[i] = hi[i];
            }
        }
        for (int i = 0; i < n; ++i) e[i] = xn[i] - g[i];
        J += quad_form(Q, e, n) + quad_form(R, u, m) + pen;
        memcpy(x, xn, sizeof(double) * (size_t)n);
        if (traj) memcpy(traj + (size_t)(k + 1) * n, x, sizeof(double) * (size_t)n);
    }
    free(uexp);
    free(x);
    free(xn);
    free(e);
    return J;
}

/* orc_cost_box for a whole SoA population (pop[q*P + c], FP32 knots).       */
ORC_EXPORT void orc_cost_population_box(const double* A, const double* B, const double* Q,
                                        const double* R, const double* w, const double* x0,
                                        const double* g, const float* pop, int n, int m, int T,
                                        int p, int P, const double* lo, const double* hi,
                                        const double* rho, int mode, double* cost) {
    int D = m * p;
#pragma omp parallel for schedule(static)
    for (int c = 0; c < P; ++c) {
        double* U = (double*)malloc(sizeof(double) * (size_t)D);
        for (int q = 0; q < D; ++q) U[q] = (double)pop[(size_t)q * P + c];
        cost[c] = orc_cost_box(A, B, Q, R, w, x0, g, U, n, m, T, p, lo, hi, rho, mode, NULL);
        free(U);
    }
}

/* ------------------------------------------------------------------------ */
/* Parameterized small-matrix formulation (Sec. IV-B, IV-E).                 */
/* Stacked states [x_1; ...; x_T] = S U + v.  S is built top-down as the     */
/* paper describes: each block row is the previous one premultiplied by A_d, */
/* plus B_d in the knot proportions of that step.  v_k = A_d v_{k-1} + w_d,  */
/* v_0 = x_0.  Then J = U'HU + 2 f'U + c0 with                               */
/*   H  = S' Qbig S + sum_k Omega_k' R Omega_k,                              */
/*   f  = S' Qbig (v - gbig),  c0 = (v - gbig)' Qbig (v - gbig),             */
/* where Omega_k (m x mp) maps the knots to u_k.  S is (T n) x (m p).        */
/* ------------------------------------------------------------------------ */
ORC_EXPORT void orc_condensed(const double* A, const double* B, const double* Q,
                              const double* R, const double* w, const double* x0,
                              const double* g, int n, int m, int T, int p, double* S,
                              double* H, double* f, double* c0) {
    int D = m * p;
    int* idx1 = (int*)malloc(sizeof(int) * (size_t)T);
    long* num = (long*)malloc(sizeof(long) * (size_t)T);
    long den = orc_knot_table(T, p, idx1, num);
    double* Sloc = S ? S : (double*)malloc(sizeof(double) * (size_t)T * n * D);
    double* v = (double*)malloc(sizeof(double) * (size_t)T * n);
    double* prevS = (double*)calloc((size_t)n * D, sizeof(double));
    double* prevv = (double*)malloc(sizeof(double) * (size_t)n);
    double* Om = (double*)malloc(sizeof(double) * (size_t)m * D);
    memcpy(prevv, x0, sizeof(double) * (size_t)n);
    memset(H, 0, sizeof(double) * (size_t)D * D);
    for (int k = 0; k < T; ++k) {
        double c = (double)num[k] / (double)den;
        memset(Om, 0, sizeof(double) * (size_t)m * D);
        for (int i = 0; i < m; ++i) {
            Om[i * D + i * p + idx1[k]] += 1.0 - c;
            if (p > 1) Om[i * D + i * p + idx1[k] + 1] += c;
        }
        double* Sk = Sloc + (size_t)k * n * D;
        for (int r = 0; r < n; ++r) {
            for (int col = 0; col < D; ++col) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += A[r * n + j] * prevS[j * D + col];
                for (int j = 0; j < m; ++j) s += B[r * m + j] * Om[j * D + col];
                Sk[r * D + col] = s;
            }
            double sv = 0.0;
            for (int j = 0; j < n; ++j) sv += A[r * n + j] * prevv[j];
            if (w) sv += w[r];
            v[(size_t)k * n + r] = sv;
        }
        memcpy(prevS, Sk, sizeof(double) * (size_t)n * D);
        memcpy(prevv, v + (size_t)k * n, sizeof(double) * (size_t)n);
        /* input term: Omega_k' R Omega_k */
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                double s = 0.0;
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < m; ++j) s += Om[i * D + a] * R[i * m + j] * Om[j * D + b];
                H[a * D + b] += s;
            }
    }
    /* state term: S' Qbig S, f, c0 */
    memset(f, 0, sizeof(double) * (size_t)D);
    double cc = 0.0;
    double* QS = (double*)malloc(sizeof(double) * (size_t)n * D);
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    for (int k = 0; k < T; ++k) {
        double* Sk = Sloc + (size_t)k * n * D;
        for (int r = 0; r < n; ++r)
            for (int col = 0; col < D; ++col) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += Q[r * n + j] * Sk[j * D + col];
                QS[r * D + col] = s;
            }
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                double s = 0.0;
                for (int r = 0; r < n; ++r) s += Sk[r * D + a] * QS[r * D + b];
                H[a * D + b] += s;
            }
        for (int r = 0; r < n; ++r) e[r] = v[(size_t)k * n + r] - g[r];
        for (int a = 0; a < D; ++a) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += QS[r * D + a] * e[r];
            f[a] += s;
        }
        cc += quad_form(Q, e, n);
    }
    *c0 = cc;
    free(QS);
    free(e);
    if (!S) free(Sloc);
    free(v);
    free(prevS);
    free(prevv);
    free(Om);
    free(idx1);
    free(num);
}

/* ------------------------------------------------------------------------ */
/* Adjoint gradient of the conv-0 cost with respect to the knots, FP64.      */
/* With e_k = x_k - g:  lambda_T = 2 Q e_T,                                  */
/*   lambda_k = A_d' lambda_{k+1} + 2 Q e_k   (k = T-1 .. 1),                */
/*   dJ/du_k  = B_d' lambda_{k+1} + 2 R u_k   (k = 0 .. T-1),                */
/*   dJ/dU(i, j) = sum_k w_{k j} dJ/du_k(i), w_{k j} the knot weights.       */
/* (Q and R symmetric.)  Returns J.                                          */
/* ------------------------------------------------------------------------ */
ORC_EXPORT double orc_grad(const double* A, const double* B, const double* Q,
                           const double* R, const double* w, const double* x0,
                           const double* g, const double* U, int n, int m, int T, int p,
                           double* grad) {
    int D = m * p;
    double* traj = (double*)malloc(sizeof(double) * (size_t)(T + 1) * n);
    double* uexp = (double*)malloc(sizeof(double) * (size_t)T * m);
    double J = orc_cost(A, B, Q, R, w, x0, g, U, n, m, T, p, 0, traj);
    expand_inputs(U, m, T, p, uexp);
    int* idx1 = (int*)malloc(sizeof(int) * (size_t)T);
    long* num = (long*)malloc(sizeof(long) * (size_t)T);
    long den = orc_knot_table(T, p, idx1, num);
    double* lam = (double*)malloc(sizeof(double) * (size_t)n);
    double* lam2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* du = (double*)malloc(sizeof(double) * (size_t)m);
    memset(grad, 0, sizeof(double) * (size_t)D);
    /* lambda_T */
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += 2.0 * Q[r * n + j] * (traj[(size_t)T * n + j] - g[j]);
        lam[r] = s;
    }
    for (int k = T - 1; k >= 0; --k) {
        /* here lam = lambda_{k+1} */
        const double* u = uexp + (size_t)k * m;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += B[r * m + i] * lam[r];
            for (int j = 0; j < m; ++j) s += 2.0 * R[i * m + j] * u[j];
            du[i] = s;
        }
        double c = (double)num[k] / (double)den;
        for (int i = 0; i < m; ++i) {
            grad[i * p + idx1[k]] += (1.0 - c) * du[i];
            if (p > 1) grad[i * p + idx1[k] + 1] += c * du[i];
        }
        if (k >= 1) {
            for (int r = 0; r < n; ++r) {
                double s = 0.0;
                for (int j = 0; j < n; ++j) s += A[j * n + r] * lam[j];
                for (int j = 0; j < n; ++j)
                    s += 2.0 * Q[r * n + j] * (traj[(size_t)k * n + j] - g[j]);
                lam2[r] = s;
            }
            memcpy(lam, lam2, sizeof(double) * (size_t)n);
        }
    }
    free(traj);
    free(uexp);
    free(idx1);
    free(num);
    free(lam);
    free(lam2);
    free(du);
    return J;
}

/* Projected-gradient refinement: `steps` times U <- clip(U - eta dJ/dU).    */
ORC_EXPORT void orc_refine(const double* A, const double* B, const double* Q,
                           const double* R, const double* w, const double* x0,
                           const double* g, const double* umin, const double* umax, int n,
                           int m, int T, int p, int steps, double eta, double* U) {
    int D = m * p;
    double* gr = (double*)malloc(sizeof(double) * (size_t)D);
    for (int s = 0; s < steps; ++s) {
        orc_grad(A, B, Q, R, w, x0, g, U, n, m, T, p, gr);
        for (int q = 0; q < D; ++q) {
            int i = q / p;
            double v = U[q] - eta * gr[q];
            if (v < umin[i]) v = umin[i];
            if (v > umax[i]) v = umax[i];
            U[q] = v;
        }
    }
    free(gr);
}

/* ------------------------------------------------------------------------ */
/* Parent selection (Alg. 1 parent line; Sec. V "taking the numParents U     */
/* arrays with lowest associated costs"): the E smallest costs, ordered by   */
/* (cost, index) ascending; NaN counts as +inf.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    double cost;
    int idx;
} keyed;

static int keyed_cmp(const void* pa, const void* pb) {
    const keyed* a = (const keyed*)pa;
    const keyed* b = (const keyed*)pb;
    if (a->cost < b->cost) return -1;
    if (a->cost > b->cost) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

ORC_EXPORT void orc_select(const double* cost, int P, int E, int* elite_idx) {
    keyed* k = (keyed*)malloc(sizeof(keyed) * (size_t)P);
    for (int c = 0; c < P; ++c) {
        double v = cost[c];
        k[c].cost = isnan(v) ? INFINITY : v;
        k[c].idx = c;
    }
    qsort(k, (size_t)P, sizeof(keyed), keyed_cmp);
    for (int e = 0; e < E; ++e) elite_idx[e] = k[e].idx;
    free(k);
}

/* ------------------------------------------------------------------------ */
/* Zero-order-hold discretization by the matrix exponential (Sec. III-A):    */
/* expm([[Ac, Bc], [0, 0]] dt) = [[Ad, Bd], [0, I]] (Van Loan).  The         */
/* exponential is the Taylor series of the scaled matrix (norm <= 1/2, 30    */
/* terms) followed by repeated squaring.                                     */
/* ------------------------------------------------------------------------ */
static void matmul(const double* X, const double* Y, double* Z, int N) {
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int k = 0; k < N; ++k) s += X[i * N + k] * Y[k * N + j];
            Z[i * N + j] = s;
        }
}

ORC_EXPORT void orc_expm(const double* M, int N, double* out) {
    double norm = 0.0;
    for (int i = 0; i < N; ++i) {
        double r = 0.0;
        for (int j = 0; j < N; ++j) r += fabs(M[i * N + j]);
        if (r > norm) norm = r;
    }
    int s = 0;
    while (norm > 0.5) {
        norm *= 0.5;
        ++s;
    }
    double scale = ldexp(1.0, -s);
    size_t NN = (size_t)N * N;
    double* X = (double*)malloc(sizeof(double) * NN);
    double* term = (double*)malloc(sizeof(double) * NN);
    double* tmp = (double*)malloc(sizeof(double) * NN);
    for (size_t t = 0; t < NN; ++t) X[t] = M[t] * scale;
    for (size_t t = 0; t < NN; ++t) out[t] = 0.0;
    for (int i = 0; i < N; ++i) out[i * N + i] = 1.0;
    memcpy(term, out, sizeof(double) * NN);
    for (int kk = 1; kk <= 30; ++kk) {
        matmul(term, X, tmp, N);
        for (size_t t = 0; t < NN; ++t) term[t] = tmp[t] / (double)kk;
        for (size_t t = 0; t < NN; ++t) out[t] += term[t];
    }
    for (int q = 0; q < s; ++q) {
        matmul(out, out, tmp, N);
        memcpy(out, tmp, sizeof(double) * NN);
    }
    free(X);
    free(term);
    free(tmp);
}

ORC_EXPORT void orc_zoh(const double* Ac, const double* Bc, int n, int m, double dt,
                        double* Ad, double* Bd) {
    int N = n + m;
    double* M = (double*)calloc((size_t)N * N, sizeof(double));
    double* E = (double*)malloc(sizeof(double) * (size_t)N * N);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) M[i * N + j] = Ac[i * n + j] * dt;
        for (int j = 0; j < m; ++j) M[i * N + n + j] = Bc[i * m + j] * dt;
    }
    orc_expm(M, N, E);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) Ad[i * n + j] = E[i * N + j];
        for (int j = 0; j < m; ++j) Bd[i * m + j] = E[i * N + n + j];
    }
    free(M);
    free(E);
}

ORC_EXPORT int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
