// Rollout + cost with the per-step product on the tensor cores (tcgen05,
// BF16 operands, FP32 accumulation in tensor memory); the knots come bred
// from breed_kernel.
//
// For a tile of 128 candidates the step x_{k+1} = x_k + D x_k + B_d u_k
// (D = A_d - I, Eq. first_order_integration in delta form) is one
// 128 x 128 x 192 contraction per step, accumulated onto the state itself:
//   X[c][i] += sum_{k<128} x_c[k] D[i][k] + sum_{j<64} u_c[j] B_d[i][j],
// with A = [x_c | u_c] (candidates x K, BF16) and B = [D | B_d] (states x K,
// BF16, constant), both K-major with the 128-byte swizzle in shared memory.
// The FP32 state X lives in tensor memory for the whole horizon (TMEM lane =
// candidate, column = state): the MMA adds the increment to it, so no thread
// keeps or updates a master copy.  Each step runs as four N = 32 column
// chunks of threads; the product is issued as NG MMA groups of N = 128 / NG
// columns (NG = 1, 2 or 4, chosen by the autotuner), each committed to its
// own mbarrier, and the 512 threads are (chunk, candidate) pairs.  A thread waits for its chunk, reads its 32 states of
// x_{k+1}, accumulates their stage cost (x_{k+1}-g)' Q (x_{k+1}-g), rounds
// them to BF16 into the next step's A row, and writes its 16 inputs of
// u_{k+1} (knots kept in registers per segment).  A is double-buffered, so
// the early chunks' epilogues overlap the later chunks' MMAs.  The input cost
// sum_k u_k' R u_k is added in closed form from the knots (Gram of the knot
// weights), in FP32.
//
// Precision: D, B_d, x and u enter the product as BF16 (relative rounding
// 2^-9); the accumulation onto the state and the cost stay FP32.  Every
// mbarrier wait is bounded: past the limit the kernel sets status bit 2,
// leaves the step loop, waits (bounded) for its MMAs in flight, frees its
// tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

constexpr int kTileCands = 128;  // M: candidates per CTA (TMEM lanes)
constexpr int kKx = 128;         // K columns for the state (n padded)
constexpr int kKu = 64;          // K columns for the input (m padded)
constexpr int kK = kKx + kKu;    // 192
constexpr int kAtomBytes = 128 * 128;  // one 64-column swizzle atom of 128 rows
constexpr int kOperandBytes = 3 * kAtomBytes;  // 128 rows x 192 BF16
constexpr uint32_t kTmemCols = 128;    // the state (accumulator)
constexpr long long kWaitPolls = 1ll << 26;
constexpr int kChunks = 4;                     // state column chunks, one MMA group each
constexpr int kCW = kKx / kChunks;             // 32 states per chunk
constexpr int kUW = kKu / kChunks;             // 16 inputs per chunk
constexpr int kThreads = kChunks * kTileCands; // thread = (chunk, candidate row)
static_assert(kCW == 32, "one 32x32b.x32 TMEM access per thread and step");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row r, column k) in a K-major 128-row operand with
// the 128-byte swizzle: 64-column atoms of 128 rows x 128 B, 16-byte chunks
// xor-ed with the row within its group of 8.
__host__ __device__ __forceinline__ uint32_t swz(int r, int k) {
    return (uint32_t)((k >> 6) * kAtomBytes + r * 128 + ((((k & 63) >> 3) ^ (r & 7)) << 4) +
                      ((k & 7) << 1));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < kWaitPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(addr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st32(uint32_t addr, const float (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(
            addr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}

// Paired FP32 add and multiply (round to nearest, sm_100 and later).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Store 8 consecutive K values (BF16) of row r starting at column k (k % 8 == 0).
__device__ __forceinline__ void put8(uint8_t* op, int r, int k, const float* v) {
    uint4 q;
    q.x = pack_bf16(v[0], v[1]);
    q.y = pack_bf16(v[2], v[3]);
    q.z = pack_bf16(v[4], v[5]);
    q.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(op + swz(r, k)) = q;
}

// Input cost rows i0 .. i1-1 of candidate `cand` for a dense R: sum over
// those rows of U_i' W y_i, y_i,a = (R U_a)_i (the knots read from the
// population, coherent with the breeding kernel before this one).  R is
// symmetric, so row l of R gives column l's weights for every own row.
__device__ __forceinline__ float input_cost_dense_rows(const RolloutArgs& a, int cand, int i0,
                                                       int i1) {
    const int p = a.p, m = a.m;
    float y[kUW], yp[kUW], up[kUW];
#pragma unroll
    for (int r = 0; r < kUW; ++r) yp[r] = up[r] = 0.0f;
    float s = 0.0f;
    for (int j = 0; j < p; ++j) {
#pragma unroll
        for (int r = 0; r < kUW; ++r) y[r] = 0.0f;
        for (int l = 0; l < m; ++l) {
            const float ul = __ldcg(a.pop_in + (size_t)(l * p + j) * a.P + cand);
#pragma unroll
            for (int r = 0; r < kUW; ++r)
                if (i0 + r < i1) y[r] = fmaf(a.rmat[l * m + i0 + r], ul, y[r]);
        }
#pragma unroll
        for (int r = 0; r < kUW; ++r) {
            if (i0 + r >= i1) continue;
            const float u = __ldcg(a.pop_in + (size_t)((i0 + r) * p + j) * a.P + cand);
            s = fmaf(a.gram[j] * u, y[r], s);
            if (j > 0) s = fmaf(a.gram[p + j - 1], fmaf(up[r], y[r], u * yp[r]), s);
            yp[r] = y[r];
            up[r] = u;
        }
    }
    return s;
}

struct Bf16Layout {
    static constexpr int kA0 = 0;                      // A buffer 0
    static constexpr int kA1 = kOperandBytes;          // A buffer 1
    static constexpr int kB = 2 * kOperandBytes;       // B = [D | B_d]
    static constexpr int kG = 3 * kOperandBytes;       // goal [128] f32
    static constexpr int kQ = kG + 128 * 4;            // diag Q [128] f32
    static constexpr int kKnots = kQ + 128 * 4;        // KnotStep[T]
    __host__ __device__ static int par(int T) { return kKnots + 16 * T; }  // int[2*128]
    __host__ __device__ static int part(int T) { return par(T) + 8 * kTileCands; }  // f32[4][128]
    __host__ __device__ static int total(int T) {
        return part(T) + 4 * kChunks * kTileCands + 1024;
    }
};

// NG: the product issued as NG MMA groups of N = 128 / NG, each committed
// to its own mbarrier (the autotuner picks NG).
template <int NG>
__global__ void __launch_bounds__(kThreads, 1) rollout_bf16_kernel(const RolloutArgs a) {
    static_assert(NG == 1 || NG == 2 || NG == 4, "MMA groups");
    constexpr int kGW = kKx / NG;  // columns (states) per MMA group
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sA[2] = {sm + Bf16Layout::kA0, sm + Bf16Layout::kA1};
    uint8_t* sB = sm + Bf16Layout::kB;
    float* sg = reinterpret_cast<float*>(sm + Bf16Layout::kG);
    float* sq = reinterpret_cast<float*>(sm + Bf16Layout::kQ);
    KnotStep* ks = reinterpret_cast<KnotStep*>(sm + Bf16Layout::kKnots);
    int* par = reinterpret_cast<int*>(sm + Bf16Layout::par(a.T));
    float* spart = reinterpret_cast<float*>(sm + Bf16Layout::part(a.T));
    __shared__ __align__(8) uint64_t mbar[kChunks];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int q = warp >> 2;                         // state chunk / input chunk of this thread
    const int row = ((warp & 3) << 5) | (tid & 31);  // candidate row = TMEM lane
    const int n = a.n, m = a.m, p = a.p, T = a.T;
    const int c0 = a.cand_begin + blockIdx.x * kTileCands;
    const int cand = c0 + row;
    pdl_launch_dependents();

    // ---- constant operand B = [D | B_d] (rows = states), goal, Q, knot table
    for (int idx = tid; idx < 128 * (kK / 8); idx += blockDim.x) {
        const int i = idx / (kK / 8), k0 = (idx % (kK / 8)) * 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e;
            float x = 0.0f;
            if (i < n) {
                if (k < kKx) x = k < n ? a.D[i * n + k] : 0.0f;
                else if (k - kKx < m) x = a.BT[(k - kKx) * n + i];
            }
            v[e] = x;
        }
        put8(sB, i, k0, v);
    }
    for (int i = tid; i < 128; i += blockDim.x) {
        sg[i] = i < n ? a.goal[i] : 0.0f;
        sq[i] = i < n ? a.qdiag[i] : 0.0f;
    }
    for (int k = tid; k < T; k += blockDim.x) ks[k] = a.ktab[k];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
#pragma unroll
        for (int g = 0; g < NG; ++g)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[g])));
        abort_sh = 0;
    }

    // ---- the knots (bred by the previous kernel) are read only after it completed
    pdl_wait_primary();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM base published
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const float* src = a.pop_in;
    const bool live = cand < a.P;

    // ---- initial state: FP32 into this thread's chunk of its TMEM lane, BF16 into A[0]
    {
        float x0[kCW];
#pragma unroll
        for (int j = 0; j < kCW; ++j) {
            const int i = q * kCW + j;
            x0[j] = i < n ? a.x0[i] : 0.0f;
        }
        tmem_st32(lane_base + q * kCW, x0);
#pragma unroll
        for (int j = 0; j < kCW; j += 8) put8(sA[0], row, q * kCW + j, x0 + j);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    // knots of the current segment (this thread's chunk of the inputs)
    float ua[kUW], ub[kUW];
    const int i0 = q * kUW;
    int seg = -1;
    float Ju = 0.0f;  // input cost of own inputs, closed form, accumulated per segment
    auto load_segment = [&](int s) {
#pragma unroll
        for (int j = 0; j < kUW; ++j) {
            const int i = i0 + j;
            ua[j] = (live && i < m) ? __ldcg(src + (size_t)(i * p + s) * a.P + cand) : 0.0f;
            ub[j] = (live && i < m && s + 1 < p) ? __ldcg(src + (size_t)(i * p + s + 1) * a.P + cand)
                                                  : 0.0f;
        }
        // segments come in order, each once: W_ss U_s^2 + 2 W_s,s+1 U_s U_s+1,
        // plus W_{p-1,p-1} U_{p-1}^2 with the last segment (diagonal R; a dense
        // R is taken after the horizon loop)
        if (a.rmat) return;
        const float wd = a.gram[s];
        const float wo = s + 1 < p ? 2.0f * a.gram[p + s] : 0.0f;
        const float wl = s + 2 == p ? a.gram[s + 1] : 0.0f;
#pragma unroll
        for (int j = 0; j < kUW; ++j) {
            if (i0 + j < m) {
                float t = wd * ua[j] * ua[j];
                t = fmaf(wo * ua[j], ub[j], t);
                t = fmaf(wl * ub[j], ub[j], t);
                Ju = fmaf(a.rdiag[i0 + j], t, Ju);
            }
        }
    };
    auto write_input = [&](uint8_t* op, const KnotStep& st) {
        if (st.idx1 != seg) {
            seg = st.idx1;
            load_segment(seg);
        }
#pragma unroll
        for (int j = 0; j < kUW; j += 8) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = fmaf(st.w1, ub[j + e], st.w0 * ua[j + e]);
            put8(op, row, kKx + i0 + j, v);
        }
    };
    write_input(sA[0], ks[0]);

    float2 jacc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                      make_float2(0.f, 0.f)};
    bool ok = true;
    int issued = -1;  // last step whose MMAs the issuing thread committed
    const float4* g4 = reinterpret_cast<const float4*>(sg + q * kCW);
    const float4* q4 = reinterpret_cast<const float4*>(sq + q * kCW);
    auto stage_cost = [&](const float (&x)[kCW]) {
#pragma unroll
        for (int j = 0; j < kCW; j += 4) {
            const float4 gg = g4[j / 4], qq = q4[j / 4];
            const float2 e01 = add2(make_float2(x[j], x[j + 1]), make_float2(-gg.x, -gg.y));
            const float2 e23 = add2(make_float2(x[j + 2], x[j + 3]), make_float2(-gg.z, -gg.w));
            jacc[(j / 4) & 3] = fma2(mul2(make_float2(qq.x, qq.y), e01), e01, jacc[(j / 4) & 3]);
            jacc[(j / 4) & 3] = fma2(mul2(make_float2(qq.z, qq.w), e23), e23, jacc[(j / 4) & 3]);
        }
    };
    const uint32_t idesc = idesc_bf16(kGW);
    const int grp = q * NG / kChunks;  // the MMA group holding this thread's chunk
    for (int k = 0; k < T; ++k) {
        uint8_t* Acur = sA[k & 1];
        uint8_t* Anext = sA[(k + 1) & 1];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (!__syncthreads_and(ok)) break;  // every thread leaves together
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // descriptors advance by (byte offset >> 4) in their start-address field;
            // group g uses rows g*kGW .. of B (rows of 128 B within each atom)
            const uint64_t ad0 = sdesc(smem_u32(Acur)), bd0 = sdesc(smem_u32(sB));
#pragma unroll
            for (int g = 0; g < NG; ++g) {
#pragma unroll
                for (int kk = 0; kk < kK / 16; ++kk) {
                    const uint32_t off = ((kk >> 2) * kAtomBytes + (kk & 3) * 32) >> 4;
                    mma_bf16(tmem + g * kGW, ad0 + off, bd0 + off + ((g * kGW * 128) >> 4),
                             idesc, 1u);
                }
                mma_commit(&mbar[g]);
            }
            issued = k;
        }
        // off the critical path: this thread's inputs of u_{k+1}, while the MMAs
        // run (Anext was last read by the previous step's MMAs, which have completed)
        if (k + 1 < T) write_input(Anext, ks[k + 1]);
        if (!mbar_wait(&mbar[grp], (uint32_t)(k & 1))) {
            ok = false;
            continue;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float x[kCW];
        tmem_ld32(lane_base + q * kCW, x);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        stage_cost(x);
        if (k + 1 < T) {
#pragma unroll
            for (int j = 0; j < kCW; j += 8) put8(Anext, row, q * kCW + j, x + j);
        }
    }
    // an abandoned step may still have MMAs in flight: wait (bounded) for them
    // before the tensor memory is freed
    if (tid == 0 && issued >= 0) {
#pragma unroll
        for (int g = 0; g < NG; ++g)
            if (!mbar_wait(&mbar[g], (uint32_t)(issued & 1))) ok = false;
    }
    if (!ok) abort_sh = 1;
    if (a.rmat && live) Ju = input_cost_dense_rows(a, cand, i0, min(i0 + kUW, m));
    float jown = Ju;
#pragma unroll
    for (int j = 0; j < 4; ++j) jown += jacc[j].x + jacc[j].y;
    spart[q * kTileCands + row] = jown;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_sh) {
        if (tid == 0 && a.status) atomicOr(a.status, 2);
    } else if (live && q == 0) {
        float J = spart[row];
#pragma unroll
        for (int c = 1; c < kChunks; ++c) J += spart[c * kTileCands + row];
        a.cost[cand] = finite_or_inf(J);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

}  // namespace

size_t rollout_bf16_smem_bytes(int T) { return (size_t)Bf16Layout::total(T); }

int rollout_bf16_threads() { return kThreads; }

bool rollout_bf16_supported(int n, int m, int T) {
    return n <= kKx && m <= kKu && rollout_bf16_smem_bytes(T) <= 227u * 1024u;
}

template <int NG>
cudaError_t launch_groups(const RolloutArgs& a, cudaStream_t st) {
    auto kern = rollout_bf16_kernel<NG>;
    const size_t smem = rollout_bf16_smem_bytes(a.T);
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    const int grid = (a.P - a.cand_begin + kTileCands - 1) / kTileCands;
    if (grid <= 0) return cudaSuccess;
    return launch_kernel(kern, dim3(grid), dim3(kThreads), smem, st, a.pdl != 0, a);
}

cudaError_t launch_rollout_bf16(const RolloutArgs& a, int groups, cudaStream_t st) {
    if (!rollout_bf16_supported(a.n, a.m, a.T)) return cudaErrorInvalidConfiguration;
    if (a.mode != kEval) return cudaErrorInvalidValue;  // breeding runs in breed_kernel
    switch (groups) {
        case 1: return launch_groups<1>(a, st);
        case 2: return launch_groups<2>(a, st);
        case 4: return launch_groups<4>(a, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace empc
