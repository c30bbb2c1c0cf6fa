// Rollout + cost with the per-step product on the tensor cores (tcgen05,
// BF16 operands, FP32 accumulation in tensor memory); the knots come bred
// from breed_kernel.
//
// For a tile of 128 candidates the step x_{k+1} = x_k + D x_k + B_d u_k
// (D = A_d - I, Eq. first_order_integration in delta form) is one
// 128 x 128 x 192 contraction per step, accumulated onto the state itself:
//   X[c][i] += sum_{j<64} u_c[j] B_d[i][j] + sum_{k<128} x_c[k] D[i][k].
// The FP32 state X lives in tensor memory for the whole horizon (TMEM lane =
// candidate, column = state): the MMAs add the increment to it, so no thread
// keeps or updates a master copy.  The A operands, bf16(x_c) and bf16(u_c),
// live in tensor memory too (two BF16 per 32-bit column, lane = candidate),
// so the MMAs read only the constant B = [D | B_d] (states x K, K-major,
// 128-byte swizzle) from shared memory, and the epilogue writes its BF16
// state with tcgen05.st instead of shared-memory stores.
//
// Roles.  One thread of a 17th warp issues every MMA.  The 512 threads of
// the other 16 warps are (32-state chunk, candidate) pairs; per step each
//   1. writes its 16 inputs of u_{k+1} (the segment's knots kept in
//      registers) into the spare input buffer while step k's MMAs run,
//   2. waits for step k's MMAs, reads its 32 states of x_{k+1} from X, and
//      signals "X read": the issuer starts step k+1 with the input MMAs
//      (X += u_{k+1} B_d'), which no longer wait for the state,
//   3. rounds the states to BF16 into the state operand and signals "state
//      written": the issuer adds the state MMAs (X += x_{k+1} D') behind them,
//   4. accumulates the stage cost (x_{k+1}-g)' Q (x_{k+1}-g) from registers
//      while those MMAs run.
// So a step's critical path is the product itself plus one TMEM read and one
// BF16 write-back; the stage cost and the inputs overlap the tensor core.
// The input cost sum_k u_k' R u_k is added in closed form from the knots
// (Gram of the knot weights), in FP32.
//
// Precision: D, B_d, x and u enter the product as BF16 (relative rounding
// 2^-9); the accumulation onto the state and the cost stay FP32.  Every
// mbarrier wait is bounded in time (one second unless the handle sets
// another limit): past the limit the kernel sets status bit 2, every thread
// leaves the step loop, the issuer waits (bounded) for its MMAs in flight,
// the tensor memory is freed and the kernel returns.  A host-side injection
// can make the issuer stop at a given step, so that the other threads' waits
// run out (the test of that path).
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
constexpr uint32_t kWaitPolls = 1u << 26;  // the final wait for MMAs in flight
constexpr uint32_t kDefaultWaitUs = 1000000u;
constexpr int kChunks = 4;                     // state column chunks
constexpr int kCW = kKx / kChunks;             // 32 states per chunk
constexpr int kUW = kKu / kChunks;             // 16 inputs per chunk
constexpr int kEpiThreads = kChunks * kTileCands;  // thread = (chunk, candidate row)
constexpr int kEpiWarps = kEpiThreads / 32;        // 16
constexpr int kThreads = kEpiThreads + 32;         // + the issuing warp
static_assert(kCW == 32, "one 32x32b.x32 TMEM access per thread and step");

// Tensor-memory columns (32-bit): the FP32 state, then the BF16 A operand
// (two values per column): the state part, and the input part twice.
constexpr uint32_t kColX = 0;                  // [0, 128)   X, FP32
constexpr uint32_t kColAx = kKx;               // [128, 192) bf16(x), 64 columns
constexpr uint32_t kColAu = kColAx + kKx / 2;  // [192, 256) bf16(u), 2 x 32 columns
constexpr uint32_t kAuCols = kKu / 2;
constexpr uint32_t kTmemCols = 256;
static_assert(kColAu + 2 * kAuCols == kTmemCols, "tensor-memory layout");

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

// D (tensor memory) += A (tensor memory, M x 16) * B (shared memory, 16 x N).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bd,
                                            uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bd), "r"(idesc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The CTA's abort flag (a shared int, by its shared-memory address).
__device__ __forceinline__ int abort_get(uint32_t flag) {
    int v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(flag) : "memory");
    return v;
}
__device__ __forceinline__ void abort_set(uint32_t flag) {
    asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(flag), "r"(1) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// %globaltimer in units of 1.024 us, 32 bits (wraps after 73 minutes; the
// differences taken below are modular).
__device__ __forceinline__ uint32_t global_us() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (uint32_t)(t >> 10);
}

// Wait for phase `parity` of an mbarrier, for at most about limit_us
// microseconds; false if it gave up (and then sets the abort flag) or another
// thread already gave up.  The clock and the flag are read every 256 polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t flag,
                                          uint32_t limit_us) {
    uint32_t t0 = 0;
    for (uint32_t it = 0; it < (1u << 31); ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255) {
            if (abort_get(flag)) return false;
            const uint32_t t = global_us();
            if (it == 255) t0 = t;
            else if (t - t0 > limit_us) break;
        }
    }
    abort_set(flag);
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

__device__ __forceinline__ void tmem_st16(uint32_t addr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15,%16};" ::"r"(addr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(addr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ float4 lds4(uint32_t saddr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(saddr));
    return v;
}

// Paired FP32 add and multiply (round to nearest, sm_100 and later).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Two values rounded to BF16 in one 32-bit word, the first in the low half
// (the lower K index, as in a K-major operand row).
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
template <int W>
__device__ __forceinline__ float input_cost_dense_rows(const RolloutArgs& a, int cand, int i0,
                                                       int i1) {
    const int p = a.p, m = a.m;
    float y[W], yp[W], up[W];
#pragma unroll
    for (int r = 0; r < W; ++r) yp[r] = up[r] = 0.0f;
    float s = 0.0f;
    for (int j = 0; j < p; ++j) {
#pragma unroll
        for (int r = 0; r < W; ++r) y[r] = 0.0f;
        for (int l = 0; l < m; ++l) {
            const float ul = __ldcg(a.pop_in + (size_t)(l * p + j) * a.P + cand);
#pragma unroll
            for (int r = 0; r < W; ++r)
                if (i0 + r < i1) y[r] = fmaf(a.rmat[l * m + i0 + r], ul, y[r]);
        }
#pragma unroll
        for (int r = 0; r < W; ++r) {
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
    static constexpr int kB = 0;                       // B = [D | B_d], rows = states
    static constexpr int kG = kOperandBytes;           // goal [128] f32
    static constexpr int kQ = kG + 128 * 4;            // diag Q [128] f32
    static constexpr int kKnots = kQ + 128 * 4;        // KnotStep[T]
    __host__ __device__ static int part(int T) { return kKnots + 16 * T; }  // f32[4][128]
    __host__ __device__ static int total(int T) {
        return part(T) + 4 * kChunks * kTileCands + 1024;
    }
};

__global__ void __launch_bounds__(kThreads, 1) rollout_bf16_kernel(const RolloutArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t* sB = sm + Bf16Layout::kB;
    float* sg = reinterpret_cast<float*>(sm + Bf16Layout::kG);
    float* sq = reinterpret_cast<float*>(sm + Bf16Layout::kQ);
    KnotStep* ks = reinterpret_cast<KnotStep*>(sm + Bf16Layout::kKnots);
    float* spart = reinterpret_cast<float*>(sm + Bf16Layout::part(a.T));
    // bar_in: X read and u_{k+1} written (16 warp arrivals); bar_x: bf16(x_{k+1})
    // written (16); bar_mma: the step's MMAs completed (one commit)
    __shared__ __align__(8) uint64_t bar_in, bar_x, bar_mma;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const uint32_t abort_f = smem_u32(&abort_sh);
    const uint32_t b_in = smem_u32(&bar_in), b_x = smem_u32(&bar_x), b_mma = smem_u32(&bar_mma);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer_warp = warp == kEpiWarps;
    const int q = warp >> 2;                         // state chunk / input chunk of this thread
    const int row = ((warp & 3) << 5) | lane;        // candidate row = TMEM lane
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
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_in)),
                     "r"(kEpiWarps));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_x)),
                     "r"(kEpiWarps));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_mma)));
        abort_sh = 0;
    }
    // B was written by ordinary stores and is read by the MMAs (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    // ---- the knots (bred by the previous kernel) are read only after it completed
    pdl_wait_primary();
    tc_fence_before();
    __syncthreads();  // TMEM base, barriers and operand B published
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    float jown = 0.0f;
    int last_commit = -1;  // issuer: last step whose MMAs were committed
    const int stall_step = a.inject ? a.inject[0] : -1;
    const uint32_t wait_us = a.inject ? (uint32_t)a.inject[1] : kDefaultWaitUs;

    if (issuer_warp) {
        // ---- the MMA issuer: step k = inputs u_k (after X was read), then the
        // state x_k (after its BF16 copy was written), one commit per step
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kKx);
            const uint64_t bd0 = sdesc(smem_u32(sB));
            for (int k = 0; k < T; ++k) {
                if (k == stall_step) break;  // injected stall: the step is never issued
                if (!mbar_wait(b_in, (uint32_t)(k & 1), abort_f, wait_us)) break;
                tc_fence_after();
                const uint32_t au = tmem + kColAu + (uint32_t)(k & 1) * kAuCols;
#pragma unroll
                for (int jj = 0; jj < kKu / 16; ++jj) {
                    const int kk = kKx / 16 + jj;  // K slice of B_d within B
                    const uint32_t off = ((kk >> 2) * kAtomBytes + (kk & 3) * 32) >> 4;
                    mma_bf16_ts(tmem + kColX, au + 8 * jj, bd0 + off, idesc);
                }
                if (!mbar_wait(b_x, (uint32_t)(k & 1), abort_f, wait_us)) {
                    mma_commit(b_mma);  // track the input MMAs already issued
                    last_commit = k;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < kKx / 16; ++kk) {
                    const uint32_t off = ((kk >> 2) * kAtomBytes + (kk & 3) * 32) >> 4;
                    mma_bf16_ts(tmem + kColX, tmem + kColAx + 8 * kk, bd0 + off, idesc);
                }
                mma_commit(b_mma);
                last_commit = k;
            }
            // MMAs still in flight are waited for (bounded) before the
            // tensor memory is freed
            if (last_commit >= 0) {
                bool done = false;
                for (uint32_t it = 0; it < kWaitPolls && !done; ++it)
                    done = mbar_try(b_mma, (uint32_t)(last_commit & 1));
                if (!done) abort_set(abort_f);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue threads: (chunk q, candidate row)
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const float* src = a.pop_in;
        const bool live = cand < a.P;
        const int i0 = q * kUW;
        int seg = -1;
        float Ju = 0.0f;  // input cost of own inputs, closed form, accumulated per segment
        // U_s and U_s+1 of this thread's inputs into its knot columns
        float u[2 * kUW];  // [0, 16) = U_s, [16, 32) = U_s+1 of the current segment
        auto load_segment = [&](int s) {
#pragma unroll
            for (int j = 0; j < kUW; ++j) {
                const int i = i0 + j;
                u[j] = (live && i < m) ? __ldcg(src + (size_t)(i * p + s) * a.P + cand) : 0.0f;
                u[kUW + j] = (live && i < m && s + 1 < p)
                                 ? __ldcg(src + (size_t)(i * p + s + 1) * a.P + cand)
                                 : 0.0f;
            }
            // segments come in order, each once (knots <= horizon): W_ss U_s^2 +
            // 2 W_s,s+1 U_s U_s+1, plus W_{p-1,p-1} U_{p-1}^2 with the last segment
            // (diagonal R; a dense R is taken after the horizon loop)
            if (!a.rmat) {
                const float wd = a.gram[s];
                const float wo = s + 1 < p ? 2.0f * a.gram[p + s] : 0.0f;
                const float wl = s + 2 == p ? a.gram[s + 1] : 0.0f;
#pragma unroll
                for (int j = 0; j < kUW; ++j) {
                    if (i0 + j < m) {
                        const float ua = u[j], ub = u[kUW + j];
                        float t = wd * ua * ua;
                        t = fmaf(wo * ua, ub, t);
                        t = fmaf(wl * ub, ub, t);
                        Ju = fmaf(a.rdiag[i0 + j], t, Ju);
                    }
                }
            }
        };
        // this thread's 16 inputs of u_k, BF16, into input buffer `buf`
        auto write_input = [&](int buf, const KnotStep& st) {
            if (st.idx1 != seg) {
                seg = st.idx1;
                load_segment(seg);
            }
            uint32_t w[kUW / 2];
#pragma unroll
            for (int j = 0; j < kUW / 2; ++j)
                w[j] = pack_bf16(fmaf(st.w1, u[kUW + 2 * j], st.w0 * u[2 * j]),
                                 fmaf(st.w1, u[kUW + 2 * j + 1], st.w0 * u[2 * j + 1]));
            tmem_st8(lane_base + kColAu + (uint32_t)buf * kAuCols + (uint32_t)(q * kUW / 2), w);
        };
        auto write_state = [&](const float (&x)[kCW]) {
            uint32_t w[kCW / 2];
#pragma unroll
            for (int j = 0; j < kCW / 2; ++j) w[j] = pack_bf16(x[2 * j], x[2 * j + 1]);
            tmem_st16(lane_base + kColAx + (uint32_t)(q * kCW / 2), w);
        };
        // publish this warp's tensor-memory stores to the issuer
        auto signal = [&](uint32_t bar) {
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar);
        };

        // initial state: FP32 into X, BF16 into the state operand, u_0
        {
            float x0[kCW];
#pragma unroll
            for (int j = 0; j < kCW; ++j) {
                const int i = q * kCW + j;
                x0[j] = i < n ? a.x0[i] : 0.0f;
            }
            tmem_st32(lane_base + kColX + q * kCW, x0);
            write_state(x0);
            write_input(0, ks[0]);
            signal(b_in);
            __syncwarp();
            if (lane == 0) mbar_arrive(b_x);
        }

        float2 jacc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        const uint32_t g_s = smem_u32(sg + q * kCW), q_s = smem_u32(sq + q * kCW);
        auto stage_cost = [&](const float (&x)[kCW]) {
#pragma unroll
            for (int j = 0; j < kCW; j += 4) {
                // goal and weights re-read every step (volatile: not hoisted
                // into 64 registers across the loop)
                const float4 gg = lds4(g_s + 4 * j), qq = lds4(q_s + 4 * j);
                const float2 e01 = add2(make_float2(x[j], x[j + 1]), make_float2(-gg.x, -gg.y));
                const float2 e23 =
                    add2(make_float2(x[j + 2], x[j + 3]), make_float2(-gg.z, -gg.w));
                jacc[0] = fma2(mul2(make_float2(qq.x, qq.y), e01), e01, jacc[0]);
                jacc[1] = fma2(mul2(make_float2(qq.z, qq.w), e23), e23, jacc[1]);
            }
            // the sums are complete here: the next step's TMEM accesses (asm
            // volatile, kept in order) cannot overlap the state's registers
            asm volatile("" : "+f"(jacc[0].x), "+f"(jacc[0].y), "+f"(jacc[1].x), "+f"(jacc[1].y));
        };
        for (int k = 0; k < T; ++k) {
            // inputs of step k+1 into the buffer step k-1's MMAs read (completed)
            if (k + 1 < T) write_input((k + 1) & 1, ks[k + 1]);
            if (!mbar_wait(b_mma, (uint32_t)(k & 1), abort_f, wait_us)) break;
            tc_fence_after();
            float x[kCW];
            tmem_ld32(lane_base + kColX + q * kCW, x);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (k + 1 < T) {
                signal(b_in);  // X read, u_{k+1} written: the input MMAs may start
                write_state(x);
                signal(b_x);   // bf16(x_{k+1}) written: the state MMAs may start
            }
            stage_cost(x);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        if (a.rmat && live) {
            // two halves of 8 rows keep the register count down
            const int i1 = min(i0 + kUW, m), im = min(i0 + kUW / 2, i1);
            Ju = input_cost_dense_rows<kUW / 2>(a, cand, i0, im) +
                 input_cost_dense_rows<kUW / 2>(a, cand, im, i1);
        }
        jown = Ju;
#pragma unroll
        for (int j = 0; j < 2; ++j) jown += jacc[j].x + jacc[j].y;
        spart[q * kTileCands + row] = jown;
    }
    tc_fence_before();
    __syncthreads();
    if (abort_get(abort_f)) {
        if (tid == 0 && a.status) atomicOr(a.status, 2);
    } else if (!issuer_warp && q == 0 && cand < a.P) {
        float J = spart[row];
#pragma unroll
        for (int c = 1; c < kChunks; ++c) J += spart[c * kTileCands + row];
        a.cost[cand] = finite_or_inf(J);
    }
    tc_fence_after();
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

cudaError_t launch_rollout_bf16(const RolloutArgs& a, cudaStream_t st) {
    if (!rollout_bf16_supported(a.n, a.m, a.T)) return cudaErrorInvalidConfiguration;
    if (a.mode != kEval) return cudaErrorInvalidValue;  // breeding runs in breed_kernel
    auto kern = rollout_bf16_kernel;
    const size_t smem = rollout_bf16_smem_bytes(a.T);
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    const int grid = (a.P - a.cand_begin + kTileCands - 1) / kTileCands;
    if (grid <= 0) return cudaSuccess;
    return launch_kernel(kern, dim3(grid), dim3(kThreads), smem, st, a.pdl != 0, a);
}

}  // namespace empc
