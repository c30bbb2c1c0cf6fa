// Condensed quadratic-form costs on the tensor cores (Sec. IV-B, IV-E):
//   J(U) = U' H U + g' U + c0
// for a population of knot vectors U (D = m p knots each).  The population
// product Y = U' H (candidates x knots) is one dense contraction of
// P x D x D, run as tcgen05 MMAs of kind::tf32 with FP32 accumulation in
// tensor memory; the per-candidate cost J_c = sum_q U_qc (Y_cq + g_q) + c0 is
// then taken in FP32 from the accumulator row.
//
// Precision: TF32 keeps 10 explicit mantissa bits, so each operand is split
// into a TF32 head and the FP32 remainder (x = hi + lo, hi rounded to TF32,
// lo = x - hi exact in FP32 and read by the tensor core to TF32), and the
// product is accumulated as hi*hi + hi*lo + lo*hi.  The dropped lo*lo term
// and the truncation of lo are below 2^-20 of each product, about the
// rounding of an FP32 dot product of this length.
//
// Tile: a CTA owns M = 128 candidates (TMEM lanes) and all N = Dp output
// columns (Dp <= 256, TMEM columns); K = Dp runs in chunks of 32 (one
// 128-byte swizzle atom of FP32 per row), double-buffered: while the MMAs of
// one chunk run, the 256 threads stage the next (the candidates' knots
// transposed to K-major rows, and the matching 32 columns of H, each split
// into head and remainder).  Every mbarrier wait is bounded: past the limit
// the kernel sets status bit 2, waits (bounded) for its MMAs in flight,
// frees its tensor memory and returns.
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

constexpr int kM = 128;                 // candidates per CTA (TMEM lanes)
constexpr int kKC = 32;                 // K elements per chunk (128 bytes of FP32)
constexpr int kThreadsTC = 256;
constexpr int kMaxN = 256;              // output columns (Dp) in one MMA
constexpr int kABytes = kM * 128;       // one operand chunk of 128 rows
constexpr long long kPolls = 1ll << 26;

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row r, k) of a K-major operand chunk with the
// 128-byte swizzle (one atom column, 32 FP32 per row, 8-row groups of 1 KB,
// 16-byte units xor-ed with the row within its group).
__device__ __forceinline__ uint32_t swz32(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 2) & 7) ^ (r & 7)) << 4) + ((k & 3) << 2));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: TF32 x TF32 -> FP32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_tf32(uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit_to(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            saddr(bar))
        : "memory");
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity) {
    for (long long it = 0; it < kPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_load32(uint32_t addr, float (&v)[32]) {
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

// Head of x rounded to TF32 (10 explicit mantissa bits, ties away from zero
// on the magnitude); the remainder x - head is exact in FP32.
__device__ __forceinline__ float tf32_head(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Shared layout (bytes from a 1024-aligned base): two stages of
// [A head | A rem | B head | B rem], then g [Dp] FP32.
struct TcLayout {
    int n;  // Dp
    __host__ __device__ explicit TcLayout(int dp) : n(dp) {}
    __host__ __device__ int b_bytes() const { return n * 128; }
    __host__ __device__ int stage_bytes() const { return 2 * kABytes + 2 * b_bytes(); }
    __host__ __device__ int a(int s, int part) const { return s * stage_bytes() + part * kABytes; }
    __host__ __device__ int b(int s, int part) const {
        return s * stage_bytes() + 2 * kABytes + part * b_bytes();
    }
    __host__ __device__ int g() const { return 2 * stage_bytes(); }
    __host__ __device__ int total() const { return g() + 4 * n + 1024; }
};

__global__ void __launch_bounds__(kThreadsTC, 1) condensed_tc_kernel(const CondArgs a, int* status) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* sm = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    const int Dp = a.Dp, D = a.D, P = a.P;
    const TcLayout L(Dp);
    float* gs = reinterpret_cast<float*>(sm + L.g());
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int c0 = blockIdx.x * kM;
    const uint32_t ncols = Dp <= 32 ? 32u : Dp <= 64 ? 64u : Dp <= 128 ? 128u : 256u;
    pdl_launch_dependents();
    for (int q = tid; q < Dp; q += kThreadsTC) gs[q] = a.g[q];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(&tmem_base_sh)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[1])));
        abort_sh = 0;
    }
    pdl_wait_primary();  // the knots come from the breeding kernel
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;
    const uint32_t idesc = idesc_tf32((uint32_t)Dp);
    const int nchunks = Dp / kKC;
    bool ok = true;
    int uses[2] = {0, 0};  // commits per stage so far (issuing thread's count)
    int waited[2] = {0, 0};
    for (int kc = 0; kc < nchunks; ++kc) {
        const int s = kc & 1;
        // the stage's previous MMAs (chunk kc - 2) must be done before it is rewritten
        if (kc >= 2) {
            if (!wait_parity(&mbar[s], (uint32_t)(waited[s] & 1))) ok = false;
            ++waited[s];
        }
        if (!__syncthreads_and(ok)) break;
        // A: candidates' knots of this chunk, K-major rows (thread: one row,
        // half the chunk's 8 units of 4 knots)
        {
            const int r = tid & (kM - 1), half = tid >> 7;
            const int c = c0 + r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int kk = (half * 4 + u) * 4;  // chunk-relative knot of the unit
                float hv[4], lv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int q = kc * kKC + kk + e;
                    const float x = (q < D && c < P) ? __ldcg(a.pop + (size_t)q * P + c) : 0.0f;
                    hv[e] = tf32_head(x);
                    lv[e] = x - hv[e];
                }
                *reinterpret_cast<float4*>(sm + L.a(s, 0) + swz32(r, kk)) =
                    make_float4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<float4*>(sm + L.a(s, 1) + swz32(r, kk)) =
                    make_float4(lv[0], lv[1], lv[2], lv[3]);
            }
        }
        // B: columns [32 kc, 32 kc + 32) of H for every output row q (H is
        // symmetric and zero-padded to Dp)
        for (int f = tid; f < Dp * (kKC / 4); f += kThreadsTC) {
            const int q = f / (kKC / 4), kk = (f % (kKC / 4)) * 4;
            const float4 h = __ldg(reinterpret_cast<const float4*>(a.H + (size_t)q * Dp +
                                                                   kc * kKC + kk));
            const float hv[4] = {h.x, h.y, h.z, h.w};
            float hh[4], hl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                hh[e] = tf32_head(hv[e]);
                hl[e] = hv[e] - hh[e];
            }
            *reinterpret_cast<float4*>(sm + L.b(s, 0) + swz32(q, kk)) =
                make_float4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<float4*>(sm + L.b(s, 1) + swz32(q, kk)) =
                make_float4(hl[0], hl[1], hl[2], hl[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ah = sdesc_sw128(saddr(sm + L.a(s, 0)));
            const uint64_t al = sdesc_sw128(saddr(sm + L.a(s, 1)));
            const uint64_t bh = sdesc_sw128(saddr(sm + L.b(s, 0)));
            const uint64_t bl = sdesc_sw128(saddr(sm + L.b(s, 1)));
#pragma unroll
            for (int ks = 0; ks < kKC / 8; ++ks) {
                const uint32_t off = (uint32_t)(ks * 32) >> 4;  // 8 TF32 = 32 bytes of K
                const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
                mma_tf32(tmem, ah + off, bh + off, idesc, acc0);
                mma_tf32(tmem, ah + off, bl + off, idesc, 1u);
                mma_tf32(tmem, al + off, bh + off, idesc, 1u);
            }
            commit_to(&mbar[s]);
        }
        ++uses[s];
    }
    // wait for every chunk's MMAs still in flight (bounded)
    for (int s = 0; s < 2; ++s)
        while (waited[s] < uses[s]) {
            if (!wait_parity(&mbar[s], (uint32_t)(waited[s] & 1))) {
                ok = false;
                break;
            }
            ++waited[s];
        }
    if (!ok) abort_sh = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (abort_sh) {
        if (tid == 0 && status) atomicOr(status, 2);
    } else if (warp < 4) {
        // epilogue: thread = candidate row (its warp's TMEM lane quarter)
        const int r = warp * 32 + (tid & 31);
        const int c = c0 + r;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        float J = 0.0f;
        for (int cb = 0; cb < Dp; cb += 32) {
            float y[32];
            tmem_load32(lane_base + (uint32_t)cb, y);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int q = cb + j;
                const float u = (q < D && c < P) ? __ldcg(a.pop + (size_t)q * P + c) : 0.0f;
                J = fmaf(u, y[j] + gs[q], J);
            }
        }
        if (c < P) a.cost[c] = finite_or_inf(J + *a.c0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(ncols));
}

}  // namespace

bool condensed_tc_supported(int Dp) { return Dp >= 32 && Dp <= kMaxN && Dp % 32 == 0; }

size_t condensed_tc_smem_bytes(int Dp) { return (size_t)TcLayout(Dp).total(); }

cudaError_t launch_condensed_tc(const CondArgs& a, int* status, cudaStream_t st, bool pdl) {
    if (!condensed_tc_supported(a.Dp)) return cudaErrorInvalidValue;
    if (a.P <= 0) return cudaSuccess;
    const size_t smem = condensed_tc_smem_bytes(a.Dp);
    if (smem > 227u * 1024u) return cudaErrorInvalidValue;
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(condensed_tc_kernel, smem, smem_cap); e != cudaSuccess) return e;
    const int grid = (a.P + kM - 1) / kM;
    return launch_kernel(condensed_tc_kernel, dim3(grid), dim3(kThreadsTC), smem, st, pdl, a,
                         status);
}

}  // namespace empc
