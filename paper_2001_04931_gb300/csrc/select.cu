// Elite selection: the E lowest-cost candidates in (cost, index) order.
//
// Algorithm 1's parent line keeps the numParents U arrays with the lowest
// costs (Sec. V, parent selection).  One CTA of 1024 threads per problem:
//   1. map each FP32 cost to an order-preserving 32-bit key (NaN as +inf);
//   2. radix-select the E-th smallest key, 8 bits per pass, with a shared
//      histogram and a warp scan of its 256 bins;
//   3. one block-wide exclusive scan of (less-than, equal) counts in index
//      order compacts the keys below the threshold plus the lowest-index
//      keys equal to it: exactly E distinct (key, index) pairs;
//   4. rank each selected pair by counting the pairs below it (E^2 shared
//      compares, E <= 2048) and scatter to rank order;
//   5. copy the best candidate's knots and cost out and bump the generation
//      counter that keys the next generation's draws.
// Fast path (steps 2-3 replaced): slots 0..E-1 always hold E candidates
// (after a warm start, the previous elites re-evaluated), so the E-th
// smallest (key, index) pair is at most K*, the largest pair among those
// slots.  When few candidates lie at or below K* they are compacted
// directly and ranked by counting; otherwise the radix select runs.
#include <cuda_runtime.h>

#include <cstdint>

#include "empc_internal.h"

namespace empc {
namespace {

constexpr int kSelThreads = 1024;
constexpr int kMaxElite = 2048;

__device__ __forceinline__ uint32_t order_key(float c) {
    if (c != c) c = __int_as_float(0x7f800000);
    const uint32_t u = __float_as_uint(c);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Exclusive block scan of one uint32 per thread (blockDim == 1024).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

// Copy the best candidate's knots and cost out; bump the generation counter.
__device__ __forceinline__ void finish_select(const float* __restrict__ cost, int P,
                                              const float* __restrict__ pop, int D,
                                              float* __restrict__ best_knots,
                                              float* __restrict__ best_cost,
                                              uint32_t* __restrict__ gen,
                                              int* __restrict__ status, int best) {
    for (int q = threadIdx.x; q < D; q += blockDim.x) best_knots[q] = pop[(size_t)q * P + best];
    if (threadIdx.x == 0) {
        const float bc = cost[best];
        *best_cost = bc;
        if (gen) *gen += 1u;
        if (status && !(bc < __int_as_float(0x7f800000))) atomicOr(status, 1);
    }
}

template <int KPT>
__global__ void __launch_bounds__(kSelThreads) select_kernel(
    const float* __restrict__ cost, int P, int E, const float* __restrict__ pop, int D,
    int* __restrict__ elite_idx, float* __restrict__ elite_cost, float* __restrict__ best_knots,
    float* __restrict__ best_cost, uint32_t* __restrict__ gen, int* __restrict__ status) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t s_digit, s_rem;
    __shared__ int s_best;
    __shared__ uint32_t s_count;
    __shared__ unsigned long long s_kstar;
    __shared__ unsigned long long s_red64[32];
    __shared__ unsigned long long sel[kMaxElite];

    const int tid = threadIdx.x;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t key[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int idx = tid * KPT + j;
        key[j] = idx < P ? order_key(cost[idx]) : 0xFFFFFFFFu;
    }

    // ---- fast path: bound from slots 0..E-1
    const int lane = tid & 31, warp = tid >> 5;
    {
        unsigned long long kmax = 0ull;
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int idx = tid * KPT + j;
            if (idx < E) kmax = max(kmax, ((unsigned long long)key[j] << 32) | (uint32_t)idx);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        if (lane == 0) s_red64[warp] = kmax;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = s_red64[lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) {
                s_kstar = v;
                s_count = 0;
            }
        }
        __syncthreads();
    }
    const unsigned long long kstar = s_kstar;
    uint32_t nbelow = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int idx = tid * KPT + j;
        nbelow += (idx < P && (((unsigned long long)key[j] << 32) | (uint32_t)idx) <= kstar);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nbelow += __shfl_xor_sync(0xffffffffu, nbelow, o);
    if (lane == 0) warp_tot[warp] = nbelow;
    __syncthreads();
    uint32_t L = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) L += warp_tot[w];
    const uint32_t cap = (uint32_t)min(kMaxElite, max(4 * E, 512));
    if (L <= cap) {
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int idx = tid * KPT + j;
            const unsigned long long k64 = ((unsigned long long)key[j] << 32) | (uint32_t)idx;
            const bool take = idx < P && k64 <= kstar;
            const uint32_t ball = __ballot_sync(0xffffffffu, take);
            uint32_t base = 0;
            if (lane == 0 && ball) base = atomicAdd(&s_count, (uint32_t)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (take) sel[base + __popc(ball & ((1u << lane) - 1u))] = k64;
        }
        __syncthreads();
        for (int e = tid; e < (int)L; e += blockDim.x) {
            const unsigned long long mine = sel[e];
            int rank = 0;
            for (int f = 0; f < (int)L; ++f) rank += sel[f] < mine;
            if (rank < E) {
                const int idx = (int)(mine & 0xFFFFFFFFull);
                elite_idx[rank] = idx;
                elite_cost[rank] = cost[idx];
                if (rank == 0) s_best = idx;
            }
        }
        __syncthreads();
        finish_select(cost, P, pop, D, best_knots, best_cost, gen, status, s_best);
        return;
    }

    // ---- radix select of the E-th smallest key
    uint32_t prefix = 0, mask = 0, rem = (uint32_t)E;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        // Costs of one population share their leading key bytes, so most
        // keys hit the same bin: aggregate equal bins within the warp and let
        // one lane per distinct bin add the count.
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const bool live = tid * KPT + j < P && (key[j] & mask) == prefix;
            const uint32_t bin = live ? (key[j] >> shift) & 0xFFu : 256u + (threadIdx.x & 31);
            const uint32_t peers = __match_any_sync(0xffffffffu, bin);
            if (live && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1))
                atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (tid < 32) {
            uint32_t loc[8], s = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                loc[b] = hist[tid * 8 + b];
                s += loc[b];
            }
            uint32_t incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += t;
            }
            const uint32_t excl = incl - s;
            if (excl < rem && rem <= incl) {
                uint32_t cum = excl;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (cum + loc[b] >= rem) {
                        s_digit = (uint32_t)(tid * 8 + b);
                        s_rem = rem - cum;
                        break;
                    }
                    cum += loc[b];
                }
            }
        }
        __syncthreads();
        prefix |= s_digit << shift;
        mask |= 0xFFu << shift;
        rem = s_rem;
        __syncthreads();
    }
    const uint32_t thr = prefix;
    const uint32_t need_eq = rem;

    // ---- compact: keys below thr, then the first need_eq keys equal to thr
    uint32_t nless = 0, neq = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        if (tid * KPT + j < P) {
            nless += key[j] < thr;
            neq += key[j] == thr;
        }
    }
    const uint32_t packed = block_exclusive_scan((nless << 16) | neq, warp_tot);
    uint32_t less_before = packed >> 16, eq_before = packed & 0xFFFFu;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const int idx = tid * KPT + j;
        if (idx >= P) continue;
        const unsigned long long k64 = ((unsigned long long)key[j] << 32) | (uint32_t)idx;
        if (key[j] < thr) {
            sel[less_before + min(eq_before, need_eq)] = k64;
            ++less_before;
        } else if (key[j] == thr) {
            if (eq_before < need_eq) sel[less_before + eq_before] = k64;
            ++eq_before;
        }
    }
    __syncthreads();

    // ---- rank by counting and scatter
    for (int e = tid; e < E; e += blockDim.x) {
        const unsigned long long mine = sel[e];
        int rank = 0;
        for (int f = 0; f < E; ++f) rank += sel[f] < mine;
        const int idx = (int)(mine & 0xFFFFFFFFull);
        elite_idx[rank] = idx;
        elite_cost[rank] = cost[idx];
        if (rank == 0) s_best = idx;
    }
    __syncthreads();
    finish_select(cost, P, pop, D, best_knots, best_cost, gen, status, s_best);
}

}  // namespace

cudaError_t launch_select(const float* cost, int P, int E, const float* pop, int D,
                          int* elite_idx, float* elite_cost, float* best_knots,
                          float* best_cost, uint32_t* gen, int* status, cudaStream_t st,
                          bool pdl) {
    if (P <= 0 || E <= 0 || E > P || E > kMaxElite) return cudaErrorInvalidValue;
    const int kpt = (P + kSelThreads - 1) / kSelThreads;
#define EMPC_SEL(K)                                                                      \
    return launch_kernel(select_kernel<K>, dim3(1), dim3(kSelThreads), 0, st, pdl, cost, P, E, \
                         pop, D, elite_idx, elite_cost, best_knots, best_cost, gen, status)
    if (kpt <= 1) EMPC_SEL(1);
    if (kpt <= 2) EMPC_SEL(2);
    if (kpt <= 4) EMPC_SEL(4);
    if (kpt <= 8) EMPC_SEL(8);
    if (kpt <= 16) EMPC_SEL(16);
    if (kpt <= 32) EMPC_SEL(32);
#undef EMPC_SEL
    return cudaErrorInvalidValue;
}

}  // namespace empc
