// Elite selection: the E lowest-cost candidates in (cost, index) order.
//
// Algorithm 1 keeps the numParents cheapest candidates as the parents of the
// next generation (Sec. V, parent selection).  One CTA of 512 threads per problem.
// Each cost maps to an order-preserving 32-bit key (NaN as +inf), paired
// with its index into a unique 64-bit (key, index) word.  The kernel picks a
// threshold key tau with at least E and at most 2048 words whose keys are at
// most tau, compacts those words into shared memory and ranks them: by
// counting when there are at most 256 (two or four lanes per word), else by
// sorting 64-word chunks (one warp each, register shuffles) and
// binary-searching the other chunks.
// Thresholds tried, in order:
//   1. the words of sixteen of the slots 0..E-1 (after a warm start those
//      slots hold the previous elites in rank order, so one of them usually
//      bounds a little more than E words), and K*, the largest word of those
//      slots (which always bounds at least E);
//   2. when those bound more than 2048 words, or more than 4 E + 256, a
//      quantile of a sorted stride sample of the words, a little above the
//      expected E/P quantile;
//   3. an exact radix select (8 bits per pass, warp-aggregated shared
//      histogram) of the E-th smallest word.
// The best candidate's knots are copied out while the words are ranked; the
// elite and best costs are decoded from the keys; the generation counter that
// keys the next generation's draws is advanced.
#include <cuda_runtime.h>

#include <cstdint>

#include "empc_internal.h"

namespace empc {
namespace {

constexpr int kSelThreads = 512;
constexpr int kMaxElite = 2048;

__device__ __forceinline__ uint32_t order_key(float c) {
    if (c != c) c = __int_as_float(0x7f800000);
    const uint32_t u = __float_as_uint(c);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Exclusive block scan of one uint32 per thread (blockDim a multiple of 32, <= 1024).
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
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
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

// The cost a key was made from: exact for every finite or infinite cost.  A
// NaN cost was keyed as +inf, so a caller that decodes +inf re-reads the cost.
__device__ __forceinline__ float key_cost(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// One compare-exchange of a bitonic network, seen from the element at
// position p holding `mine` whose partner p ^ j holds `other`.
__device__ __forceinline__ unsigned long long bitonic_keep(unsigned long long mine,
                                                           unsigned long long other, int p,
                                                           int j, int k) {
    const bool lower = (p & j) == 0, up = (p & k) == 0;
    return (lower == up) ? min(mine, other) : max(mine, other);
}

// Sort the 64 words s[0..64) within one warp (two per lane, bitonic network
// over register shuffles), in place.
__device__ __forceinline__ void warp_sort64(unsigned long long* s) {
    const int lane = (int)(threadIdx.x & 31u);
    const int p0 = 2 * lane;
    unsigned long long v0 = s[p0], v1 = s[p0 + 1];
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 1) {
                const unsigned long long lo = min(v0, v1), hi = max(v0, v1);
                const bool up = (p0 & k) == 0;
                v0 = up ? lo : hi;
                v1 = up ? hi : lo;
            } else {
                const unsigned long long o0 = __shfl_xor_sync(0xffffffffu, v0, j >> 1);
                const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, v1, j >> 1);
                v0 = bitonic_keep(v0, o0, p0, j, k);
                v1 = bitonic_keep(v1, o1, p0 + 1, j, k);
            }
        }
    }
    __syncwarp();
    s[p0] = v0;
    s[p0 + 1] = v1;
    __syncwarp();
}

// Rank the L distinct words s[0..L) (L <= kMaxElite): sort them in chunks
// of 64 (one warp per chunk), then rank each word as its place in its own
// chunk plus, for every other chunk, the number of smaller words there
// (binary search).  visit(rank, word) is called once per word, by the thread
// that ranked it.  Pads s up to a multiple of 64; every thread of the block
// must call it; the caller synchronizes after it.
template <class Visit>
__device__ __forceinline__ void rank_words(unsigned long long* s, int L, Visit&& visit) {
    const int Lp = (L + 63) & ~63;
    for (int i = L + (int)threadIdx.x; i < Lp; i += blockDim.x) s[i] = ~0ull;
    __syncthreads();
    const int C = Lp >> 6;
    for (int c = (int)(threadIdx.x >> 5); c < C; c += (int)(blockDim.x >> 5)) warp_sort64(s + 64 * c);
    __syncthreads();
    for (int e = (int)threadIdx.x; e < L; e += blockDim.x) {
        const unsigned long long x = s[e];
        const int ce = e >> 6;
        int rank = e & 63;
        for (int c = 0; c < C; ++c) {
            if (c == ce) continue;
            const unsigned long long* ch = s + 64 * c;
            int pos = 0;
#pragma unroll
            for (int step = 32; step > 0; step >>= 1)
                if (ch[pos + step - 1] < x) pos += step;
            if (pos == 63 && ch[63] < x) pos = 64;
            rank += pos;
        }
        visit(rank, x);
    }
}

// Number of words whose key is at most ktau, block-wide (every thread gets it).
template <int KPT>
__device__ __forceinline__ uint32_t count_at_most(const unsigned long long (&w)[KPT],
                                                  uint32_t ktau, uint32_t* warp_tot) {
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) c += (uint32_t)(w[j] >> 32) <= ktau;
    c = __reduce_add_sync(0xffffffffu, c);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = c;
    __syncthreads();
    uint32_t L = 0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) L += warp_tot[w2];
    return L;
}

template <int KPT>
__global__ void __launch_bounds__(kSelThreads, 1) select_kernel(
    const float* cost, int P, int E, const float* pop, int D,
    int* elite_idx, float* elite_cost, float* best_knots,
    float* best_cost, uint32_t* gen, int* status) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t s_digit, s_rem;
    __shared__ uint32_t s_count;
    __shared__ unsigned long long sel[kMaxElite];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the costs come from the kernel this one may overlap: every read of them
    // below is a coherent (L2) load issued after the wait
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const uint32_t gen0 = (tid == 0 && gen) ? *gen : 0u;  // advanced at the end
    constexpr unsigned long long kNone = ~0ull;
    unsigned long long w[KPT];  // (key, index); kNone past P
    if constexpr (KPT >= 16) {
        // a thread's KPT consecutive costs as 16-byte loads (the buffer starts
        // 16-byte aligned and KPT is a multiple of 4): a quarter of the scalar
        // loads' requests (measured at 16384 candidates; smaller populations
        // keep the scalar loads)
#pragma unroll
        for (int j = 0; j < KPT; j += 4) {
            const int idx = tid * KPT + j;
            float v[4];
            if (idx + 3 < P) {
                const float4 t = __ldcg(reinterpret_cast<const float4*>(cost + idx));
                v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = idx + u < P ? __ldcg(cost + idx + u) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                w[j + u] = idx + u < P ? (((unsigned long long)order_key(v[u]) << 32) |
                                          (uint32_t)(idx + u))
                                       : kNone;
        }
    } else {
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const int idx = tid * KPT + j;
            w[j] = idx < P ? (((unsigned long long)order_key(__ldcg(cost + idx)) << 32) |
                              (uint32_t)idx)
                           : kNone;
        }
    }

    // ---- 1. thresholds from the slots 0..E-1: sixteen slot words and K*
    // Thread i < 16 reads threshold i's slot itself, so the slot keys, the
    // per-warp maxima of slots 0..E-1 and the zeroed totals need one barrier
    // before the counting, and the warp counts one more before the choice.
    constexpr int kThr = 16;
    __shared__ uint32_t s_thr[kThr];
    __shared__ uint32_t s_kmax[32];
    __shared__ uint32_t s_tot[kThr + 1];
    uint32_t tau;  // threshold key: the words with keys at most tau are ranked
    uint32_t L;
    {
        if (tid < kThr) {
            // slot (i+1) E / kThr - 1 supplies threshold i; a threshold no slot
            // supplies bounds nothing
            const int slot = (tid + 1) * E / kThr - 1;
            s_thr[tid] = slot >= 0 ? order_key(__ldcg(cost + slot)) : 0u;
        }
        if (tid <= kThr) s_tot[tid] = 0u;
        if (tid == 0) s_count = 0u;  // the compaction's reservations
        uint32_t kmax = 0u;
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if (tid * KPT + j < E) kmax = max(kmax, (uint32_t)(w[j] >> 32));
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0) s_kmax[warp] = kmax;
        __syncthreads();
        uint32_t thr[kThr + 1];
#pragma unroll
        for (int i = 0; i < kThr; ++i) thr[i] = s_thr[i];
        thr[kThr] = 0u;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) thr[kThr] = max(thr[kThr], s_kmax[w2]);
        uint32_t c[kThr + 1];
#pragma unroll
        for (int i = 0; i <= kThr; ++i) c[i] = 0;
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const uint32_t kj = (uint32_t)(w[j] >> 32);
#pragma unroll
            for (int i = 0; i <= kThr; ++i) c[i] += kj <= thr[i];
        }
#pragma unroll
        for (int i = 0; i <= kThr; ++i) {
            c[i] = __reduce_add_sync(0xffffffffu, c[i]);
            if (lane == 0) atomicAdd(&s_tot[i], c[i]);
        }
        __syncthreads();
        // the threshold bounding the fewest words, but at least E (K* always does)
        tau = thr[kThr];
        L = s_tot[kThr];
#pragma unroll
        for (int i = 0; i < kThr; ++i) {
            const uint32_t ci = s_tot[i];
            if (ci >= (uint32_t)E && ci < L) {
                L = ci;
                tau = thr[i];
            }
        }
    }

    // ---- 2. a sample quantile when none of them admits at most 2048, or
    // admits many more words than E (ranking a 512-word sample costs less)
    if (L > (uint32_t)kMaxElite || L > 4u * (uint32_t)E + 256u) {
        const int S = min((int)blockDim.x, (P + KPT - 1) / KPT);  // threads holding a word
        __shared__ uint32_t s_ts;
        sel[tid] = tid < S ? w[0] : kNone;                        // stride-KPT sample
        const int r = min(S - 1, (int)((1.25 * E * S) / P) + 8);
        rank_words(sel, (int)blockDim.x, [&](int rank, unsigned long long x) {
            if (rank == r) s_ts = (uint32_t)(x >> 32);
        });
        __syncthreads();
        const uint32_t ts = s_ts;
        const uint32_t Ls = count_at_most<KPT>(w, ts, warp_tot);
        if (Ls >= (uint32_t)E && Ls < L && Ls <= (uint32_t)kMaxElite) {
            tau = ts;
            L = Ls;
        }
    }

    if (L <= (uint32_t)kMaxElite) {
        // ---- compact the words at or below tau, sort, keep the first E: one
        // reservation per warp for up to 16 of its words each (s_count was
        // zeroed before the threshold phase's first barrier)
        constexpr int kG = KPT < 16 ? KPT : 16;
        const uint32_t below = (1u << lane) - 1u;
#pragma unroll
        for (int j0 = 0; j0 < KPT; j0 += kG) {
            uint32_t ball[kG], tot = 0;
#pragma unroll
            for (int j = 0; j < kG; ++j) {
                ball[j] = __ballot_sync(0xffffffffu, (uint32_t)(w[j0 + j] >> 32) <= tau);
                tot += (uint32_t)__popc(ball[j]);
            }
            uint32_t base = 0;
            if (lane == 0 && tot) base = atomicAdd(&s_count, tot);
            base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
            for (int j = 0; j < kG; ++j) {
                if ((ball[j] >> lane) & 1u) sel[base + __popc(ball[j] & below)] = w[j0 + j];
                base += (uint32_t)__popc(ball[j]);
            }
        }
    } else {
        // ---- 3. exact radix select of the E-th smallest key
        uint32_t prefix = 0, mask = 0, rem = (uint32_t)E;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
            __syncthreads();
            // Costs of one population share their leading key bytes, so most
            // keys hit the same bin: aggregate equal bins within the warp and
            // let one lane per distinct bin add the count.
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                const uint32_t kj = (uint32_t)(w[j] >> 32);
                const bool live = w[j] != kNone && (kj & mask) == prefix;
                const uint32_t bin = live ? (kj >> shift) & 0xFFu : 256u + lane;
                const uint32_t peers = __match_any_sync(0xffffffffu, bin);
                if (live && lane == (uint32_t)(__ffs(peers) - 1))
                    atomicAdd(&hist[bin], (uint32_t)__popc(peers));
            }
            __syncthreads();
            if (tid < 32) {
                uint32_t loc[8], sum = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    loc[b] = hist[tid * 8 + b];
                    sum += loc[b];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (tid >= o) incl += t;
                }
                const uint32_t excl = incl - sum;
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
        // keys below thr, then the first need_eq keys equal to thr in index order
        uint32_t nless = 0, neq = 0;
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (w[j] != kNone) {
                const uint32_t kj = (uint32_t)(w[j] >> 32);
                nless += kj < thr;
                neq += kj == thr;
            }
        }
        const uint32_t packed = block_exclusive_scan((nless << 16) | neq, warp_tot);
        uint32_t less_before = packed >> 16, eq_before = packed & 0xFFFFu;
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (w[j] == kNone) continue;
            const uint32_t kj = (uint32_t)(w[j] >> 32);
            if (kj < thr) {
                sel[less_before + min(eq_before, need_eq)] = w[j];
                ++less_before;
            } else if (kj == thr) {
                if (eq_before < need_eq) sel[less_before + eq_before] = w[j];
                ++eq_before;
            }
        }
        L = (uint32_t)E;
    }
    __syncthreads();
    // The best word (rank 0): every warp finds it, so the best plan's loads
    // are in flight while the words are ranked.
    unsigned long long bw = kNone;
    for (int f = lane; f < (int)L; f += 32) bw = min(bw, sel[f]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bw = min(bw, __shfl_xor_sync(0xffffffffu, bw, o));
    const int best = (int)(bw & 0xFFFFFFFFull);
    // issued now, stored after the ranking: a store would wait for its load
    const float bk0 = tid < D ? __ldcg(pop + (size_t)tid * P + best) : 0.0f;
    const float kInf = __int_as_float(0x7f800000);
    auto keep = [&](int rank, unsigned long long x) {
        if (rank < E) {
            const int idx = (int)(x & 0xFFFFFFFFull);
            float c = key_cost((uint32_t)(x >> 32));
            if (c == kInf) c = __ldcg(cost + idx);  // +inf or NaN
            elite_idx[rank] = idx;
            elite_cost[rank] = c;
        }
    };
    if (L <= 256u) {
        // few words: S adjacent lanes rank each word by counting the words
        // below it, each over a 1/S share of them (every lane of a group reads
        // the same word in each iteration: a broadcast), then add up their counts
        const int S = L <= 128u ? 4 : 2;
        const int e = tid / S, part = tid % S;
        if (warp * 32 / S < (int)L) {  // warp-uniform: the warp holds a word
            const int f0 = part * (int)L / S, f1 = (part + 1) * (int)L / S;
            const unsigned long long mine = e < (int)L ? sel[e] : kNone;
            int rank = 0;
            for (int f = f0; f < f1; ++f) rank += sel[f] < mine;
            for (int o = 1; o < S; o <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
            if (part == 0 && e < (int)L) keep(rank, mine);
        }
    } else {
        rank_words(sel, (int)L, keep);
    }
    if (tid < D) best_knots[tid] = bk0;
    for (int q = tid + (int)blockDim.x; q < D; q += blockDim.x)
        best_knots[q] = __ldcg(pop + (size_t)q * P + best);
    if (tid == 0) {
        float bc = key_cost((uint32_t)(bw >> 32));
        if (bc == kInf) bc = __ldcg(cost + best);
        *best_cost = bc;
        if (gen) *gen = gen0 + 1u;
        if (status && !(bc < kInf)) atomicOr(status, 1);
    }
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
    if (kpt <= 64) EMPC_SEL(64);
#undef EMPC_SEL
    return cudaErrorInvalidValue;
}

}  // namespace empc
