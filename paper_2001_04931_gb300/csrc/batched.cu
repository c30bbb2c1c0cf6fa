// Batched EMPC: many independent problems of uneven size in one persistent
// launch (no counterpart in the paper, whose GPU runs one problem at a time).
//
// Work is a generation-major queue of items; within a generation, first the
// breeding items (problem, candidate chunk), then the rollout items (problem,
// candidate tile), longest problems first.  Every CTA loops: take the next
// ticket.  A breeding item waits until its problem has finished selecting the
// previous generation, then breeds its chunk of candidates with the whole
// CTA (one thread per candidate and 4-knot group, as the single-problem
// breeding kernel does) and counts itself done.  A rollout item waits until
// every breeding item of its problem's generation is done, then rolls out the
// bred tile (the warp-synchronous tile of rollout_warp.cuh, reading
// populations through L2) and counts the tile done.  The CTA that completes a
// problem's last tile of a generation selects that problem's elites and then
// publishes the problem as ready for the next generation.  There is no
// grid-wide barrier: problems advance independently.  Every wait is for an
// item with an earlier ticket, taken by a CTA that is already running and
// that itself waits only on earlier tickets, so no co-residency of the grid
// is needed for progress (the grid is sized to fill the GPU once).
// Waits are bounded by the %globaltimer clock: past the limit the kernel sets
// an error flag that the host reports as EMPC_ETIMEOUT, and every CTA leaves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "host_tables.h"
#include "rollout_warp.cuh"

namespace empc {
namespace {

struct BatchProblem {
    RolloutArgs a;  // model, sizes, breeding parameters, cost and elite buffers
    float* pop[2];
    float* elite_cost;
    float* best_knots;
    float* best_cost;
    int* status;
    int nx;          // compiled state dimension
    int tiles;       // tiles per generation
    int tile_cands;  // candidates per tile
    int breeds;      // breeding items per generation
    int breed_cands; // candidates per breeding item
};

// Candidates per breeding item.
constexpr int kBreedChunk = 256;

struct BatchArgs {
    const BatchProblem* probs;
    const int2* items;  // (problem, tile) per generation, in work order
    int n_items;
    int generations;
    int cold_first;
    int parity;  // every population reads pop[parity] at launch
    unsigned* ticket;
    unsigned* done;   // tiles completed, per problem (cumulative over generations)
    unsigned* ready;  // generations selected, per problem
    unsigned* bred;   // breeding items completed, per problem (cumulative)
    int* error;
    int stall_problem;  // fault injection: this problem never publishes (-1: none)
    unsigned long long timeout_ns;
    int bt_floats, ks_floats, slice_floats, key_words, sel_cap;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void store_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t order_key(float c) {
    if (c != c) c = __int_as_float(0x7f800000);
    const uint32_t u = __float_as_uint(c);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

struct SelectScratch {
    uint32_t hist[256];
    unsigned long long red[32];
    uint32_t digit, rem, count;
    unsigned long long kstar;
    int best;
};

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, SelectScratch& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s.red[warp] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int w = 0; w < nw; ++w) r = max(r, s.red[w]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, SelectScratch& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s.red[warp] = v;
    __syncthreads();
    unsigned long long r = 0;
    for (int w = 0; w < nw; ++w) r += s.red[w];
    __syncthreads();
    return r;
}

// Exclusive scan over the block of one value per thread.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, SelectScratch& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s.red[warp] = incl;
    __syncthreads();
    unsigned long long base = 0;
    for (int w = 0; w < warp; ++w) base += s.red[w];
    (void)nw;
    __syncthreads();
    return base + incl - v;
}

// Block-level elite selection of one problem (the E lowest (cost, index)
// pairs, NaN as +inf), as select.cu does it for one CTA of 1024 threads:
// the bound from slots 0..E-1 when few candidates lie below it, else a radix
// select of the E-th key; then ranking by counting.  Costs and the
// population are read through L2 (written by other CTAs of this launch).
__device__ void block_select(const BatchProblem& P, const float* pop, uint32_t* skey,
                             unsigned long long* sel, int cap, SelectScratch& s) {
    const RolloutArgs& a = P.a;
    const int Pn = a.P, E = a.E, D = a.m * a.p;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < Pn; i += nthr) skey[i] = order_key(__ldcg(a.cost + i));
    __syncthreads();
    auto k64 = [&](int i) { return ((unsigned long long)skey[i] << 32) | (uint32_t)i; };
    unsigned long long kmax = 0;
    for (int i = tid; i < E; i += nthr) kmax = max(kmax, k64(i));
    const unsigned long long kstar = block_max_u64(kmax, s);
    unsigned long long below = 0;
    for (int i = tid; i < Pn; i += nthr) below += k64(i) <= kstar;
    const unsigned long long L = block_sum_u64(below, s);
    int nsel;
    if (L <= (unsigned long long)cap) {
        if (tid == 0) s.count = 0;
        __syncthreads();
        const int lane = tid & 31;
        for (int base = 0; base < Pn; base += nthr) {
            const int i = base + tid;
            const bool take = i < Pn && k64(i) <= kstar;
            const uint32_t ball = __ballot_sync(0xffffffffu, take);
            uint32_t pos = 0;
            if (lane == 0 && ball) pos = atomicAdd(&s.count, (uint32_t)__popc(ball));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (take) sel[pos + __popc(ball & ((1u << lane) - 1u))] = k64(i);
        }
        nsel = (int)L;
    } else {
        uint32_t prefix = 0, mask = 0, rem = (uint32_t)E;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 256; i += nthr) s.hist[i] = 0;
            __syncthreads();
            for (int base = 0; base < Pn; base += nthr) {
                const int i = base + tid;
                const bool live = i < Pn && (skey[i] & mask) == prefix;
                const uint32_t bin = live ? (skey[i] >> shift) & 0xFFu : 256u + (tid & 31);
                const uint32_t peers = __match_any_sync(0xffffffffu, bin);
                if (live && (tid & 31) == (uint32_t)(__ffs(peers) - 1))
                    atomicAdd(&s.hist[bin], (uint32_t)__popc(peers));
            }
            __syncthreads();
            if (tid < 32) {
                uint32_t loc[8], sum = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    loc[q] = s.hist[tid * 8 + q];
                    sum += loc[q];
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
                    for (int q = 0; q < 8; ++q) {
                        if (cum + loc[q] >= rem) {
                            s.digit = (uint32_t)(tid * 8 + q);
                            s.rem = rem - cum;
                            break;
                        }
                        cum += loc[q];
                    }
                }
            }
            __syncthreads();
            prefix |= s.digit << shift;
            mask |= 0xFFu << shift;
            rem = s.rem;
            __syncthreads();
        }
        // compaction in index order: each thread owns a contiguous chunk
        const int ch = (Pn + nthr - 1) / nthr;
        const int lo = min(Pn, tid * ch), hi = min(Pn, lo + ch);
        unsigned long long nless = 0, neq = 0;
        for (int i = lo; i < hi; ++i) {
            nless += skey[i] < prefix;
            neq += skey[i] == prefix;
        }
        const unsigned long long pk = block_excl_scan((nless << 32) | neq, s);
        unsigned long long lb = pk >> 32, eb = pk & 0xFFFFFFFFull;
        for (int i = lo; i < hi; ++i) {
            if (skey[i] < prefix) {
                sel[lb + min(eb, (unsigned long long)rem)] = k64(i);
                ++lb;
            } else if (skey[i] == prefix) {
                if (eb < rem) sel[lb + eb] = k64(i);
                ++eb;
            }
        }
        nsel = E;
    }
    __syncthreads();
    for (int e = tid; e < nsel; e += nthr) {
        const unsigned long long mine = sel[e];
        int rank = 0;
        for (int f = 0; f < nsel; ++f) rank += sel[f] < mine;
        if (rank < E) {
            const int idx = (int)(mine & 0xFFFFFFFFull);
            const_cast<int*>(a.elite_idx)[rank] = idx;
            P.elite_cost[rank] = __ldcg(a.cost + idx);
            if (rank == 0) s.best = idx;
        }
    }
    __syncthreads();
    const int best = s.best;
    for (int q = tid; q < D; q += nthr) P.best_knots[q] = __ldcg(pop + (size_t)q * Pn + best);
    if (tid == 0) {
        const float bc = __ldcg(a.cost + best);
        *P.best_cost = bc;
        atomicAdd(const_cast<uint32_t*>(a.gen), 1u);
        if (!(bc < __int_as_float(0x7f800000))) atomicOr(P.status, 1);
    }
}

__device__ __forceinline__ int xr_of(int nx) {
    switch (nx) {
        case 4: return 4;
        case 8: return 8;
        case 16: return 16;
        case 24: return 24;
        case 32: return 32;
        case 40: return 48;
        case 48: return 48;
        case 56: return 64;
        default: return 64;
    }
}

template <int WPC, int C>
__global__ void __launch_bounds__(WPC * 32) batched_kernel(const BatchArgs b) {
    extern __shared__ __align__(16) float smem[];
    __shared__ SelectScratch ss;
    __shared__ unsigned s_ticket;
    __shared__ int s_flag;
    float* BTs = smem;
    KnotStep* ks = reinterpret_cast<KnotStep*>(smem + b.bt_floats);
    float* slices = smem + b.bt_floats + b.ks_floats;
    uint32_t* skey = reinterpret_cast<uint32_t*>(slices + WPC * b.slice_floats);
    unsigned long long* sel = reinterpret_cast<unsigned long long*>(skey + b.key_words);
    const int warp = threadIdx.x >> 5;
    const unsigned total = (unsigned)b.n_items * (unsigned)b.generations;
    int staged = -1;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(b.ticket, 1u);
        __syncthreads();
        const unsigned ticket = s_ticket;
        if (ticket >= total) break;
        const int g = (int)(ticket / (unsigned)b.n_items);
        const int2 it = b.items[ticket % (unsigned)b.n_items];
        const BatchProblem& P = b.probs[it.x];
        const bool breeding = it.y < 0;
        if (threadIdx.x == 0) {
            int ok = 1;
            // breeding waits for the previous generation's selection, a
            // rollout tile for all of this generation's breeding
            const unsigned* ctr = breeding ? b.ready + it.x : b.bred + it.x;
            const unsigned need =
                breeding ? (unsigned)g : (unsigned)(g + 1) * (unsigned)P.breeds;
            if (need > 0) {
                const unsigned long long t0 = global_ns();
                while (load_acquire(ctr) < need) {
                    if (*(volatile int*)b.error) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > b.timeout_ns) {
                        atomicOr(b.error, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            s_flag = ok;
        }
        __syncthreads();
        if (!s_flag) break;
        RolloutArgs a = P.a;
        a.mode = (g == 0 && b.cold_first) ? kCold : kWarm;
        a.pop_in = P.pop[b.parity ^ (g & 1)];
        a.pop_out = P.pop[b.parity ^ ((g + 1) & 1)];
        a.cand_begin = 0;
        a.pdl = 0;
        if (breeding) {
            // candidates [cb, ce) of generation g into pop_out: one thread per
            // (candidate, 4-knot group), consecutive threads on consecutive
            // candidates (coalesced stores)
            const uint32_t gen = *(volatile const uint32_t*)a.gen;
            const int D = a.m * a.p, nq = (D + 3) >> 2;
            const int cb = (-1 - it.y) * P.breed_cands;
            const int nc = min(a.P, cb + P.breed_cands) - cb;
            for (int w = threadIdx.x; w < nc * nq; w += blockDim.x) {
                const int c = cb + w % nc, quad = w / nc;
                int s1 = 0, s2 = -1;
                if (a.mode == kWarm) parents_of<true>(a, c, gen, s1, s2);
                float v[4];
                breed_quad<true>(a, c, quad, gen, s1, s2, v);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (quad * 4 + e < D) a.pop_out[(size_t)(quad * 4 + e) * a.P + c] = v[e];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(b.bred + it.x, 1u);
            }
            continue;
        }
        // the rollout evaluates the bred population
        a.mode = kEval;
        a.pop_in = a.pop_out;
        if (staged != it.x) {
            const int xr = xr_of(P.nx);
            for (int i = threadIdx.x; i < a.m * xr; i += blockDim.x) {
                const int row = i % xr, col = i / xr;
                BTs[i] = row < a.n ? a.BT[col * a.n + row] : 0.0f;
            }
            for (int k = threadIdx.x; k < a.T; k += blockDim.x) ks[k] = a.ktab[k];
            __syncthreads();
            staged = it.x;
        }
        const int c0 = it.y * P.tile_cands + warp * (P.tile_cands / WPC);
        float* W = slices + warp * b.slice_floats;
        if (c0 < a.P) {
            switch (P.nx) {
                case 4: warp_tile<4, C, true>(a, c0, W, BTs, ks); break;
                case 8: warp_tile<8, C, true>(a, c0, W, BTs, ks); break;
                case 16: warp_tile<16, C, true>(a, c0, W, BTs, ks); break;
                case 24: warp_tile<24, C, true>(a, c0, W, BTs, ks); break;
                case 32: warp_tile<32, C, true>(a, c0, W, BTs, ks); break;
                case 40: warp_tile<40, C, true>(a, c0, W, BTs, ks); break;
                case 48: warp_tile<48, C, true>(a, c0, W, BTs, ks); break;
                case 56: warp_tile<56, C, true>(a, c0, W, BTs, ks); break;
                default: warp_tile<64, C, true>(a, c0, W, BTs, ks); break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned old = atomicAdd(b.done + it.x, 1u);
            s_flag = old + 1u == (unsigned)(P.tiles * (g + 1));
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            block_select(P, a.pop_out, skey, sel, b.sel_cap, ss);
            __syncthreads();
            if (threadIdx.x == 0 && it.x != b.stall_problem) {
                __threadfence();
                store_release(b.ready + it.x, (unsigned)(g + 1));
            }
        }
    }
}

// Compiled launch shapes: (warps per CTA, candidates per lane).
struct BatchShape {
    int wpc, cands;
};
constexpr int kNumBatchShapes = 4;
constexpr BatchShape kBatchShapes[kNumBatchShapes] = {{4, 2}, {2, 2}, {4, 4}, {2, 4}};

using BatchKernel = void (*)(BatchArgs);
BatchKernel batch_kernel_of(int shape) {
    switch (shape) {
        case 0: return batched_kernel<4, 2>;
        case 1: return batched_kernel<2, 2>;
        case 2: return batched_kernel<4, 4>;
        default: return batched_kernel<2, 4>;
    }
}

int nrg_host(int nx) { return nx == 4 ? 2 : nx == 8 ? 4 : nx <= 24 ? 8 : nx <= 48 ? 16 : 32; }
int nx_class(int n) {
    static const int kNx[] = {4, 8, 16, 24, 32, 40, 48, 56, 64};
    for (int v : kNx)
        if (n <= v) return v;
    return 0;
}

struct GraphKeyB {
    int G, cold, parity;
    bool operator<(const GraphKeyB& o) const {
        return std::tie(G, cold, parity) < std::tie(o.G, o.cold, o.parity);
    }
};

}  // namespace
}  // namespace empc

using empc::BatchArgs;
using empc::BatchProblem;

struct empc_batch_s {
    int count = 0;
    std::vector<int> n, m, T, p, P, E, D, nx, knot_off;
    int total_knots = 0;
    double state_steps_per_gen = 0;
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;      // the batch's own stream
    cudaStream_t run_stream = nullptr;  // where solves run (own stream unless set)
    char* arena = nullptr;
    BatchProblem* d_probs = nullptr;
    std::vector<BatchProblem> h_probs;
    int2* d_items[empc::kNumBatchShapes] = {};
    int n_items[empc::kNumBatchShapes] = {};
    unsigned* d_counters = nullptr;  // ticket | done[count] | ready[count] | bred[count]
    int* d_error = nullptr;
    float* d_best_knots = nullptr;   // [total_knots]
    float* d_best_costs = nullptr;   // [count]
    int* d_status = nullptr;         // [count]
    float* h_stage = nullptr;        // pinned image of the result span (knots .. error)
    size_t result_floats = 0;        // floats from the best knots to the error word
    size_t off_costs_rel = 0, off_status_rel = 0, off_error_rel = 0;  // within that span
    std::vector<int> tgt_off;        // problem's offset in the x0 / goal blocks
    std::vector<empc::HostTables> rot;  // per problem: its x -> z rotation (Vt) if Q is dense
    size_t tgt_floats = 0;           // floats of one block (x0 block, then goal block)
    float* d_targets = nullptr;      // device: x0 block | goal block
    float* h_targets = nullptr;      // pinned staging of the same
    cudaEvent_t tgt_done = nullptr;  // the last targets copy has read h_targets
    int shape = 0, grid = 0;
    size_t smem = 0;
    int bt_floats = 0, ks_floats = 0, slice_floats[empc::kNumBatchShapes] = {}, key_words = 0,
        sel_cap = 0;
    int parity = 0;
    bool has_pop = false;
    int stall_problem = -1;
    unsigned long long timeout_ns = 1000000000ull;
    float tuned_us = 0.0f;
    std::map<empc::GraphKeyB, cudaGraphExec_t> graphs;
    std::string err;
};

namespace {

empc_status bfail(empc_batch b, empc_status s, const std::string& msg) {
    if (b) b->err = msg;
    empc::set_thread_error(s, msg.c_str());
    return s;
}

#define EMPC_BCUDA(b, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return bfail((b), EMPC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void free_batch(empc_batch b) {
    if (!b) return;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    if (b->arena) cudaFree(b->arena);
    if (b->h_stage) cudaFreeHost(b->h_stage);
    if (b->h_targets) cudaFreeHost(b->h_targets);
    if (b->tgt_done) cudaEventDestroy(b->tgt_done);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

BatchArgs batch_args(empc_batch b, int G, bool cold, int parity) {
    BatchArgs a{};
    a.probs = b->d_probs;
    a.items = b->d_items[b->shape];
    a.n_items = b->n_items[b->shape];
    a.generations = G;
    a.cold_first = cold ? 1 : 0;
    a.parity = parity;
    a.ticket = b->d_counters;
    a.done = b->d_counters + 1;
    a.ready = b->d_counters + 1 + b->count;
    a.bred = b->d_counters + 1 + 2 * (size_t)b->count;
    a.error = b->d_error;
    a.stall_problem = b->stall_problem;
    a.timeout_ns = b->timeout_ns;
    a.bt_floats = b->bt_floats;
    a.ks_floats = b->ks_floats;
    a.slice_floats = b->slice_floats[b->shape];
    a.key_words = b->key_words;
    a.sel_cap = b->sel_cap;
    return a;
}

size_t batch_smem(empc_batch b, int shape) {
    const int wpc = empc::kBatchShapes[shape].wpc;
    return sizeof(float) * ((size_t)b->bt_floats + b->ks_floats + (size_t)wpc * b->slice_floats[shape] +
                            b->key_words) +
           sizeof(unsigned long long) * (size_t)b->sel_cap;
}

// Enqueue one launch: reset the counters, run G generations.
cudaError_t enqueue_batch(empc_batch b, int G, bool cold, int parity, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(unsigned) * (1 + 3 * (size_t)b->count), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->d_error, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(b->d_status, 0, sizeof(int) * (size_t)b->count, st)) != cudaSuccess) return e;
    BatchArgs a = batch_args(b, G, cold, parity);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(32 * empc::kBatchShapes[b->shape].wpc);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, empc::batch_kernel_of(b->shape), a);
}

empc_status configure_shape(empc_batch b, int shape) {
    auto kern = empc::batch_kernel_of(shape);
    const size_t smem = batch_smem(b, shape);
    if (smem > 227u * 1024u) return bfail(b, EMPC_EUNSUPPORTED, "batch does not fit in shared memory");
    // raise the kernel's limit on this device, never lower it: another batch
    // on the device may launch the same kernel with more shared memory
    cudaFuncAttributes fa{};
    EMPC_BCUDA(b, cudaFuncGetAttributes(&fa, kern));
    if ((int)smem > fa.maxDynamicSharedSizeBytes)
        EMPC_BCUDA(b, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    EMPC_BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      &per_sm, kern, 32 * empc::kBatchShapes[shape].wpc, smem));
    if (per_sm < 1) return bfail(b, EMPC_EUNSUPPORTED, "batched kernel does not fit on an SM");
    b->shape = shape;
    b->smem = smem;
    b->grid = per_sm * b->sms;
    return EMPC_OK;
}

}  // namespace

extern "C" {

empc_status empc_batch_create(const empc_problem_desc* probs, int count, const empc_config* cfg_in,
                              empc_batch* out) {
    if (!out) return bfail(nullptr, EMPC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!probs || count < 1) return bfail(nullptr, EMPC_EINVAL, "need count >= 1 problems");
    empc_config cfg;
    if (cfg_in) cfg = *cfg_in; else empc_config_default(&cfg);
    if (cfg.refine_steps != 0 || cfg.precision != EMPC_FP32)
        return bfail(nullptr, EMPC_EUNSUPPORTED, "batched solves are FP32 without refinement");
    if (cfg.gate < 0 || cfg.gate > 2 || cfg.p_cross_256 < 0 || cfg.p_cross_256 > 256 ||
        cfg.p_mutate_256 < 0 || cfg.p_mutate_256 > 256)
        return bfail(nullptr, EMPC_EINVAL, "bad breeding parameters");
    empc_batch b = new empc_batch_s();
    b->count = count;
    std::vector<empc::HostTables> tabs(count);
    size_t floats = 0;
    auto reserve = [&](size_t k) {  // 16-byte aligned sub-arrays
        const size_t at = floats;
        floats += (k + 3) / 4 * 4;
        return at;
    };
    struct Off {
        size_t D, BT, qd, rd, rmat, gram, ks, lo, hi, pop0, pop1, cost, elite, ecost, gen, status;
    };
    std::vector<Off> off(count);
    for (int i = 0; i < count; ++i) {
        const empc_problem_desc& d = probs[i];
        std::string msg;
        empc_status vs = empc::validate_problem(d.A, d.B, d.Q, d.R, d.bounds, d.n, d.m, d.horizon,
                                                d.knots, d.pop, msg);
        if (vs != EMPC_OK) {
            free_batch(b);
            return bfail(nullptr, vs, "problem " + std::to_string(i) + ": " + msg);
        }
        if (d.n > 64) {
            free_batch(b);
            return bfail(nullptr, EMPC_EUNSUPPORTED, "batched problems need n <= 64");
        }
        if (!d.x0 || !d.x_goal || !empc::all_finite(d.x0, d.n) || !empc::all_finite(d.x_goal, d.n)) {
            free_batch(b);
            return bfail(nullptr, EMPC_EINVAL, "problem " + std::to_string(i) + ": bad x0 / x_goal");
        }
        const int E = d.elite > 0 ? d.elite : std::max(1, d.pop / 16);
        if (E > d.pop || E > 2048) {
            free_batch(b);
            return bfail(nullptr, EMPC_EINVAL, "problem " + std::to_string(i) + ": bad elite count");
        }
        vs = empc::build_tables(d.A, d.B, d.Q, d.R, d.bounds, d.n, d.m, d.horizon, d.knots,
                                tabs[i], msg);
        if (vs != EMPC_OK) {
            free_batch(b);
            return bfail(nullptr, vs, "problem " + std::to_string(i) + ": " + msg);
        }
        b->n.push_back(d.n);
        b->m.push_back(d.m);
        b->T.push_back(d.horizon);
        b->p.push_back(d.knots);
        b->P.push_back(d.pop);
        b->E.push_back(E);
        b->D.push_back(d.m * d.knots);
        b->nx.push_back(empc::nx_class(d.n));
        b->knot_off.push_back(b->total_knots);
        b->total_knots += d.m * d.knots;
        b->state_steps_per_gen += (double)d.pop * d.horizon;
        Off& o = off[i];
        const size_t DP = (size_t)d.m * d.knots * d.pop;
        o.D = reserve((size_t)d.n * d.n);
        o.BT = reserve((size_t)d.m * d.n);
        o.qd = reserve(d.n);
        o.rd = reserve(d.m);
        o.rmat = tabs[i].dense_r ? reserve((size_t)d.m * d.m) : 0;
        o.gram = reserve(2 * (size_t)d.knots);
        o.ks = reserve(4 * (size_t)d.horizon);
        o.lo = reserve(d.m);
        o.hi = reserve(d.m);
        // start and goal live in two contiguous blocks (one copy updates all)
        b->tgt_off.push_back((int)b->tgt_floats);
        b->tgt_floats += (size_t)(d.n + 3) / 4 * 4;
        o.pop0 = reserve(DP);
        o.pop1 = reserve(DP);
        o.cost = reserve(d.pop);
        o.elite = reserve(E);
        o.ecost = reserve(E);
        o.gen = reserve(1);
        o.status = reserve(1);
    }
    const size_t off_tgt = reserve(2 * b->tgt_floats);
    const size_t off_best = reserve(b->total_knots);
    const size_t off_bcost = reserve(count);
    const size_t off_bstat = reserve(count);
    const size_t off_counters = reserve(1 + 3 * (size_t)count);
    const size_t off_error = reserve(1);
    const size_t off_probs = reserve(sizeof(BatchProblem) / 4 * (size_t)count + 4);
    size_t off_items[empc::kNumBatchShapes];
    // work lists, per launch shape: tiles of each problem, longest first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (double)b->T[x] * b->nx[x] * b->nx[x] > (double)b->T[y] * b->nx[y] * b->nx[y];
    });
    std::vector<std::vector<int2>> items(empc::kNumBatchShapes);
    std::vector<std::vector<int>> tiles(empc::kNumBatchShapes, std::vector<int>(count)),
        tcands(empc::kNumBatchShapes, std::vector<int>(count));
    for (int s = 0; s < empc::kNumBatchShapes; ++s) {
        const empc::BatchShape sh = empc::kBatchShapes[s];
        // a generation: every problem's breeding items, then its rollout tiles
        for (int i : order) {
            const int nb = (b->P[i] + empc::kBreedChunk - 1) / empc::kBreedChunk;
            for (int c = 0; c < nb; ++c) items[s].push_back(make_int2(i, -1 - c));
        }
        for (int i : order) {
            const int cpt = sh.wpc * (32 / empc::nrg_host(b->nx[i])) * sh.cands;
            const int nt = (b->P[i] + cpt - 1) / cpt;
            tiles[s][i] = nt;
            tcands[s][i] = cpt;
            for (int t = 0; t < nt; ++t) items[s].push_back(make_int2(i, t));
        }
        b->n_items[s] = (int)items[s].size();
        off_items[s] = reserve(2 * items[s].size());
    }
    // shared-memory layout: the largest B table, knot table, warp slice and key array
    int max_T = 0, max_P = 0, max_E = 0;
    for (int i = 0; i < count; ++i) {
        const int xr = empc::nrg_host(b->nx[i]) * ((b->nx[i] + empc::nrg_host(b->nx[i]) - 1) /
                                                   empc::nrg_host(b->nx[i]));
        b->bt_floats = std::max(b->bt_floats, empc::round_up(b->m[i] * xr, 4));
        max_T = std::max(max_T, b->T[i]);
        max_P = std::max(max_P, b->P[i]);
        max_E = std::max(max_E, b->E[i]);
        for (int s = 0; s < empc::kNumBatchShapes; ++s) {
            const int nrg = empc::nrg_host(b->nx[i]);
            const int cpw = (32 / nrg) * empc::kBatchShapes[s].cands;
            const int xs = (cpw + 3) / 4 * 4;
            const int sl = empc::round_up(2 * xr * xs + (b->D[i] + 2) * xs, 4);
            b->slice_floats[s] = std::max(b->slice_floats[s], sl);
        }
    }
    b->ks_floats = 4 * max_T;
    b->key_words = empc::round_up(max_P, 4);
    b->sel_cap = std::max(std::min(2048, std::max(4 * max_E, 512)), max_E);

    // host image of the arena
    std::vector<float> img(floats, 0.0f);
    auto put = [&](size_t at, const void* src, size_t bytes) { std::memcpy(&img[at], src, bytes); };
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaStreamCreate(&b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->arena, floats * sizeof(float));
    b->result_floats = off_error + 1 - off_best;
    b->off_costs_rel = off_bcost - off_best;
    b->off_status_rel = off_bstat - off_best;
    b->off_error_rel = off_error - off_best;
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_stage, sizeof(float) * b->result_floats);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_targets, sizeof(float) * 2 * b->tgt_floats);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->tgt_done, cudaEventDisableTiming);
    if (e == cudaSuccess) std::memset(b->h_targets, 0, sizeof(float) * 2 * b->tgt_floats);
    if (e != cudaSuccess) {
        free_batch(b);
        return bfail(nullptr, EMPC_ECUDA, std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    float* base = reinterpret_cast<float*>(b->arena);
    b->h_probs.resize(count);
    b->rot.resize(count);
    for (int i = 0; i < count; ++i) {  // keep only what empc_batch_set_targets needs
        b->rot[i].rotated = tabs[i].rotated;
        b->rot[i].Vt = tabs[i].Vt;
    }
    for (int i = 0; i < count; ++i) {
        const empc_problem_desc& d = probs[i];
        const empc::HostTables& t = tabs[i];
        const Off& o = off[i];
        put(o.D, t.D.data(), sizeof(float) * t.D.size());
        put(o.BT, t.BT.data(), sizeof(float) * t.BT.size());
        put(o.qd, t.qd.data(), sizeof(float) * t.qd.size());
        put(o.rd, t.rd.data(), sizeof(float) * t.rd.size());
        if (t.dense_r) put(o.rmat, t.rmat.data(), sizeof(float) * t.rmat.size());
        put(o.gram, t.gram.data(), sizeof(float) * t.gram.size());
        put(o.ks, t.ks.data(), sizeof(empc::KnotStep) * t.ks.size());
        put(o.lo, t.lo.data(), sizeof(float) * t.lo.size());
        put(o.hi, t.hi.data(), sizeof(float) * t.hi.size());
        {
            std::vector<double> zx(d.n), zg(d.n);  // rollout coordinates (Q's eigenbasis)
            t.rotate(d.x0, zx.data(), d.n);
            t.rotate(d.x_goal, zg.data(), d.n);
            for (int k = 0; k < d.n; ++k) {
                img[off_tgt + b->tgt_off[i] + k] = (float)zx[k];
                img[off_tgt + b->tgt_floats + b->tgt_off[i] + k] = (float)zg[k];
            }
        }
        BatchProblem& bp = b->h_probs[i];
        std::memset(&bp, 0, sizeof(bp));
        empc::RolloutArgs& a = bp.a;
        a.D = base + o.D;
        a.BT = base + o.BT;
        a.qdiag = base + o.qd;
        a.rdiag = base + o.rd;
        a.rmat = t.dense_r ? base + o.rmat : nullptr;
        a.gram = base + o.gram;
        a.ktab = reinterpret_cast<const empc::KnotStep*>(base + o.ks);
        a.x0 = base + off_tgt + b->tgt_off[i];
        a.goal = base + off_tgt + b->tgt_floats + b->tgt_off[i];
        a.umin = base + o.lo;
        a.umax = base + o.hi;
        a.n = d.n;
        a.m = d.m;
        a.T = d.horizon;
        a.p = d.knots;
        a.P = d.pop;
        a.E = b->E[i];
        a.cost = base + o.cost;
        a.elite_idx = reinterpret_cast<int*>(base + o.elite);
        a.seed = d.seed;
        a.gen = reinterpret_cast<uint32_t*>(base + o.gen);
        a.sigma = d.sigma > 0.0f ? d.sigma : cfg.sigma;
        a.sigma_dev = nullptr;
        a.pc256 = cfg.p_cross_256;
        a.pm256 = cfg.p_mutate_256;
        a.gate = cfg.gate;
        bp.pop[0] = base + o.pop0;
        bp.pop[1] = base + o.pop1;
        bp.elite_cost = base + o.ecost;
        bp.best_knots = base + off_best + b->knot_off[i];
        bp.best_cost = base + off_bcost + i;
        bp.status = reinterpret_cast<int*>(base + off_bstat + i);
        bp.nx = b->nx[i];
        bp.breed_cands = empc::kBreedChunk;
        bp.breeds = (d.pop + empc::kBreedChunk - 1) / empc::kBreedChunk;
    }
    b->d_targets = base + off_tgt;
    b->d_probs = reinterpret_cast<BatchProblem*>(base + off_probs);
    b->d_counters = reinterpret_cast<unsigned*>(base + off_counters);
    b->d_error = reinterpret_cast<int*>(base + off_error);
    b->d_best_knots = base + off_best;
    b->d_best_costs = base + off_bcost;
    b->d_status = reinterpret_cast<int*>(base + off_bstat);
    for (int s = 0; s < empc::kNumBatchShapes; ++s) {
        b->d_items[s] = reinterpret_cast<int2*>(base + off_items[s]);
        put(off_items[s], items[s].data(), sizeof(int2) * items[s].size());
    }
    // per-shape tile sizes go in the descriptors at configure time
    e = cudaMemcpy(b->arena, img.data(), sizeof(float) * floats, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return bfail(nullptr, EMPC_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    }
    // autotune the launch shape on one cold generation
    float best = 1e30f;
    int best_shape = -1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int forced = cfg.tile > 0 ? cfg.tile - 1 : -1;
    for (int s = 0; s < empc::kNumBatchShapes; ++s) {
        if (forced >= 0 && s != forced) continue;
        if (configure_shape(b, s) != EMPC_OK) continue;
        for (int i = 0; i < count; ++i) {
            b->h_probs[i].tiles = tiles[s][i];
            b->h_probs[i].tile_cands = tcands[s][i];
        }
        if (cudaMemcpy(b->d_probs, b->h_probs.data(), sizeof(BatchProblem) * count,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            continue;
        float t_min = 1e30f;
        bool good = true;
        for (int rep = 0; rep < 2 && good; ++rep) {
            cudaEventRecord(e0, b->stream);
            good = enqueue_batch(b, 1, true, 0, b->stream) == cudaSuccess;
            cudaEventRecord(e1, b->stream);
            good = good && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            t_min = std::min(t_min, ms);
        }
        int errflag = 0;
        cudaMemcpy(&errflag, b->d_error, sizeof(int), cudaMemcpyDeviceToHost);
        if (good && !errflag && t_min < best) {
            best = t_min;
            best_shape = s;
        }
        cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_shape < 0) {
        free_batch(b);
        return bfail(nullptr, EMPC_EUNSUPPORTED, "no batched launch shape ran");
    }
    configure_shape(b, best_shape);
    for (int i = 0; i < count; ++i) {
        b->h_probs[i].tiles = tiles[best_shape][i];
        b->h_probs[i].tile_cands = tcands[best_shape][i];
    }
    e = cudaMemcpy(b->d_probs, b->h_probs.data(), sizeof(BatchProblem) * count, cudaMemcpyHostToDevice);
    // the tuning runs advanced the draw counters: start the real solves at generation 0
    for (int i = 0; i < count && e == cudaSuccess; ++i)
        e = cudaMemset(const_cast<uint32_t*>(b->h_probs[i].a.gen), 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        free_batch(b);
        return bfail(nullptr, EMPC_ECUDA, std::string("batch setup: ") + cudaGetErrorString(e));
    }
    b->tuned_us = best * 1000.0f;
    *out = b;
    return EMPC_OK;
}

namespace {

// Launch `generations` generations (cached graph) on the run stream.
empc_status batch_launch(empc_batch b, int generations) {
    const empc::GraphKeyB key{generations, b->has_pop ? 0 : 1, b->parity};
    cudaGraphExec_t exec = nullptr;
    auto it = b->graphs.find(key);
    if (it != b->graphs.end()) {
        exec = it->second;
    } else {
        EMPC_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_batch(b, generations, !b->has_pop, b->parity, b->stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bfail(b, EMPC_ECUDA, std::string("batch capture: ") +
                                            cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(b, EMPC_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        b->graphs[key] = exec;
    }
    EMPC_BCUDA(b, cudaGraphLaunch(exec, b->run_stream ? b->run_stream : b->stream));
    b->parity ^= generations & 1;
    b->has_pop = true;
    return EMPC_OK;
}

}  // namespace

empc_status empc_batch_solve_device(empc_batch b, int generations) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    if (generations < 1) return bfail(b, EMPC_EINVAL, "need generations >= 1");
    return batch_launch(b, generations);
}

empc_status empc_batch_set_stream(empc_batch b, void* stream) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    b->run_stream = static_cast<cudaStream_t>(stream);
    return EMPC_OK;
}

empc_status empc_batch_solve(empc_batch b, int generations, float* best_knots, float* best_costs) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    if (generations < 1 || !best_knots || !best_costs)
        return bfail(b, EMPC_EINVAL, "need generations >= 1 and output buffers");
    empc_status ls = batch_launch(b, generations);
    if (ls != EMPC_OK) return ls;
    cudaStream_t rs = b->run_stream ? b->run_stream : b->stream;
    float* st = b->h_stage;
    // best knots, best costs, statuses and the error word are one span of the arena
    EMPC_BCUDA(b, cudaMemcpyAsync(st, b->d_best_knots, sizeof(float) * b->result_floats,
                                  cudaMemcpyDeviceToHost, rs));
    EMPC_BCUDA(b, cudaStreamSynchronize(rs));
    int errflag;
    std::memcpy(&errflag, st + b->off_error_rel, sizeof(int));
    if (errflag) {
        b->has_pop = false;  // populations of an interrupted launch are not usable
        return bfail(b, EMPC_ETIMEOUT, "a batched wait ran out of time");
    }
    std::memcpy(best_knots, st, sizeof(float) * b->total_knots);
    std::memcpy(best_costs, st + b->off_costs_rel, sizeof(float) * b->count);
    for (int i = 0; i < b->count; ++i) {
        int sbits;
        std::memcpy(&sbits, st + b->off_status_rel + i, sizeof(int));
        if (sbits & 1) return bfail(b, EMPC_ENONFINITE, "problem " + std::to_string(i) + ": best cost is not finite");
    }
    return EMPC_OK;
}

empc_status empc_batch_set_targets(empc_batch b, const double* x0, const double* x_goal) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    if (!x0 || !x_goal) return bfail(b, EMPC_EINVAL, "NULL x0 / x_goal");
    size_t total = 0;
    for (int i = 0; i < b->count; ++i) total += (size_t)b->n[i];
    if (!empc::all_finite(x0, total) || !empc::all_finite(x_goal, total))
        return bfail(b, EMPC_EINVAL, "non-finite x0 / x_goal");
    // the previous copy must have read the staging buffer before it is rewritten
    EMPC_BCUDA(b, cudaEventSynchronize(b->tgt_done));
    float* h = b->h_targets;
    size_t at = 0;
    std::vector<double> zx, zg;
    for (int i = 0; i < b->count; ++i) {
        float* hx = h + b->tgt_off[i];
        float* hg = h + b->tgt_floats + b->tgt_off[i];
        zx.resize(b->n[i]);
        zg.resize(b->n[i]);
        b->rot[i].rotate(x0 + at, zx.data(), b->n[i]);
        b->rot[i].rotate(x_goal + at, zg.data(), b->n[i]);
        for (int k = 0; k < b->n[i]; ++k) {
            hx[k] = (float)zx[k];
            hg[k] = (float)zg[k];
        }
        at += (size_t)b->n[i];
    }
    cudaStream_t rs = b->run_stream ? b->run_stream : b->stream;
    EMPC_BCUDA(b, cudaMemcpyAsync(b->d_targets, h, sizeof(float) * 2 * b->tgt_floats,
                                  cudaMemcpyHostToDevice, rs));
    EMPC_BCUDA(b, cudaEventRecord(b->tgt_done, rs));
    return EMPC_OK;
}

empc_status empc_batch_reset(empc_batch b) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    b->has_pop = false;
    return EMPC_OK;
}

empc_status empc_batch_get_state(empc_batch b, int index, float* dev_pop, float* dev_cost,
                                 int* dev_elite) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    if (index < 0 || index >= b->count) return bfail(b, EMPC_EINVAL, "index out of range");
    if (!b->has_pop) return bfail(b, EMPC_ESTATE, "no population yet (solve first)");
    const BatchProblem& bp = b->h_probs[index];
    const size_t DP = (size_t)b->D[index] * b->P[index];
    cudaStream_t rs = b->run_stream ? b->run_stream : b->stream;
    if (dev_pop)
        EMPC_BCUDA(b, cudaMemcpyAsync(dev_pop, bp.pop[b->parity], sizeof(float) * DP,
                                      cudaMemcpyDeviceToDevice, rs));
    if (dev_cost)
        EMPC_BCUDA(b, cudaMemcpyAsync(dev_cost, bp.a.cost, sizeof(float) * b->P[index],
                                      cudaMemcpyDeviceToDevice, rs));
    if (dev_elite)
        EMPC_BCUDA(b, cudaMemcpyAsync(dev_elite, bp.a.elite_idx, sizeof(int) * b->E[index],
                                      cudaMemcpyDeviceToDevice, rs));
    EMPC_BCUDA(b, cudaStreamSynchronize(rs));
    return EMPC_OK;
}

empc_status empc_batch_get_info(empc_batch b, empc_batch_info* info) {
    if (!b || !info) return bfail(b, EMPC_EINVAL, "NULL batch or info");
    std::memset(info, 0, sizeof(*info));
    info->count = b->count;
    info->total_knots = b->total_knots;
    info->ctas = b->grid;
    info->warps_per_cta = empc::kBatchShapes[b->shape].wpc;
    info->cands_per_lane = empc::kBatchShapes[b->shape].cands;
    info->items_per_generation = b->n_items[b->shape];
    info->state_steps_per_generation = b->state_steps_per_gen;
    info->tuned_us = b->tuned_us;
    info->h2d_bytes_targets = (int)(sizeof(float) * 2 * b->tgt_floats);
    info->d2h_bytes_solve = (int)(sizeof(float) * b->result_floats);
    return EMPC_OK;
}

empc_status empc_batch_inject_stall(empc_batch b, int problem, double timeout_s) {
    if (!b) return bfail(nullptr, EMPC_EINVAL, "NULL batch");
    if (problem >= b->count || !(timeout_s > 0.0))
        return bfail(b, EMPC_EINVAL, "problem out of range or bad timeout");
    b->stall_problem = problem < 0 ? -1 : problem;
    b->timeout_ns = (unsigned long long)(timeout_s * 1e9);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return EMPC_OK;
}

void empc_batch_destroy(empc_batch b) { free_batch(b); }

const char* empc_batch_last_error(empc_batch b) { return b ? b->err.c_str() : empc_last_error(nullptr); }

}  // extern "C"
