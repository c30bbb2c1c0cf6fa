// Fused crossover + mutation kernel (and the cold-start draw): the breeding
// lines of Algorithm 1 for every candidate of one generation (Sec. V: two
// parents drawn from the elites, each knot inherited from one of them, a
// gated N(0, sigma) perturbation per input, clipped to the bounds; elites
// copied unchanged).  One thread per (candidate, 4-knot group), so even a
// few thousand candidates give the GPU enough warps to hide the latency of
// the Philox rounds and the parent-knot gathers; the rollout kernel that
// follows only loads the bred knots.  Threads of a block take consecutive
// candidates, so every population store is coalesced.
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

constexpr int kBreedThreads = 128;

__global__ void __launch_bounds__(kBreedThreads) breed_kernel(const RolloutArgs a) {
    pdl_launch_dependents();
    // the elites, the generation counter and the parents' knots come from the
    // previous kernels
    pdl_wait_primary();
    const int c = a.cand_begin + blockIdx.x * kBreedThreads + threadIdx.x;
    if (c >= a.P) return;
    const uint32_t gen = a.gen ? *a.gen : 0u;
    const int D = a.m * a.p;
    if (a.mode == kWarm) {
        const int quad = blockIdx.y;
        int s1, s2;
        parents_of<false>(a, c, gen, s1, s2);
        float v[4];
        breed_quad<false>(a, c, quad, gen, s1, s2, v);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (quad * 4 + w < D) a.pop_out[(size_t)(quad * 4 + w) * a.P + c] = v[w];
    } else {
        const int quad = blockIdx.y;
        float v[4];
        breed_quad<false>(a, c, quad, gen, 0, -1, v);
#pragma unroll
        for (int w = 0; w < 4; ++w)
            if (quad * 4 + w < D) a.pop_out[(size_t)(quad * 4 + w) * a.P + c] = v[w];
    }
}

}  // namespace

cudaError_t launch_breed(const RolloutArgs& a, cudaStream_t st) {
    if (a.mode != kWarm && a.mode != kCold) return cudaErrorInvalidValue;
    const int count = a.P - a.cand_begin;
    if (count <= 0) return cudaSuccess;
    const int D = a.m * a.p;
    const dim3 grid((count + kBreedThreads - 1) / kBreedThreads, (D + 3) / 4);
    return launch_kernel(breed_kernel, grid, dim3(kBreedThreads), 0, st, a.pdl != 0, a);
}

}  // namespace empc
