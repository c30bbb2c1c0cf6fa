// Internal declarations shared by the EMPC CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace empc {

// Breeding mode of the fused breed + rollout + cost kernel.
enum BreedMode : int { kEval = 0, kCold = 1, kWarm = 2 };

// Per-step knot table entry: u_k = w0 U_idx1 + w1 U_idx1+1 (Sec. IV-C).
struct KnotStep {
    int idx1;
    float w0;
    float w1;
    int pad;
};

// Everything the fused kernel reads.  Device pointers, FP32.
struct RolloutArgs {
    // model
    const float* D;      // [n][n] row-major, D = A_d - I (delta form)
    const float* BT;     // [m][n] = B_d transposed
    const float* qdiag;  // [n]   state weights: diag(Q), or Q's eigenvalues when the
                         //       rollouts run in Q's eigenbasis (non-diagonal Q)
    const float* rdiag;  // [m]   diagonal of R (read when rmat is null)
    const float* rmat;   // [m][m] symmetric R when it is not diagonal, else null
    const float* gram;   // [2p]  input-cost Gram: diag W_aa (p), off-diag W_a,a+1 (p)
    const KnotStep* ktab;  // [T]
    const float* x0;     // [n]
    const float* goal;   // [n]
    const float* umin;   // [m]
    const float* umax;   // [m]
    int n, m, T, p, P;
    // population
    const float* pop_in;  // warm: previous population; eval: population to score
    float* pop_out;       // cold/warm: the bred population (SoA [m p][P])
    float* cost;          // [P]
    const int* elite_idx;  // [E] previous elites in rank order (warm)
    int E;
    // breeding
    int mode;
    uint64_t seed;
    const uint32_t* gen;  // device generation counter
    float sigma;
    const float* sigma_dev;  // if set, the mutation sigma is read here (set per solve)
    int pc256, pm256, gate;
    // state-box hook (Sec. V: hard stops and non-convex state costs inside the
    // simulation): [3][n] lo, hi, rho on the device, read when box_mode != 0;
    // box_mode bit 0 stops the state at [lo, hi], bit 1 adds rho d^2
    const float* box;
    int box_mode;
    // constant disturbance w_d of Eq. first_order_integration: [n] on the
    // device, or null (zero)
    const float* wd;
    int cand_begin;  // first candidate this launch covers (later ones up to P)
    int pdl;         // launch with programmatic stream serialization
    int* status;     // bit 1 (value 2): a bounded device wait gave up (may be null)
    // tensor-core rollout only, on the device or null: [0] the step at which
    // the MMA issuer stops (a host-side stall injection; -1: none), [1] the
    // limit of each of its waits in microseconds (null: one second)
    const int* inject;
};

// Launch `kern` with an optional programmatic-stream-serialization attribute
// (programmatic dependent launch on the previous kernel of the stream).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t st, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Dynamic shared memory above 48 KiB needs the kernel's limit raised, and the
// limit is kept per device: cap[d] records what was set on device d (zero:
// nothing yet).  The attribute call is made only when the need grows, so a
// launch recorded into a CUDA graph after the first one makes none.
constexpr int kMaxDevices = 64;
template <typename Kern>
cudaError_t raise_smem_limit(Kern kern, size_t smem, int (&cap)[kMaxDevices]) {
    if (smem <= 48u * 1024u) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if ((int)smem <= cap[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cap[dev] = (int)smem;
    return e;
}

// Adjoint-gradient / refinement kernel arguments (grad.cu).
struct GradArgs {
    const float* D;
    const float* BT;
    const float* qdiag;
    const float* rdiag;
    const float* rmat;    // dense symmetric R [m][m], or null (diagonal, rdiag)
    const float* gram;
    const KnotStep* ktab;
    const float* x0;
    const float* goal;
    const float* umin;
    const float* umax;
    int n, m, T, p;
    const float* pop_in;  // SoA knots, stride ld_in
    int ld_in;
    const int* index;     // candidate c reads column index[c] (null: column c)
    int count;            // candidates processed
    float* grad;          // SoA gradient output, stride ld_grad (steps == 0)
    int ld_grad;
    float* cost;          // cost[count] of the final knots (may be null)
    float* pop_out;       // refined knots, column c, stride ld_out (steps > 0)
    int ld_out;
    int ce;               // checkpoint interval
    int steps;            // projected-gradient steps (0: gradient only)
    float eta;            // step size
    const float* wd;      // constant disturbance w_d [n], or null (zero)
};

cudaError_t launch_grad(const GradArgs& a, int nx, int cands, int wpc, cudaStream_t st);
size_t grad_smem_bytes(int nx, int nrg, int cands, int wpc, int n, int m, int p, int T, int ce);

// Condensed quadratic-form costs J = U'HU + g'U + c0 of a population
// (condensed.cu).  H is Dp x Dp (zero-padded, symmetric), g and c0 on device.
struct CondArgs {
    const float* H;    // [Dp][Dp]
    const float* g;    // [Dp] (zero past D)
    const float* c0;   // [1]
    const float* pop;  // SoA knots [D][P]
    float* cost;       // [P]
    int D, Dp, P;
};
int condensed_pad(int D);
bool condensed_supported(int D);
cudaError_t launch_condensed(const CondArgs& a, cudaStream_t st, bool pdl);
// The same costs with the product on the tensor cores (condensed_tc.cu):
// tcgen05 kind::tf32 with head/remainder splits, for padded Dp <= 256;
// status bit 2 (value 2) reports a bounded wait that gave up.
bool condensed_tc_supported(int Dp);
cudaError_t launch_condensed_tc(const CondArgs& a, int* status, cudaStream_t st, bool pdl);

// Fused crossover + mutation (warm) or cold-start draw of candidates
// cand_begin .. P-1 into pop_out (breed.cu).
cudaError_t launch_breed(const RolloutArgs& a, cudaStream_t st);

// BF16 tensor-core rollout (rollout_bf16.cu): n <= 128, m <= 64.
// The product in `groups` (1, 2 or 4) MMA groups; evaluates pop_in (kEval).
cudaError_t launch_rollout_bf16(const RolloutArgs& a, cudaStream_t st);
bool rollout_bf16_supported(int n, int m, int T);
size_t rollout_bf16_smem_bytes(int T);
int rollout_bf16_threads();

// Rollout tile.  kind 0 (block): ceil(n/rows) threads per candidate group,
// `groups` candidate groups per CTA, one block barrier per step.  kind 1
// (warp): each warp owns whole candidates (32/nrg groups of `cands`), `groups`
// warps per CTA, one warp barrier per step.
struct TileShape {
    int kind;   // 0 block, 1 warp, 2 BF16 tensor-core tile of 128 candidates
    int nx;     // compiled state dimension (>= n)
    int rows;   // state rows per thread
    int cands;  // candidates per thread (1, 2 or 4)
    int groups; // candidate groups per CTA (block) or warps per CTA (warp)
};

// Launch the fused kernel.  Returns cudaErrorInvalidConfiguration when the
// shape is not compiled or does not fit.
cudaError_t launch_rollout(const RolloutArgs& a, const TileShape& s, cudaStream_t st);
// Shapes compiled for state dimension n, in autotuning order.
int rollout_shapes(int n, TileShape* out, int cap);
// Whether the shape fits (registers, threads, shared memory) for this problem.
bool rollout_shape_supported(const TileShape& s, int n, int m, int p, int T);
size_t rollout_smem_bytes(const TileShape& s, int n, int m, int p, int T);
int rollout_threads(const TileShape& s, int n);
int rollout_cands_per_cta(const TileShape& s, int n);

// Per-family entry points (rollout_block.cu, rollout_warp.cu).
cudaError_t launch_rollout_block(const RolloutArgs& a, const TileShape& s, cudaStream_t st);
cudaError_t launch_rollout_warp(const RolloutArgs& a, const TileShape& s, cudaStream_t st);
int block_max_threads(const TileShape& s);
int warp_max_threads(const TileShape& s);
int warp_nrg(int nx);
// The warp family's compiled state class for n <= 64 (4 .. 64), else 0.
int warp_class_nx(int n);

// Elite selection: E lowest of P costs by (cost, index), NaN as +inf.
// Writes elite_idx[E], elite_cost[E], best_knots[m p] and increments *gen.
cudaError_t launch_select(const float* cost, int P, int E, const float* pop, int D,
                          int* elite_idx, float* elite_cost, float* best_knots,
                          float* best_cost, uint32_t* gen, int* status, cudaStream_t st,
                          bool pdl = false);

// z = Vt x and zg = Vt g for device vectors of n <= 128 entries: FP64 sums
// of the FP64 rotation Vt [n][n] (row i = eigenvector i of Q), rounded once
// to FP32 (rotate.cu).
cudaError_t launch_rotate(const double* Vt, const float* x, const float* g, float* zx, float* zg,
                          int n, cudaStream_t st);

// Record a failure message for empc_last_error(NULL) on this thread; returns s.
int set_thread_error(int s, const char* msg);

}  // namespace empc
