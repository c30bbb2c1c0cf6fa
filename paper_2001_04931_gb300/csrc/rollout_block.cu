// Fused breed + knot expansion + rollout + cost, block-synchronous family,
// and the shape dispatch shared by both families.
//
// One CTA owns a tile of candidates for the whole horizon (Algorithm 1: each
// simulation block breeds its candidates, simulates them and accumulates the
// stage cost; Sec. V).  Unlike the paper's one-block-per-simulation,
// one-thread-per-state layout, a CTA here steps a whole candidate tile as a
// small GEMM per time step.  Thread (rg, cg) keeps rows rg*R .. rg*R+R-1 of
// D = A_d - I in registers for the whole rollout (D-stationary) and updates
// them for C candidates; the state tile X[k][cand] is double-buffered in
// shared memory (one block barrier per step).  Costs are reduced over the row
// groups in a fixed order.  This family covers every state size up to 128
// (R = 1 for n > 64); the warp-synchronous family (rollout_warp.cu) covers
// n <= 64 without block barriers.
#include <cuda_runtime.h>

#include "rollout_common.cuh"

namespace empc {
namespace {

struct BlockLayout {
    int xs, off_x, off_u, off_bt, off_k, off_par, off_box, total;
    __host__ __device__ BlockLayout(int nx, int ptile, int m, int p, int T) {
        xs = round_up(ptile, 4);
        off_x = 0;
        off_u = off_x + 2 * nx * xs;
        off_bt = off_u + m * p * xs;
        off_k = round_up(off_bt + m * nx, 4);
        off_par = off_k + 4 * T;
        off_box = off_par + 2 * xs;
        total = off_box + 4 * nx;
    }
};

template <int NX, int R, int C>
__global__ void rollout_block_kernel(const RolloutArgs a) {
    extern __shared__ __align__(16) float smem[];
    const int n = a.n, m = a.m;
    const int nrg = (n + R - 1) / R;
    const int ncg = blockDim.x / nrg;
    const int ptile = ncg * C;
    const BlockLayout L(NX, ptile, m, a.p, a.T);
    const int xs = L.xs;
    float* X = smem + L.off_x;
    float* Us = smem + L.off_u;
    float* BTs = smem + L.off_bt;
    KnotStep* ks = reinterpret_cast<KnotStep*>(smem + L.off_k);
    int* par = reinterpret_cast<int*>(smem + L.off_par);
    const int c0 = a.cand_begin + blockIdx.x * ptile;
    const int tid = threadIdx.x;
    const int rg = tid % nrg;
    const int cg = tid / nrg;
    pdl_launch_dependents();

    // the initial state and the model tables, with batched loads (none
    // depends on the previous kernel)
    batched_fill(X, 2 * NX * xs, tid, blockDim.x, [&](int i) {
        const int k = (i / xs) % NX;
        return (i < NX * xs && k < n) ? a.x0[k] : 0.0f;
    });
    batched_fill(BTs, m * NX, tid, blockDim.x, [&](int i) {
        const int row = i % NX, col = i / NX;
        return row < n ? a.BT[col * n + row] : 0.0f;
    });
    batched_fill(reinterpret_cast<float*>(ks), 4 * a.T, tid, blockDim.x,
                 [&](int i) { return reinterpret_cast<const float*>(a.ktab)[i]; });
    float* Bx = smem + L.off_box;
    const bool hooks = has_hooks(a);
    if (hooks) stage_box(a, Bx, NX, tid, blockDim.x);
    float d[R][NX], qd[R], gl[R], xo[R][C], jsum[C];
    load_rows<NX, R, C>(a, rg * R, d, qd, gl, xo);
    pdl_wait_primary();
    const uint32_t gen = a.gen ? *a.gen : 0u;
    fill_knots<false>(a, Us, xs, par, c0, ptile, gen, tid, blockDim.x);  // ends with a barrier
    if (hooks)
        horizon_loop<NX, R, C, false, true>(a, d, X, NX, xs, BTs, NX, Us, ks, rg * R, cg * C, xo,
                                            qd, gl, jsum, Bx);
    else
        horizon_loop<NX, R, C, false>(a, d, X, NX, xs, BTs, NX, Us, ks, rg * R, cg * C, xo, qd,
                                      gl, jsum);

    // reduce the row groups in order, then add the input cost
    float* Jred = X;  // every state read is done (barrier at the end of the loop)
#pragma unroll
    for (int c = 0; c < C; ++c) Jred[rg * xs + cg * C + c] = jsum[c];
    __syncthreads();
    for (int t = tid; t < ptile; t += blockDim.x) {
        const int cand = c0 + t;
        if (cand >= a.P) continue;
        float J = 0.0f;
        for (int g = 0; g < nrg; ++g) J += Jred[g * xs + t];
        J += input_cost_part(a, Us, xs, t, 0, 1);
        a.cost[cand] = finite_or_inf(J);
    }
}

template <int NX, int R, int C>
cudaError_t launch_shape(const RolloutArgs& a, int groups, cudaStream_t st) {
    const int nrg = (a.n + R - 1) / R;
    const int ptile = groups * C;
    const BlockLayout L(NX, ptile, a.m, a.p, a.T);
    const size_t smem = sizeof(float) * (size_t)L.total;
    auto kern = rollout_block_kernel<NX, R, C>;
    static int smem_cap[kMaxDevices] = {};
    if (cudaError_t e = raise_smem_limit(kern, smem, smem_cap); e != cudaSuccess) return e;
    const int grid = (a.P - a.cand_begin + ptile - 1) / ptile;
    if (grid <= 0) return cudaSuccess;
    return launch_kernel(kern, dim3(grid), dim3(nrg * groups), smem, st, a.pdl != 0, a);
}

template <int NX, int R, int C>
int max_threads_of() {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, rollout_block_kernel<NX, R, C>) != cudaSuccess) return 0;
    return fa.maxThreadsPerBlock;
}

#define EMPC_BLOCK_NX_CASES(X) X(4, 2) X(8, 2) X(16, 2) X(24, 2) X(32, 2) X(40, 2) X(48, 2) \
    X(56, 2) X(64, 2) X(128, 1)

}  // namespace

cudaError_t launch_rollout_block(const RolloutArgs& a, const TileShape& s, cudaStream_t st) {
#define EMPC_CASE(NXV, RV)                                                       \
    if (s.nx == NXV && s.rows == RV) {                                           \
        if (s.cands == 2) return launch_shape<NXV, RV, 2>(a, s.groups, st);      \
        if (s.cands == 4) return launch_shape<NXV, RV, 4>(a, s.groups, st);      \
    }
    EMPC_BLOCK_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return cudaErrorInvalidConfiguration;
}

int block_max_threads(const TileShape& s) {
#define EMPC_CASE(NXV, RV)                                              \
    if (s.nx == NXV && s.rows == RV) {                                  \
        if (s.cands == 2) return max_threads_of<NXV, RV, 2>();          \
        if (s.cands == 4) return max_threads_of<NXV, RV, 4>();          \
    }
    EMPC_BLOCK_NX_CASES(EMPC_CASE)
#undef EMPC_CASE
    return 0;
}

// ---------------------------------------------------------------------------
// Shape dispatch for both families.
// ---------------------------------------------------------------------------
static int compiled_nx(int n) {
    static const int kNx[] = {4, 8, 16, 24, 32, 40, 48, 56, 64, 128};
    for (int v : kNx)
        if (n <= v) return v;
    return 0;
}

int warp_class_nx(int n) {
    const int nx = compiled_nx(n);
    return nx <= 64 ? nx : 0;
}

int rollout_shapes(int n, TileShape* out, int cap) {
    const int nx = compiled_nx(n);
    int k = 0;
    if (nx == 0) return 0;
    auto push = [&](TileShape s) {
        if (k < cap) out[k] = s;
        ++k;
    };
    if (nx <= 64) {  // warp-synchronous family
        const int nrg = warp_nrg(nx);
        const int rows = (nx + nrg - 1) / nrg;
        // 7 warps a CTA: where 8 leave SMs idle (4096 candidates of 2 per
        // lane fill 128 CTAs of 8 warps), 147 CTAs of 7 use nearly all 152
        for (int cands : {2, 1, 4})
            for (int wpc : {1, 2, 4, 8, 7}) push(TileShape{1, nx, rows, cands, wpc});
    }
    const int rows = nx == 128 ? 1 : 2;
    const int nrg = (n + rows - 1) / rows;
    for (int cands : {2, 4})
        for (int g = 1; g <= 64; g *= 2)
            if (nrg * g >= 32 && nrg * g <= 1024) push(TileShape{0, nx, rows, cands, g});
    return k;
}

int rollout_threads(const TileShape& s, int n) {
    if (s.kind == 2) return rollout_bf16_threads();
    if (s.kind == 1) return 32 * s.groups;
    return ((n + s.rows - 1) / s.rows) * s.groups;
}

int rollout_cands_per_cta(const TileShape& s, int n) {
    if (s.kind == 2) return 128;
    if (s.kind == 1) return s.groups * (32 / warp_nrg(s.nx)) * s.cands;
    (void)n;
    return s.groups * s.cands;
}

size_t rollout_smem_bytes(const TileShape& s, int n, int m, int p, int T) {
    if (s.kind == 2) return rollout_bf16_smem_bytes(T);
    if (s.kind == 1) {
        const int nrg = warp_nrg(s.nx);
        const int xr = nrg * s.rows;
        const int cpw = (32 / nrg) * s.cands;
        const int xsw = round_up(cpw, 4);
        const int per_warp = round_up(2 * xr * xsw + m * p * xsw + 2 * xsw, 4);
        const int head = round_up(m * xr, 4) + 4 * T + round_up(n * (s.nx + 2), 4) +
                         round_up(4 * xr, 4) + round_up(xr, 4);
        return sizeof(float) * (size_t)(head + s.groups * per_warp);
    }
    const BlockLayout L(s.nx, s.groups * s.cands, m, p, T);
    return sizeof(float) * (size_t)L.total;
}

bool rollout_shape_supported(const TileShape& s, int n, int m, int p, int T) {
    if (s.nx != compiled_nx(n)) return false;
    const int threads = rollout_threads(s, n);
    if (threads <= 0 || threads > 1024) return false;
    const int maxt = s.kind == 1 ? warp_max_threads(s) : block_max_threads(s);
    if (maxt < threads) return false;
    return rollout_smem_bytes(s, n, m, p, T) <= 227u * 1024u;
}

cudaError_t launch_rollout(const RolloutArgs& a, const TileShape& s, cudaStream_t st) {
    if (s.kind == 2) return launch_rollout_bf16(a, st);
    if (s.nx != compiled_nx(a.n)) return cudaErrorInvalidConfiguration;
    return s.kind == 1 ? launch_rollout_warp(a, s, st) : launch_rollout_block(a, s, st);
}

}  // namespace empc
