// Rotation of start states and goals into the eigenbasis of a non-diagonal
// state weight Q (z = V' x), for device inputs.  With Q_s = V diag(lambda) V'
// the cost (x - g)' Q (x - g) of Eq. mpc_problem is (z - V'g)' diag(lambda)
// (z - V'g), and the model becomes z_{k+1} = V'A V z_k + V'B u_k: the same
// cost for every knot vector, with a diagonal weight in the rollouts.
#include <cuda_runtime.h>

#include "empc_internal.h"

namespace empc {
namespace {

// Thread i < n: zx[i]; thread n + i: zg[i].  FP64 sums, rounded once.
__global__ void rotate_kernel(const double* Vt, const float* x, const float* g, float* zx,
                              float* zg, int n) {
    const int t = threadIdx.x;
    if (t >= 2 * n) return;
    const int i = t < n ? t : t - n;
    const float* v = t < n ? x : g;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(Vt[(size_t)i * n + j], (double)v[j], s);
    (t < n ? zx : zg)[i] = (float)s;
}

}  // namespace

cudaError_t launch_rotate(const double* Vt, const float* x, const float* g, float* zx, float* zg,
                          int n, cudaStream_t st) {
    if (n < 1 || n > 128) return cudaErrorInvalidValue;
    rotate_kernel<<<1, 256, 0, st>>>(Vt, x, g, zx, zg, n);
    return cudaGetLastError();
}

}  // namespace empc
