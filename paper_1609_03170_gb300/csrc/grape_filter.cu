// grape_filter.cu - Gaussian filtering of the controls and its chain rule
// (App. A of the paper, after Motzoi et al.).
//
// N piecewise-constant controls u[j][k] of length Dt are smoothed into M
// subpixel amplitudes s[n][k] of length dt, the slices the propagation then
// runs on:  s[n][k] = sum_j T_k[n][j] u[j][k]  with the error-function
// transfer matrix  T_k[n][j] = (erf(w0_k (n dt - j Dt)/2) - erf(w0_k (n dt -
// (j+1) Dt)/2)) / 2  (0-based n, j).  The gradient with respect to the
// controls is the transposed sum  g_u[j][k] = sum_n T_k[n][j] g_s[n][k].
//
// T is computed on the fly in FP64 (CUDA's erf).  erf(x) rounds to +-1
// exactly for |x| > 5.93, so an entry is exactly zero once both arguments
// pass kSat = 6.5 on the same side: each output sums only the band of terms
// that can be non-zero, in ascending index order, and equals the dense sum
// up to those exact zeros.  One thread per output; the work is a few erf
// per term, negligible next to the propagation it feeds.
#include "grape_internal.h"

#include <cmath>

namespace {

constexpr double kSat = 6.5;

__device__ __forceinline__ double transfer(double t, int j, double Dt, double w) {
    return 0.5 * (erf(0.5 * w * (t - j * Dt)) - erf(0.5 * w * (t - (j + 1) * Dt)));
}

__global__ void __launch_bounds__(256) filter_apply_kernel(const FilterArgs a) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)a.M * a.R) return;
    const int n = (int)(idx / a.R), k = (int)(idx % a.R);
    const double t = n * a.dt, w = a.w0[k];
    const double reach = 2.0 * kSat / w;           // |t - edge| beyond which erf saturates
    const int j0 = max(0, (int)floor((t - reach) / a.Dt) - 1);
    const int j1 = min(a.N - 1, (int)ceil((t + reach) / a.Dt));
    double acc = 0.0;
    for (int j = j0; j <= j1; ++j) acc = fma(transfer(t, j, a.Dt, w), a.in[(size_t)j * a.R + k], acc);
    a.out[(size_t)n * a.R + k] = acc;
}

__global__ void __launch_bounds__(256) filter_adjoint_kernel(const FilterArgs a) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)a.N * a.R) return;
    const int j = (int)(idx / a.R), k = (int)(idx % a.R);
    const double w = a.w0[k];
    const double reach = 2.0 * kSat / w;
    const int n0 = max(0, (int)floor((j * a.Dt - reach) / a.dt) - 1);
    const int n1 = min(a.M - 1, (int)ceil(((j + 1) * a.Dt + reach) / a.dt) + 1);
    double acc = 0.0;
    for (int n = n0; n <= n1; ++n)
        acc = fma(transfer(n * a.dt, j, a.Dt, w), a.in[(size_t)n * a.R + k], acc);
    a.out[(size_t)j * a.R + k] = acc;
}

}  // namespace

cudaError_t grape_launch_filter(const FilterArgs &a, bool adjoint, cudaStream_t s) {
    const long long n = (long long)(adjoint ? a.N : a.M) * a.R;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (adjoint) filter_adjoint_kernel<<<blocks, 256, 0, s>>>(a);
    else filter_apply_kernel<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}
