// Kernels around the sparse Cholesky factorization of M_cond: the value
// gather from the lower CSR of the assembled matrix into the permuted full
// pattern the factorization reads, and the symmetric permutation of
// right-hand sides and solutions.
#include "acopf_internal.h"

namespace acopf {
namespace {

constexpr int kPermThreads = 256;

// out[t] = in[idx[t]]
__global__ void __launch_bounds__(kPermThreads) k_gather(double* __restrict__ out,
                                                         const double* __restrict__ in,
                                                         const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[t] = in[__ldg(idx + t)];
}

// out[idx[t]] = in[t]  (idx a permutation)
__global__ void __launch_bounds__(kPermThreads) k_scatter(double* __restrict__ out,
                                                          const double* __restrict__ in,
                                                          const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[__ldg(idx + t)] = in[t];
}

int perm_grid(int n) { return n > 0 ? min(ceil_div(n, kPermThreads), 4096) : 0; }

}  // namespace

cudaError_t launch_gather(double* out, const double* in, const int32_t* idx, int n,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<perm_grid(n), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_scatter(double* out, const double* in, const int32_t* idx, int n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter<<<perm_grid(n), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

}  // namespace acopf
