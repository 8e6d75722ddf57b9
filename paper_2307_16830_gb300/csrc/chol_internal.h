// Device view of the supernodal factor and the launchers of chol.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace acopf {

// Device copies of the symbolic arrays (see symbolic.h) and the factor.
struct CholDev {
  int32_t n;
  const int32_t* sn_first;   // ns + 1
  const int32_t* sn_rowptr;  // ns + 1
  const int32_t* rowidx;
  const int64_t* sn_off;     // ns + 1
  const int32_t* kid_ptr;    // ns + 1
  const int32_t* kid;
  const int32_t* rel_off;    // ns
  const int32_t* relmap;
  const int64_t* u_off;      // ns + 1
  const int64_t* z_off;      // ns + 1
  const int32_t* level_sn;   // ns
  double* Lx;                // the supernodal blocks
  double* Ux;                // the update matrices
  double* Zx;                // the update vectors of a solve
  int32_t* bad;              // smallest failed pivot column (>= n: none)
};

cudaError_t launch_gather(double* out, const double* in, const int32_t* idx, int n,
                          cudaStream_t s);
cudaError_t launch_scatter(double* out, const double* in, const int32_t* idx, int n,
                           cudaStream_t s);
cudaError_t launch_chol_assemble(double* Lx, const int64_t* amap, const double* kvals,
                                 int64_t nnz, cudaStream_t s);
// Supernodes have at most this many columns.
constexpr int kCholMaxWidth = 64;

// One level of the supernodal tree: level_sn[begin .. begin + count), the
// first n_large of them handled by a whole block each (panel staged in
// `staged` doubles of shared memory when it fits, update matrix by the
// tiles[tile_begin .. + n_tiles) of a second launch), the rest by a warp.
cudaError_t launch_chol_factor_level(const CholDev& d, int begin, int count, int n_large,
                                     double tol, int staged, const int4* tiles, int tile_begin,
                                     int n_tiles, cudaStream_t s);
cudaError_t launch_chol_fwd_level(const CholDev& d, int begin, int count, int n_large, double* y,
                                  cudaStream_t s);
cudaError_t launch_chol_bwd_level(const CholDev& d, int begin, int count, int n_large, double* x,
                                  cudaStream_t s);

}  // namespace acopf
