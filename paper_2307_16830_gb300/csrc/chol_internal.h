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
// Supernodes have at most this many columns; a large supernode's panel
// (and its update matrix, when both fit) is staged in at most this many
// doubles of shared memory.
constexpr int kCholMaxWidth = 64;
constexpr int kCholPanelDoubles = 20480;
// Small supernodes (one warp each): at most this many rows and columns.
constexpr int kCholWarpRows = 32;
constexpr int kCholWarpCols = 8;
// A child's rows below its columns fit a row-map scratch of this size.
constexpr int kCholMaxRelRows = 4096;

// Supernodes level_sn[begin .. begin + count): either all by a whole block
// each (n_large == count), with `stage` doubles of shared memory (the
// largest block staging), or all by a warp each (n_large == 0), with
// `stage` doubles per warp (the largest panel plus update matrix of the
// group); then the update-matrix tiles tiles[tile_begin .. + n_tiles) in a
// second launch.
cudaError_t launch_chol_factor_level(const CholDev& d, int begin, int count, int n_large,
                                     double tol, int stage, const int4* tiles, int tile_begin,
                                     int n_tiles, cudaStream_t s);
// Dynamic shared memory of such a launch, and the opt-in that lets the
// factor kernel use `bytes` of it (set once, before any launch or capture).
size_t chol_factor_smem_bytes(int count, int n_large, int stage);
cudaError_t chol_allow_smem(size_t bytes);
cudaError_t launch_chol_fwd_level(const CholDev& d, int begin, int count, int n_large, double* y,
                                  cudaStream_t s);
cudaError_t launch_chol_bwd_level(const CholDev& d, int begin, int count, int n_large, double* x,
                                  cudaStream_t s);

}  // namespace acopf
