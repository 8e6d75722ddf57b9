// Numeric sparse Cholesky factorization of M_cond and solves with it.
//
// The factor L of P M_cond P' is stored in supernodes (dense column-major
// blocks, see symbolic.h).  The factorization is multifrontal and runs the
// supernodal elimination tree level by level, leaves first: one block per
// supernode of a level (1) adds its children's update matrices into its
// panel and its own update matrix (extend-add, one child after the other),
// (2) factors its panel: a dense Cholesky of the diagonal block and the
// scaled rows below it, and (3) subtracts L21 L21' from its update matrix,
// which its parent adds in turn.  A pivot that is not above the tolerance
// (or is NaN) is recorded (the smallest column, so the result does not
// depend on the schedule) and replaced by 1 so the arithmetic stays finite;
// the factorization then counts as failed.  The forward solve passes update
// vectors up the tree the same way; the backward solve runs the levels root
// first, each supernode reading its ancestors' solved entries.  Every sum
// has a fixed order: results are bit-reproducible.
#include "chol_internal.h"

#include <algorithm>

namespace acopf {
namespace {

constexpr int kCholThreads = 256;
constexpr int kMaxWidth = kCholMaxWidth;
constexpr int kPanelDoubles = kCholPanelDoubles;
// row-map scratch: a child's rows (a large supernode's children have at most
// kRelScratch rows below their columns; a small one's at most kCholWarpRows)
constexpr int kRelScratch = kCholMaxRelRows;
static_assert(kRelScratch >= kCholWarpRows * (kCholThreads / 32), "warp row-map slices");
constexpr int kPermThreads = 256;

__global__ void __launch_bounds__(kPermThreads) k_gather(double* __restrict__ out,
                                                         const double* __restrict__ in,
                                                         const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[t] = in[__ldg(idx + t)];
}

__global__ void __launch_bounds__(kPermThreads) k_scatter(double* __restrict__ out,
                                                          const double* __restrict__ in,
                                                          const int32_t* __restrict__ idx, int n) {
  for (int t = blockIdx.x * kPermThreads + threadIdx.x; t < n; t += gridDim.x * kPermThreads)
    out[__ldg(idx + t)] = in[t];
}

// Lx[amap[k]] = kvals[k] (Lx zeroed before)
__global__ void __launch_bounds__(kPermThreads) k_chol_assemble(double* __restrict__ Lx,
                                                                const int64_t* __restrict__ amap,
                                                                const double* __restrict__ kvals,
                                                                int64_t nnz) {
  for (int64_t k = int64_t(blockIdx.x) * kPermThreads + threadIdx.x; k < nnz;
       k += int64_t(gridDim.x) * kPermThreads)
    Lx[__ldg(amap + k)] = kvals[k];
}

// A supernode is handled by a group of NT threads: a whole block (NT =
// kCholThreads) for the large supernodes of a level, one warp (NT = 32) for
// the small ones.
template <int NT>
__device__ __forceinline__ void group_sync() {
  if constexpr (NT == 32)
    __syncwarp();
  else
    __syncthreads();
}

// The panel of supernode t after its children's contributions: column by
// column (every thread takes the same pivot and its reciprocal), P of
// leading dimension h; the trailing columns go one per warp, rows over
// the lanes.
template <int NT>
__device__ void factor_panel(double* __restrict__ P, int h, int w, int f, int tid, double tol,
                             int32_t* bad) {
  constexpr int NW = NT / 32;
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < w; ++k) {
    double p = P[size_t(k) * h + k];
    if (!(p > tol)) {
      if (tid == 0) atomicMin(bad, f + k);
      p = 1.0;
    }
    const double r = sqrt(p), rinv = 1.0 / r;
    group_sync<NT>();
    if (tid == 0) P[size_t(k) * h + k] = r;
    for (int i = k + 1 + tid; i < h; i += NT) P[size_t(k) * h + i] *= rinv;
    group_sync<NT>();
    for (int j = k + 1 + warp; j < w; j += NW) {
      const double ljk = P[size_t(k) * h + j];
      for (int i = j + lane; i < h; i += 32) P[size_t(j) * h + i] -= P[size_t(k) * h + i] * ljk;
    }
    group_sync<NT>();
  }
}

// U -= L21 L21' on the lower triangle (U of leading dimension m = h - w),
// a column per warp, rows over the lanes.
template <int NT>
__device__ void form_update(const double* __restrict__ P, int h, int w, int tid,
                            double* __restrict__ U) {
  constexpr int NW = NT / 32;
  const int lane = tid & 31, m = h - w;
  for (int j = tid >> 5; j < m; j += NW)
    for (int i = j + lane; i < m; i += 32) {
      double acc = 0.0;
      for (int k = 0; k < w; ++k) acc = fma(P[size_t(k) * h + w + i], P[size_t(k) * h + w + j], acc);
      U[size_t(j) * m + i] -= acc;
    }
}

// Extend-add of t's children's update matrices, one child at a time: the
// entries in t's columns go to the panel P (leading dimension h), the rest
// to t's update matrix U (leading dimension h - w).  The child's row map is
// staged in `srel` (a shared array of at least the child's row count) and
// each thread keeps kBatch entries of the child's update matrix in flight.
template <int NT>
__device__ void extend_add(const CholDev& d, int t, int tid, double* __restrict__ P, int h,
                           int w, double* __restrict__ U, int* __restrict__ srel) {
  constexpr int kBatch = 4;
  const int m = h - w;
  for (int q = __ldg(d.kid_ptr + t); q < __ldg(d.kid_ptr + t + 1); ++q) {
    const int c = __ldg(d.kid + q);
    const int mc = (__ldg(d.sn_rowptr + c + 1) - __ldg(d.sn_rowptr + c)) -
                   (__ldg(d.sn_first + c + 1) - __ldg(d.sn_first + c));
    const double* __restrict__ Uc = d.Ux + __ldg(d.u_off + c);
    const int32_t* __restrict__ rel = d.relmap + __ldg(d.rel_off + c);
    for (int i = tid; i < mc; i += NT) srel[i] = __ldg(rel + i);
    group_sync<NT>();
    const int total = mc * mc;
    for (int base = tid; base < total; base += kBatch * NT) {
      double v[kBatch];
      int jj[kBatch], ii[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int idx = base + u * NT;
        jj[u] = idx / mc;
        ii[u] = idx - jj[u] * mc;
        v[u] = idx < total && ii[u] >= jj[u] ? Uc[idx] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (base + u * NT >= total || ii[u] < jj[u]) continue;
        const int ri = srel[ii[u]], rj = srel[jj[u]];
        if (rj < w)
          P[size_t(rj) * h + ri] += v[u];
        else
          U[size_t(rj - w) * m + (ri - w)] += v[u];
      }
    }
    group_sync<NT>();
  }
}

__device__ void factor_small(const CholDev& d, int t, int lane, double tol,
                             double* __restrict__ ws, int* __restrict__ srel) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ Ut = d.Ux + __ldg(d.u_off + t);
  double* __restrict__ P = ws;
  double* __restrict__ U = ws + h * w;
  for (int idx = lane; idx < h * w; idx += 32) P[idx] = Lt[idx];
  for (int idx = lane; idx < m * m; idx += 32) U[idx] = 0.0;
  __syncwarp();
  extend_add<32>(d, t, lane, P, h, w, U, srel);
  factor_panel<32>(P, h, w, f, lane, tol, d.bad);
  form_update<32>(P, h, w, lane, U);
  __syncwarp();
  for (int idx = lane; idx < h * w; idx += 32) Lt[idx] = P[idx];
  for (int idx = lane; idx < m * m; idx += 32) Ut[idx] = U[idx];
}

// A large supernode by a whole block: children and panel in shared memory
// when the panel fits kPanelDoubles; when the panel and the update matrix
// fit together, the update matrix too, and U_t -= L21 L21' is formed here;
// otherwise k_chol_syrk forms it afterwards.
__device__ void factor_large(const CholDev& d, int t, double tol, double* __restrict__ sp,
                             int* __restrict__ srel) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ Ut = d.Ux + __ldg(d.u_off + t);
  const int pw = h * w;
  const bool pan = pw <= kPanelDoubles, full = pw + m * m <= kPanelDoubles;
  double* __restrict__ P = pan ? sp : Lt;
  double* __restrict__ U = full ? sp + pw : Ut;
  if (pan)
    for (int idx = threadIdx.x; idx < pw; idx += kCholThreads) sp[idx] = Lt[idx];
  if (full)
    for (int idx = threadIdx.x; idx < m * m; idx += kCholThreads) U[idx] = 0.0;
  __syncthreads();
  extend_add<kCholThreads>(d, t, threadIdx.x, P, h, w, U, srel);
  factor_panel<kCholThreads>(P, h, w, f, threadIdx.x, tol, d.bad);
  if (full) {
    form_update<kCholThreads>(P, h, w, threadIdx.x, U);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * m; idx += kCholThreads) Ut[idx] = U[idx];
  }
  if (pan)
    for (int idx = threadIdx.x; idx < pw; idx += kCholThreads) Lt[idx] = sp[idx];
}

// The children's update vectors of t: entries in t's columns go to y, the
// rest to t's update vector zt.
template <int NT>
__device__ void add_children_z(const CholDev& d, int t, int tid, int f, int w,
                               double* __restrict__ y, double* __restrict__ zt) {
  for (int q = __ldg(d.kid_ptr + t); q < __ldg(d.kid_ptr + t + 1); ++q) {
    const int c = __ldg(d.kid + q);
    const int mc = (__ldg(d.sn_rowptr + c + 1) - __ldg(d.sn_rowptr + c)) -
                   (__ldg(d.sn_first + c + 1) - __ldg(d.sn_first + c));
    const double* __restrict__ zc = d.Zx + __ldg(d.z_off + c);
    const int32_t* __restrict__ rel = d.relmap + __ldg(d.rel_off + c);
    for (int ii = tid; ii < mc; ii += NT) {
      const int r = __ldg(rel + ii);
      if (r < w)
        y[f + r] += zc[ii];
      else
        zt[r - w] += zc[ii];
    }
    group_sync<NT>();
  }
}

// Forward substitution of one supernode by one warp (small supernodes):
// the children's update vectors, the diagonal block, then its own update
// vector z_t -= L21 y_t.
__device__ void forward_small(const CholDev& d, int t, int lane, double* __restrict__ y) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ zt = d.Zx + __ldg(d.z_off + t);
  add_children_z<32>(d, t, lane, f, w, y, zt);
  for (int k = 0; k < w; ++k) {
    const double yk = y[f + k] / Lt[size_t(k) * h + k];
    __syncwarp();
    if (lane == 0) y[f + k] = yk;
    for (int i = k + 1 + lane; i < w; i += 32) y[f + i] -= Lt[size_t(k) * h + i] * yk;
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) {
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(Lt[size_t(k) * h + w + i], y[f + k], acc);
    zt[i] -= acc;
  }
}

// The same by a whole block, the diagonal block and y_t staged in shared
// memory and the triangular solve done by the first warp.
__device__ void forward_large(const CholDev& d, int t, double* __restrict__ y,
                              double* __restrict__ sL, double* __restrict__ sy) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  double* __restrict__ zt = d.Zx + __ldg(d.z_off + t);
  add_children_z<kCholThreads>(d, t, threadIdx.x, f, w, y, zt);
  for (int idx = threadIdx.x; idx < w * w; idx += kCholThreads) {
    const int k = idx / w, i = idx - k * w;
    sL[idx] = Lt[size_t(k) * h + i];
  }
  for (int k = threadIdx.x; k < w; k += kCholThreads) sy[k] = y[f + k];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int k = 0; k < w; ++k) {
      const double yk = sy[k] / sL[k * w + k];
      __syncwarp();
      if (lane == 0) sy[k] = yk;
      for (int i = k + 1 + lane; i < w; i += 32) sy[i] -= sL[k * w + i] * yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += kCholThreads) y[f + k] = sy[k];
  for (int i = threadIdx.x; i < m; i += kCholThreads) {
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(Lt[size_t(k) * h + w + i], sy[k], acc);
    zt[i] -= acc;
  }
}

// Backward substitution of one supernode: x_t -= L21' x(R_t below) (one
// warp per column, a fixed reduction tree), then the transposed diagonal
// block (by a warp; from shared memory in the block form).
__device__ void backward_small(const CholDev& d, int t, int lane, double* __restrict__ x) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int r0 = __ldg(d.sn_rowptr + t), h = __ldg(d.sn_rowptr + t + 1) - r0;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  for (int k = 0; k < w; ++k) {
    double acc = 0.0;
    for (int i = w + lane; i < h; i += 32)
      acc = fma(Lt[size_t(k) * h + i], x[__ldg(d.rowidx + r0 + i)], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[f + k] -= acc;
  }
  __syncwarp();
  for (int k = w - 1; k >= 0; --k) {
    const double xk = x[f + k] / Lt[size_t(k) * h + k];
    __syncwarp();
    if (lane == 0) x[f + k] = xk;
    for (int i = lane; i < k; i += 32) x[f + i] -= Lt[size_t(i) * h + k] * xk;
    __syncwarp();
  }
}

__device__ void backward_large(const CholDev& d, int t, double* __restrict__ x,
                               double* __restrict__ sL, double* __restrict__ sx) {
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int r0 = __ldg(d.sn_rowptr + t), h = __ldg(d.sn_rowptr + t + 1) - r0;
  const double* __restrict__ Lt = d.Lx + __ldg(d.sn_off + t);
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < w; k += kCholThreads / 32) {
    double acc = 0.0;
    for (int i = w + lane; i < h; i += 32)
      acc = fma(Lt[size_t(k) * h + i], x[__ldg(d.rowidx + r0 + i)], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sx[k] = x[f + k] - acc;
  }
  for (int idx = threadIdx.x; idx < w * w; idx += kCholThreads) {
    const int k = idx / w, i = idx - k * w;
    sL[idx] = Lt[size_t(k) * h + i];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = w - 1; k >= 0; --k) {
      const double xk = sx[k] / sL[k * w + k];
      __syncwarp();
      if (lane == 0) sx[k] = xk;
      for (int i = lane; i < k; i += 32) sx[i] -= sL[i * w + k] * xk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += kCholThreads) x[f + k] = sx[k];
}

// One level: blocks [0, n_large) take the level's first n_large supernodes
// one per block; the remaining blocks take the rest one per warp.
constexpr int kWarpsPerBlock = kCholThreads / 32;

__device__ __forceinline__ int level_item(int n_large, int count, int& tid, bool& whole) {
  if (int(blockIdx.x) < n_large) {
    whole = true;
    tid = threadIdx.x;
    return blockIdx.x;
  }
  whole = false;
  tid = threadIdx.x & 31;
  const int q = n_large + (int(blockIdx.x) - n_large) * kWarpsPerBlock + int(threadIdx.x >> 5);
  return q < count ? q : -1;
}

// `stage`: doubles of shared memory per warp (small supernodes) or per
// block (large ones) behind the row-map scratch.
__global__ void __launch_bounds__(kCholThreads) k_chol_factor(CholDev d, int begin, int count,
                                                               int n_large, double tol,
                                                               int stage) {
  extern __shared__ double sp[];
  __shared__ int srel_all[kRelScratch];
  int tid;
  bool whole;
  const int q = level_item(n_large, count, tid, whole);
  if (q < 0) return;
  const int t = __ldg(d.level_sn + begin + q);
  if (whole) {
    factor_large(d, t, tol, sp, srel_all);
  } else {
    const int warp = threadIdx.x >> 5;
    factor_small(d, t, tid, tol, sp + warp * stage, srel_all + warp * kCholWarpRows);
  }
}

// U_t -= L21 L21' for the large supernodes of a level, one 32 x 32 tile of
// U_t per block: tiles[i] = {t, tile row, tile column, 0}, lower tiles only.
constexpr int kTile = 32;
__global__ void __launch_bounds__(kCholThreads) k_chol_syrk(CholDev d, const int4* __restrict__ tiles,
                                                             int begin) {
  __shared__ double A[kTile][kMaxWidth + 1], B[kTile][kMaxWidth + 1];
  const int4 tl = __ldg(tiles + begin + blockIdx.x);
  const int t = tl.x;
  const int f = __ldg(d.sn_first + t), w = __ldg(d.sn_first + t + 1) - f;
  const int h = __ldg(d.sn_rowptr + t + 1) - __ldg(d.sn_rowptr + t), m = h - w;
  const double* __restrict__ L21 = d.Lx + __ldg(d.sn_off + t) + w;  // column k at L21[k h]
  double* __restrict__ Ut = d.Ux + __ldg(d.u_off + t);
  const int i0 = tl.y * kTile, j0 = tl.z * kTile;
  for (int idx = threadIdx.x; idx < kTile * w; idx += kCholThreads) {
    const int r = idx % kTile, k = idx / kTile;
    A[r][k] = i0 + r < m ? L21[size_t(k) * h + i0 + r] : 0.0;
    B[r][k] = j0 + r < m ? L21[size_t(k) * h + j0 + r] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x % kTile, r0 = threadIdx.x / kTile;
  const int j = j0 + c;
  for (int r = r0; r < kTile; r += kCholThreads / kTile) {
    const int i = i0 + r;
    if (i >= m || j >= m || i < j) continue;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(A[r][k], B[c][k], acc);
    Ut[size_t(j) * m + i] -= acc;
  }
}

__global__ void __launch_bounds__(kCholThreads) k_chol_fwd(CholDev d, int begin, int count,
                                                            int n_large, double* __restrict__ y) {
  __shared__ double sL[kMaxWidth * kMaxWidth], sy[kMaxWidth];
  int tid;
  bool whole;
  const int q = level_item(n_large, count, tid, whole);
  if (q < 0) return;
  const int t = __ldg(d.level_sn + begin + q);
  if (whole)
    forward_large(d, t, y, sL, sy);
  else
    forward_small(d, t, tid, y);
}

__global__ void __launch_bounds__(kCholThreads) k_chol_bwd(CholDev d, int begin, int count,
                                                            int n_large, double* __restrict__ x) {
  __shared__ double sL[kMaxWidth * kMaxWidth], sx[kMaxWidth];
  int tid;
  bool whole;
  const int q = level_item(n_large, count, tid, whole);
  if (q < 0) return;
  const int t = __ldg(d.level_sn + begin + q);
  if (whole)
    backward_large(d, t, x, sL, sx);
  else
    backward_small(d, t, tid, x);
}

int level_blocks(int count, int n_large) {
  return n_large + (count - n_large + kWarpsPerBlock - 1) / kWarpsPerBlock;
}

int grid_for(int64_t n, int threads) {
  return n > 0 ? int(std::min<int64_t>((n + threads - 1) / threads, 4096)) : 0;
}

}  // namespace

cudaError_t launch_gather(double* out, const double* in, const int32_t* idx, int n,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<grid_for(n, kPermThreads), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_scatter(double* out, const double* in, const int32_t* idx, int n,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter<<<grid_for(n, kPermThreads), kPermThreads, 0, s>>>(out, in, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_chol_assemble(double* Lx, const int64_t* amap, const double* kvals,
                                 int64_t nnz, cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  k_chol_assemble<<<grid_for(nnz, kPermThreads), kPermThreads, 0, s>>>(Lx, amap, kvals, nnz);
  return cudaGetLastError();
}

size_t chol_factor_smem_bytes(int count, int n_large, int stage) {
  return size_t(n_large > 0 || count == 0 ? stage : kWarpsPerBlock * stage) * sizeof(double);
}

cudaError_t chol_allow_smem(size_t bytes) {
  if (bytes + kRelScratch * sizeof(int) <= 48 * 1024) return cudaSuccess;  // the default
  return cudaFuncSetAttribute(k_chol_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(bytes));
}

cudaError_t launch_chol_factor_level(const CholDev& d, int begin, int count, int n_large,
                                     double tol, int stage, const int4* tiles, int tile_begin,
                                     int n_tiles, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (count > 0) {
    const size_t smem = chol_factor_smem_bytes(count, n_large, stage);
    k_chol_factor<<<level_blocks(count, n_large), kCholThreads, smem, s>>>(d, begin, count,
                                                                            n_large, tol, stage);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n_tiles > 0) {
    k_chol_syrk<<<n_tiles, kCholThreads, 0, s>>>(d, tiles, tile_begin);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_chol_fwd_level(const CholDev& d, int begin, int count, int n_large, double* y,
                                  cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chol_fwd<<<level_blocks(count, n_large), kCholThreads, 0, s>>>(d, begin, count, n_large, y);
  return cudaGetLastError();
}

cudaError_t launch_chol_bwd_level(const CholDev& d, int begin, int count, int n_large, double* x,
                                  cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_chol_bwd<<<level_blocks(count, n_large), kCholThreads, 0, s>>>(d, begin, count, n_large, x);
  return cudaGetLastError();
}

}  // namespace acopf
