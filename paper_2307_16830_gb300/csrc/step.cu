// Condensation around M_cond and step recovery (Sec. IV.C), sm_103a, FP64.
//
// Elementwise work per variable and per constraint row, plus the two
// sparse products with the Jacobian the path needs: A' w for the condensed
// right-hand side (gathered per variable over its Jacobian entries) and A dx
// for the slack step (gathered per row).  Every sum runs in a fixed order
// (ascending Jacobian slot), so results do not depend on scheduling.  A
// bound at +-inf contributes nothing: its inverse gap is taken as zero.
#include <cuda_runtime.h>

#include "acopf_internal.h"
#include "fp64_device.cuh"

namespace acopf {
namespace {

constexpr int kStepThreads = 256;
constexpr int kResMax = 4;  // maxima per residual block (kResPart values in all)

__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }

// Tests on the bit pattern (integer pipe; the FP64 pipe is the scarce one):
// a finite value, and |v| in [2^-500, 2^500).
__device__ __forceinline__ bool is_finite_bits(double v) {
  return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool mid_range(double v) {
  const unsigned e = static_cast<unsigned>(__double_as_longlong(v) >> 52) & 0x7ffu;
  return e - 523u < 1000u;
}

// (v - lo)^-1 and (hi - v)^-1, zero at an infinite bound.  With both bounds
// finite one reciprocal serves both: with a = v - lo, b = hi - v,
// 1/a = b (ab)^-1 and 1/b = a (ab)^-1 (a few ulps), when a and b are in a
// range where ab cannot overflow or underflow.
__device__ __forceinline__ void inv_gaps(double v, double lo, double hi, double& il,
                                         double& iu) {
  const bool fl = is_finite_bits(lo), fh = is_finite_bits(hi);
  const double a = v - lo, b = hi - v;
  if (fl && fh && mid_range(a) && mid_range(b)) {
    const double r = recip_nr(a * b);
    il = b * r;
    iu = a * r;
    return;
  }
  il = fl ? recip(a) : 0.0;
  iu = fh ? recip(b) : 0.0;
}

// Rows: Sigma_s, q_s and w = C q_s + D q_y, with C = (dc Sigma_s + 1 + dc dw)^-1
// and D = (Sigma_s + dw) C (C = 1, D = Sigma_s without regularisation).
template <bool REG>
__global__ void __launch_bounds__(kStepThreads) k_condense_rows(DevStep st, StepIterate it,
                                                                double dw, double dc,
                                                                double* __restrict__ sigma_s,
                                                                double* __restrict__ q_s) {
  const int r = blockIdx.x * kStepThreads + threadIdx.x;
  if (r < st.m) {
    double il, iu;
    inv_gaps(ldg(it.s + r), ldg(it.sl + r), ldg(it.su + r), il, iu);
    const double sig = fma(ldg(it.zl_s + r), il, ldg(it.zu_s + r) * iu);
    const double q = fma(il, ldg(it.p_zl_s + r), fma(-iu, ldg(it.p_zu_s + r), ldg(it.p_s + r)));
    const double py = ldg(it.p_y + r);
    double w;
    if constexpr (REG) {
      const double C = recip(fma(dc, sig, fma(dc, dw, 1.0)));
      w = C * fma(sig + dw, py, q);  // C q_s + D q_y with D = (Sigma_s + dw) C
    } else {
      w = fma(sig, py, q);
    }
    sigma_s[r] = sig;
    q_s[r] = q;
    st.w[r] = w;
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Columns: Sigma_x, q_x and rhs = q_x + A' w (w from the row kernel).
__global__ void __launch_bounds__(kStepThreads) k_condense_cols(DevStep st, StepIterate it,
                                                               const double* __restrict__ J,
                                                               double* __restrict__ sigma_x,
                                                               double* __restrict__ rhs) {
  const int j = blockIdx.x * kStepThreads + threadIdx.x;
  double q = 0.0;
  int k0 = 0, k1 = 0;
  if (j < st.n) {  // independent of the row kernel: before the grid dependency
    double il, iu;
    inv_gaps(ldg(it.x + j), ldg(it.xl + j), ldg(it.xu + j), il, iu);
    sigma_x[j] = fma(ldg(it.zl_x + j), il, ldg(it.zu_x + j) * iu);
    q = fma(il, ldg(it.p_zl_x + j), fma(-iu, ldg(it.p_zu_x + j), ldg(it.p_x + j)));
    k0 = __ldg(st.jt_ptr + j);
    k1 = __ldg(st.jt_ptr + j + 1);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (j >= st.n) return;
  double acc = 0.0;
  for (int k = k0; k < k1; ++k)
    acc = fma(ldg(J + __ldg(st.jt_slot + k)), __ldcg(st.w + __ldg(st.jt_row + k)), acc);
  rhs[j] = q + acc;
}

// Recovery.  Blocks [0, nrb) take rows: A dx, ds = C (A dx + dc q_s - q_y),
// dy = (Sigma_s + dw) ds - q_s, dzl_s, dzu_s; the rest take columns: dzl_x, dzu_x.
template <bool REG>
__global__ void __launch_bounds__(kStepThreads) k_recover(
    DevStep st, StepIterate it, const double* __restrict__ J, double dw, double dc,
    const double* __restrict__ sigma_s, const double* __restrict__ q_s,
    const double* __restrict__ dx, double* __restrict__ ds_out, double* __restrict__ dy_out,
    double* __restrict__ dzl_x, double* __restrict__ dzu_x, double* __restrict__ dzl_s,
    double* __restrict__ dzu_s, int nrb) {
  if (static_cast<int>(blockIdx.x) < nrb) {
    const int r = blockIdx.x * kStepThreads + threadIdx.x;
    if (r >= st.m) return;
    const int k0 = __ldg(st.jr_ptr + r), k1 = __ldg(st.jr_ptr + r + 1);
    double adx = 0.0;
    for (int k = k0; k < k1; ++k)
      adx = fma(ldg(J + __ldg(st.jr_slot + k)), ldg(dx + __ldg(st.jr_col + k)), adx);
    const double sig = ldg(sigma_s + r), q = ldg(q_s + r), py = ldg(it.p_y + r);
    double ds;
    if constexpr (REG) {
      const double C = recip(fma(dc, sig, fma(dc, dw, 1.0)));
      ds = C * (fma(dc, q, adx) - py);
    } else {
      ds = adx - py;
    }
    ds_out[r] = ds;
    dy_out[r] = fma(sig + dw, ds, -q);
    double il, iu;
    inv_gaps(ldg(it.s + r), ldg(it.sl + r), ldg(it.su + r), il, iu);
    dzl_s[r] = il * fma(-ldg(it.zl_s + r), ds, ldg(it.p_zl_s + r));
    dzu_s[r] = iu * fma(ldg(it.zu_s + r), ds, ldg(it.p_zu_s + r));
  } else {
    const int j = (blockIdx.x - nrb) * kStepThreads + threadIdx.x;
    if (j >= st.n) return;
    const double d = ldg(dx + j);
    double il, iu;
    inv_gaps(ldg(it.x + j), ldg(it.xl + j), ldg(it.xu + j), il, iu);
    dzl_x[j] = il * fma(-ldg(it.zl_x + j), d, ldg(it.p_zl_x + j));
    dzu_x[j] = iu * fma(ldg(it.zu_x + j), d, ldg(it.p_zu_x + j));
  }
}

int blocks_for(int count) { return (count + kStepThreads - 1) / kStepThreads; }

// Scaled residual of the first-order conditions.  A grid of a fixed number
// of blocks per device strides over the variables (dual residual grad f -
// A'y - zl_x + zu_x, complementarity of the variable bounds), then over the
// rows (y - zl_s + zu_s, g - s, complementarity of the slack bounds, |y|).
// Each block leaves max |r_d|, max |r_p|, max |r_c|, max |r_c| at a second
// mu, sum |y|, sum |z| and the count of finite bounds (sums in a fixed order
// for the fixed grid; maxima are order-free) for k_residual_final, which
// writes out = [E, max|r_d|, max|r_p|, max|r_c|, ||y||_1, ||z||_1, n_z, s_d,
// s_c] and, for the two-mu form, out[9] = E at the second mu.
// Maxima of absolute values are taken on the bit patterns (a non-negative
// double orders like its bits as an unsigned integer; NaN bits exceed every
// number's, so a NaN propagates) and counts are integers: both off the FP64
// pipe, which the sums and products keep busy.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffULL;
}

// DUAL: also max |r_c| at a second barrier parameter mu2 (the iteration's
// test at mu = 0 and its barrier test at mu from one pass).
template <bool DUAL>
__global__ void __launch_bounds__(kStepThreads) k_kkt_residual(
    DevStep st, StepIterate it, const double* __restrict__ y, const double* __restrict__ grad,
    const double* __restrict__ cons, const double* __restrict__ J, double mu, double mu2) {
  // max |r_d|, |r_p|, |r_c|, |r_c at mu2| (bits)
  unsigned long long mx[kResMax] = {0ull, 0ull, 0ull, 0ull};
  double ysum = 0.0, zsum = 0.0;
  long long nz = 0;
  const int stride = gridDim.x * kStepThreads;
  for (int j = blockIdx.x * kStepThreads + threadIdx.x; j < st.n; j += stride) {
    // A'y over the variable's Jacobian entries in slot order, four in flight
    double aty = 0.0;
    int k = __ldg(st.jt_ptr + j);
    const int k1 = __ldg(st.jt_ptr + j + 1);
    for (; k + 4 <= k1; k += 4) {
      int sl[4], rw[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sl[u] = __ldg(st.jt_slot + k + u);
        rw[u] = __ldg(st.jt_row + k + u);
      }
      double jv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        jv[u] = ldg(J + sl[u]);
        yv[u] = ldg(y + rw[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) aty = fma(jv[u], yv[u], aty);
    }
    for (; k < k1; ++k) aty = fma(ldg(J + __ldg(st.jt_slot + k)), ldg(y + __ldg(st.jt_row + k)), aty);
    const double zl = ldg(it.zl_x + j), zu = ldg(it.zu_x + j), x = ldg(it.x + j);
    mx[0] = max(mx[0], abs_bits(ldg(grad + j) - aty - zl + zu));
    const double lo = ldg(it.xl + j), hi = ldg(it.xu + j);
    if (is_finite_bits(lo)) {
      mx[2] = max(mx[2], abs_bits(fma(zl, x - lo, -mu)));
      if constexpr (DUAL) mx[3] = max(mx[3], abs_bits(fma(zl, x - lo, -mu2)));
      zsum += fabs(zl);
      ++nz;
    }
    if (is_finite_bits(hi)) {
      mx[2] = max(mx[2], abs_bits(fma(zu, hi - x, -mu)));
      if constexpr (DUAL) mx[3] = max(mx[3], abs_bits(fma(zu, hi - x, -mu2)));
      zsum += fabs(zu);
      ++nz;
    }
  }
  for (int r = blockIdx.x * kStepThreads + threadIdx.x; r < st.m; r += stride) {
    const double yr = ldg(y + r), zl = ldg(it.zl_s + r), zu = ldg(it.zu_s + r);
    const double sr = ldg(it.s + r);
    mx[0] = max(mx[0], abs_bits(yr - zl + zu));
    mx[1] = max(mx[1], abs_bits(ldg(cons + r) - sr));
    ysum += fabs(yr);
    const double lo = ldg(it.sl + r), hi = ldg(it.su + r);
    if (is_finite_bits(lo)) {
      mx[2] = max(mx[2], abs_bits(fma(zl, sr - lo, -mu)));
      if constexpr (DUAL) mx[3] = max(mx[3], abs_bits(fma(zl, sr - lo, -mu2)));
      zsum += fabs(zl);
      ++nz;
    }
    if (is_finite_bits(hi)) {
      mx[2] = max(mx[2], abs_bits(fma(zu, hi - sr, -mu)));
      if constexpr (DUAL) mx[3] = max(mx[3], abs_bits(fma(zu, hi - sr, -mu2)));
      zsum += fabs(zu);
      ++nz;
    }
  }
  // Block reduction: shuffle trees (fixed order), then the warps in order.
  __shared__ unsigned long long shm[kStepThreads / 32][kResMax];
  __shared__ double shs[kStepThreads / 32][2];
  __shared__ long long shn[kStepThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < kResMax; ++q) mx[q] = max(mx[q], __shfl_down_sync(0xffffffffu, mx[q], o));
    ysum += __shfl_down_sync(0xffffffffu, ysum, o);
    zsum += __shfl_down_sync(0xffffffffu, zsum, o);
    nz += __shfl_down_sync(0xffffffffu, nz, o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kResMax; ++q) shm[warp][q] = mx[q];
    shs[warp][0] = ysum;
    shs[warp][1] = zsum;
    shn[warp] = nz;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long bm[kResMax] = {0ull, 0ull, 0ull, 0ull};
    double bs[2] = {0.0, 0.0};
    long long bn = 0;
    for (int w = 0; w < kStepThreads / 32; ++w) {
      for (int q = 0; q < kResMax; ++q) bm[q] = max(bm[q], shm[w][q]);
      bs[0] += shs[w][0];
      bs[1] += shs[w][1];
      bn += shn[w];
    }
    double* out = st.res_part + kResPart * blockIdx.x;
    for (int q = 0; q < kResMax; ++q) out[q] = __longlong_as_double(static_cast<long long>(bm[q]));
    out[4] = bs[0];
    out[5] = bs[1];
    out[6] = static_cast<double>(bn);  // exact below 2^53
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The larger of two non-negative doubles (or NaN), compared as bits.
__device__ __forceinline__ double max_bits(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// One block: the blocks' parts in a fixed order (each thread a strided
// subset in ascending order, then fixed trees), and the scaled residual.
__global__ void __launch_bounds__(kStepThreads) k_residual_final(DevStep st, int nb, int dual,
                                                                 double* __restrict__ out) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  double c[kResPart] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // kResMax maxima, then 3 sums
  constexpr int U = 4;  // blocks fetched per round, all loads in flight together
  for (int b0 = threadIdx.x; b0 < nb; b0 += U * kStepThreads) {
    double t[U][kResPart];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int b = b0 + u * kStepThreads;
#pragma unroll
      for (int q = 0; q < kResPart; ++q) t[u][q] = b < nb ? __ldcg(st.res_part + kResPart * b + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int q = 0; q < kResMax; ++q) c[q] = max_bits(c[q], t[u][q]);
#pragma unroll
      for (int q = kResMax; q < kResPart; ++q) c[q] += t[u][q];
    }
  }
  __shared__ double sh[kStepThreads / 32][kResPart];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < kResMax; ++q) c[q] = max_bits(c[q], __shfl_down_sync(0xffffffffu, c[q], o));
#pragma unroll
    for (int q = kResMax; q < kResPart; ++q) c[q] += __shfl_down_sync(0xffffffffu, c[q], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < kResPart; ++q) sh[warp][q] = c[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < kResPart; ++q) c[q] = sh[0][q];
    for (int w = 1; w < kStepThreads / 32; ++w) {
      for (int q = 0; q < kResMax; ++q) c[q] = max_bits(c[q], sh[w][q]);
      for (int q = kResMax; q < kResPart; ++q) c[q] += sh[w][q];
    }
    const double smax = 100.0;  // s_max of the scaling
    const double nz = c[6];
    const double s_d = fmax(smax, (c[4] + c[5]) / (static_cast<double>(st.m) + nz)) / smax;
    const double s_c = nz > 0.0 ? fmax(smax, c[5] / nz) / smax : 1.0;
    out[0] = fmax(fmax(c[0] / s_d, c[1]), c[2] / s_c);
    out[1] = c[0];
    out[2] = c[1];
    out[3] = c[2];
    out[4] = c[4];
    out[5] = c[5];
    out[6] = nz;
    out[7] = s_d;
    out[8] = s_c;
    if (dual) out[9] = fmax(fmax(c[0] / s_d, c[1]), c[3] / s_c);  // E at the second mu
  }
}

}  // namespace

cudaError_t launch_condense(const DevStep& st, const StepIterate& it, const double* jvals,
                            double delta_w, double delta_c, double* sigma_x, double* sigma_s,
                            double* q_s, double* rhs, bool pdl, cudaStream_t s) {
  const bool reg = delta_w != 0.0 || delta_c != 0.0;
  const int rb = blocks_for(st.m), cb = blocks_for(st.n);
  if (rb > 0) {
    if (reg)
      k_condense_rows<true><<<rb, kStepThreads, 0, s>>>(st, it, delta_w, delta_c, sigma_s, q_s);
    else
      k_condense_rows<false><<<rb, kStepThreads, 0, s>>>(st, it, delta_w, delta_c, sigma_s, q_s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (cb == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cb);
  cfg.blockDim = dim3(kStepThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl && rb > 0) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_condense_cols, st, it, jvals, sigma_x, rhs);
}

int residual_blocks(int sms) { return 4 * sms; }

cudaError_t launch_kkt_residual(const DevStep& st, const StepIterate& it, const double* y,
                                const double* grad, const double* cons, const double* jvals,
                                double mu, double* out, cudaStream_t s) {
  return launch_kkt_residual2(st, it, y, grad, cons, jvals, mu, -1.0, out, s);
}

cudaError_t launch_kkt_residual2(const DevStep& st, const StepIterate& it, const double* y,
                                 const double* grad, const double* cons, const double* jvals,
                                 double mu, double mu2, double* out, cudaStream_t s) {
  const int dual = mu2 >= 0.0;
  if (dual)
    k_kkt_residual<true><<<st.res_blocks, kStepThreads, 0, s>>>(st, it, y, grad, cons, jvals, mu,
                                                                 mu2);
  else
    k_kkt_residual<false><<<st.res_blocks, kStepThreads, 0, s>>>(st, it, y, grad, cons, jvals,
                                                                  mu, 0.0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(kStepThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_residual_final, st, st.res_blocks, dual, out);
}

cudaError_t launch_recover(const DevStep& st, const StepIterate& it, const double* jvals,
                           double delta_w, double delta_c, const double* sigma_s,
                           const double* q_s, const double* dx, double* ds, double* dy,
                           double* dzl_x, double* dzu_x, double* dzl_s, double* dzu_s,
                           cudaStream_t s) {
  const int rb = blocks_for(st.m), cb = blocks_for(st.n);
  if (rb + cb == 0) return cudaSuccess;
  if (delta_w != 0.0 || delta_c != 0.0)
    k_recover<true><<<rb + cb, kStepThreads, 0, s>>>(st, it, jvals, delta_w, delta_c, sigma_s,
                                                     q_s, dx, ds, dy, dzl_x, dzu_x, dzl_s,
                                                     dzu_s, rb);
  else
    k_recover<false><<<rb + cb, kStepThreads, 0, s>>>(st, it, jvals, delta_w, delta_c, sigma_s,
                                                      q_s, dx, ds, dy, dzl_x, dzu_x, dzl_s,
                                                      dzu_s, rb);
  return cudaGetLastError();
}

}  // namespace acopf
