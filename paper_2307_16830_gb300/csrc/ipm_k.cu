// Vector kernels of the condensed-space interior-point iteration (Algorithm
// 1): the Newton right-hand side (minus the conditions of Eq. first), the
// step-size bounds and the barrier terms of the line search, the trial
// point, the update of the multipliers, and the feasibility restoration's
// slack projection, Gauss-Newton right-hand side, step bound and trials.  Reductions run over a fixed
// grid (4 blocks per SM): per-block partials in a fixed order, then one
// block combining them in block order, so every result is reproducible.
#include "fp64_device.cuh"
#include "ipm_internal.h"

namespace acopf {
namespace {

constexpr int kIpmThreads = 256;

__device__ __forceinline__ bool finite_bound(double v) { return isfinite(v); }

// Block reduction of NV values, the first NMIN by min, the rest by sum, in a
// fixed order; thread 0 writes them to out[NV * blockIdx.x ..].
template <int NV, int NMIN>
__device__ void block_reduce(double (&v)[NV], double* __restrict__ out) {
  __shared__ double sh[kIpmThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double u = __shfl_down_sync(0xffffffffu, v[q], o);
      v[q] = q < NMIN ? fmin(v[q], u) : v[q] + u;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[warp][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) b[q] = sh[0][q];
    for (int w = 1; w < kIpmThreads / 32; ++w)
#pragma unroll
      for (int q = 0; q < NV; ++q) b[q] = q < NMIN ? fmin(b[q], sh[w][q]) : b[q] + sh[w][q];
#pragma unroll
    for (int q = 0; q < NV; ++q) out[NV * blockIdx.x + q] = b[q];
  }
}

// One block: combines nb partial records of NV values in block order.
template <int NV, int NMIN>
__global__ void __launch_bounds__(kIpmThreads) k_ipm_final(const double* __restrict__ part,
                                                            int nb, double* __restrict__ out) {
  double v[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = q < NMIN ? INFINITY : 0.0;
  for (int b = threadIdx.x; b < nb; b += kIpmThreads)
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double u = part[NV * b + q];
      v[q] = q < NMIN ? fmin(v[q], u) : v[q] + u;
    }
  __shared__ double tmp[NV];
  // reuse block_reduce's tree with a single block's record
  block_reduce<NV, NMIN>(v, tmp);
  __syncthreads();
  if (threadIdx.x < NV) out[threadIdx.x] = tmp[threadIdx.x];
}

// Newton right-hand side: minus the conditions of Eq. first at the iterate.
__global__ void __launch_bounds__(kIpmThreads) k_ipm_rhs(DevStep st, IpmVec v, double mu) {
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < st.n; j += stride) {
    double aty = 0.0;
    for (int k = __ldg(st.jt_ptr + j), k1 = __ldg(st.jt_ptr + j + 1); k < k1; ++k)
      aty = fma(v.jvals[__ldg(st.jt_slot + k)], v.y[__ldg(st.jt_row + k)], aty);
    const double x = v.x[j], zl = v.zl_x[j], zu = v.zu_x[j], lo = v.xl[j], hi = v.xu[j];
    v.p_x[j] = -(v.grad[j] - aty - zl + zu);
    v.p_zl_x[j] = finite_bound(lo) ? mu - zl * (x - lo) : 0.0;
    v.p_zu_x[j] = finite_bound(hi) ? mu - zu * (hi - x) : 0.0;
  }
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < st.m; r += stride) {
    const double s = v.s[r], zl = v.zl_s[r], zu = v.zu_s[r], lo = v.sl[r], hi = v.su[r];
    v.p_s[r] = -(v.y[r] - zl + zu);
    v.p_y[r] = -(v.cons[r] - s);
    v.p_zl_s[r] = finite_bound(lo) ? mu - zl * (s - lo) : 0.0;
    v.p_zu_s[r] = finite_bound(hi) ? mu - zu * (hi - s) : 0.0;
  }
}

// Step bounds and barrier terms at the iterate, per block:
// [primal fraction-to-boundary alpha, dual alpha, grad phi' d, sum log gaps].
// The FP64 unit bounds these passes, so each gap's reciprocal is the
// three-operation one (within an ulp), the step bounds compare ratios
// tau gap / |dv| through reciprocals of the step components, and the
// logarithms are summed as one logarithm of their product per thread.
__device__ __forceinline__ void primal_terms(double v, double dv, double lo, double hi, double tau,
                                             double mu, double (&a)[4], LogSum& lg) {
  if (finite_bound(lo)) {
    const double gap = v - lo;
    if (dv < 0.0) a[0] = fmin(a[0], -tau * gap * recip(dv));
    a[2] = fma(-mu * dv, recip(gap), a[2]);
    lg.add(gap);
  }
  if (finite_bound(hi)) {
    const double gap = hi - v;
    if (dv > 0.0) a[0] = fmin(a[0], tau * gap * recip(dv));
    a[2] = fma(mu * dv, recip(gap), a[2]);
    lg.add(gap);
  }
}

__device__ __forceinline__ void dual_term(double z, double dz, double tau, double (&a)[4]) {
  if (dz < 0.0) a[1] = fmin(a[1], -tau * z * recip(dz));
}

__global__ void __launch_bounds__(kIpmThreads) k_ipm_dir(IpmVec v, int n, int m, double tau,
                                                          double mu, double* __restrict__ part) {
  double a[4] = {1.0, 1.0, 0.0, 0.0};
  LogSum lg;
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double dx = v.dx[j];
    a[2] = fma(v.grad[j], dx, a[2]);
    primal_terms(v.x[j], dx, v.xl[j], v.xu[j], tau, mu, a, lg);
    dual_term(v.zl_x[j], v.dzl_x[j], tau, a);
    dual_term(v.zu_x[j], v.dzu_x[j], tau, a);
  }
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride) {
    primal_terms(v.s[r], v.ds[r], v.sl[r], v.su[r], tau, mu, a, lg);
    dual_term(v.zl_s[r], v.dzl_s[r], tau, a);
    dual_term(v.zu_s[r], v.dzu_s[r], tau, a);
  }
  a[3] = lg.value();
  block_reduce<4, 2>(a, part);
}

// Trial point x_t = x + alpha dx, s_t = s + alpha ds.
__global__ void __launch_bounds__(kIpmThreads) k_ipm_trial(IpmVec v, int n, int m, double alpha) {
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride)
    v.xt[j] = fma(alpha, v.dx[j], v.x[j]);
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride)
    v.st[r] = fma(alpha, v.ds[r], v.s[r]);
}

// Second-order correction's constraint residual: c = a (cons - s) + (ct - st)
// for the first correction (cons, s: the current iterate), c = a c + (ct -
// st) for the next ones; py = -c, the corrected Newton right-hand side's
// constraint part.
__global__ void __launch_bounds__(kIpmThreads) k_soc_rhs(double* __restrict__ c,
                                                          double* __restrict__ py,
                                                          const double* __restrict__ cons,
                                                          const double* __restrict__ sv,
                                                          const double* __restrict__ ct,
                                                          const double* __restrict__ st,
                                                          double a, int m) {
  const int stride = gridDim.x * kIpmThreads;
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride) {
    const double prev = cons ? cons[r] - sv[r] : c[r];
    const double cr = fma(a, prev, ct[r] - st[r]);
    c[r] = cr;
    py[r] = -cr;
  }
}

// At a point (x, s) with its constraint values: [sum |g - s|, sum log gaps].
__global__ void __launch_bounds__(kIpmThreads) k_ipm_measure(IpmVec v, const double* __restrict__ x,
                                                              const double* __restrict__ s,
                                                              const double* __restrict__ cons,
                                                              int n, int m,
                                                              double* __restrict__ part) {
  double a[2] = {0.0, 0.0};
  LogSum lg;
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double lo = v.xl[j], hi = v.xu[j], xj = x[j];
    if (finite_bound(lo)) lg.add(xj - lo);
    if (finite_bound(hi)) lg.add(hi - xj);
  }
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride) {
    const double lo = v.sl[r], hi = v.su[r], sr = s[r];
    a[0] += fabs(cons[r] - sr);
    if (finite_bound(lo)) lg.add(sr - lo);
    if (finite_bound(hi)) lg.add(hi - sr);
  }
  a[1] = lg.value();
  block_reduce<2, 0>(a, part);
}

// Accepted step: y <- y - alpha dy (the printed system's Delta y is minus
// the Newton step of y), z <- z + alpha_z dz, then the safeguard
// z in [mu/(kappa gap), kappa mu/gap] at the new point (already in x, s).
// (hi_c = kappa mu, lo_c = mu / kappa: one reciprocal of the gap for both limits,
// within an ulp)
__device__ __forceinline__ double reset_z(double z, double gap, double hi_c, double lo_c) {
  const double ig = recip(gap);
  return fmax(fmin(z, hi_c * ig), lo_c * ig);
}

__global__ void __launch_bounds__(kIpmThreads) k_ipm_accept(IpmVec v, int n, int m, double alpha,
                                                             double alpha_z, double mu,
                                                             double kappa) {
  const double hi_c = kappa * mu, lo_c = mu / kappa;
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double x = v.x[j], lo = v.xl[j], hi = v.xu[j];
    if (finite_bound(lo)) v.zl_x[j] = reset_z(fma(alpha_z, v.dzl_x[j], v.zl_x[j]), x - lo, hi_c, lo_c);
    if (finite_bound(hi)) v.zu_x[j] = reset_z(fma(alpha_z, v.dzu_x[j], v.zu_x[j]), hi - x, hi_c, lo_c);
  }
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride) {
    const double s = v.s[r], lo = v.sl[r], hi = v.su[r];
    const double yr = fma(-alpha, v.dy[r], v.y[r]);
    v.y[r] = yr;
    v.ym[r] = -yr;
    if (finite_bound(lo)) v.zl_s[r] = reset_z(fma(alpha_z, v.dzl_s[r], v.zl_s[r]), s - lo, hi_c, lo_c);
    if (finite_bound(hi)) v.zu_s[r] = reset_z(fma(alpha_z, v.dzu_s[r], v.zu_s[r]), hi - s, hi_c, lo_c);
  }
}

// ---------------------------------------------------------------------------
// feasibility restoration (the oracle's `restoration`, reading d10)
// ---------------------------------------------------------------------------
// At x with its constraint values g: the slacks follow g clipped onto the
// pushed slack box [lo_s, hi_s] (s = clip(g)), the violation is
// r = g - s, w = 1 where r != 0 (the assembly's D), and per block
// [sum |r|, sum r^2].
__global__ void __launch_bounds__(kIpmThreads) k_resto_slack(
    const double* __restrict__ cons, const double* __restrict__ lo_s,
    const double* __restrict__ hi_s, int m, double* __restrict__ s, double* __restrict__ r,
    double* __restrict__ w, double* __restrict__ part) {
  double a[2] = {0.0, 0.0};
  const int stride = gridDim.x * kIpmThreads;
  for (int k = blockIdx.x * kIpmThreads + threadIdx.x; k < m; k += stride) {
    const double g = cons[k];
    const double sk = fmin(fmax(g, lo_s[k]), hi_s[k]);
    const double rk = g - sk;
    s[k] = sk;
    if (r) r[k] = rk;
    if (w) w[k] = rk != 0.0 ? 1.0 : 0.0;
    a[0] += fabs(rk);
    a[1] = fma(rk, rk, a[1]);
  }
  block_reduce<2, 0>(a, part);
}

// The gradient of the restoration merit psi at x, minus (the solve's
// right-hand side), and the diagonal sigma = mu_R (1/(x-l)^2 + 1/(u-x)^2)
// + zeta: -(A'(w r) + mu_R (1/(u-x) - 1/(x-l)) + zeta (x - x_R)).  A'(w r)
// is gathered per variable in slot order (w r = r: r is 0 where w is).
__global__ void __launch_bounds__(kIpmThreads) k_resto_grad(
    DevStep st, const double* __restrict__ jvals, const double* __restrict__ r,
    const double* __restrict__ x, const double* __restrict__ xr, const double* __restrict__ xl,
    const double* __restrict__ xu, double mu_r, double zeta, double* __restrict__ rhs,
    double* __restrict__ sigma) {
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < st.n; j += stride) {
    double atr = 0.0;
    for (int k = __ldg(st.jt_ptr + j), k1 = __ldg(st.jt_ptr + j + 1); k < k1; ++k)
      atr = fma(jvals[__ldg(st.jt_slot + k)], r[__ldg(st.jt_row + k)], atr);
    const double xj = x[j], lo = xl[j], hi = xu[j];
    double g = fma(zeta, xj - xr[j], atr), sg = zeta;
    if (finite_bound(lo)) {
      const double il = 1.0 / (xj - lo);
      g -= mu_r * il;
      sg = fma(mu_r * il, il, sg);
    }
    if (finite_bound(hi)) {
      const double iu = 1.0 / (hi - xj);
      g += mu_r * iu;
      sg = fma(mu_r * iu, iu, sg);
    }
    rhs[j] = -g;
    sigma[j] = sg;
  }
}

// Per block: [fraction-to-boundary step of x along dx (tau), -rhs' dx (the
// merit's slope), sum of log gaps of x, ||x - x_R||^2].
__global__ void __launch_bounds__(kIpmThreads) k_resto_dir(
    const double* __restrict__ x, const double* __restrict__ dx, const double* __restrict__ rhs,
    const double* __restrict__ xr, const double* __restrict__ xl, const double* __restrict__ xu,
    int n, double tau, double* __restrict__ part) {
  double a[4] = {1.0, 0.0, 0.0, 0.0};
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double xj = x[j], d = dx[j], lo = xl[j], hi = xu[j];
    a[1] = fma(-rhs[j], d, a[1]);
    if (finite_bound(lo)) {
      if (d < 0.0) a[0] = fmin(a[0], -tau * (xj - lo) / d);
      a[2] += log(xj - lo);
    }
    if (finite_bound(hi)) {
      if (d > 0.0) a[0] = fmin(a[0], tau * (hi - xj) / d);
      a[2] += log(hi - xj);
    }
    const double e = xj - xr[j];
    a[3] = fma(e, e, a[3]);
  }
  block_reduce<4, 1>(a, part);
}

// x_t = x + alpha dx, and per block [sum log gaps of x_t, ||x_t - x_R||^2].
__global__ void __launch_bounds__(kIpmThreads) k_resto_trial(
    const double* __restrict__ x, const double* __restrict__ dx, const double* __restrict__ xr,
    const double* __restrict__ xl, const double* __restrict__ xu, int n, double alpha,
    double* __restrict__ xt, double* __restrict__ part) {
  double a[2] = {0.0, 0.0};
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double v = fma(alpha, dx[j], x[j]), lo = xl[j], hi = xu[j];
    xt[j] = v;
    if (finite_bound(lo)) a[0] += log(v - lo);
    if (finite_bound(hi)) a[0] += log(hi - v);
    const double e = v - xr[j];
    a[1] = fma(e, e, a[1]);
  }
  block_reduce<2, 0>(a, part);
}

// After restoration: y = 0 and the bound multipliers on the central path,
// z = mu / gap at every finite bound of (x, s).
__global__ void __launch_bounds__(kIpmThreads) k_resto_duals(IpmVec v, int n, int m, double mu) {
  const int stride = gridDim.x * kIpmThreads;
  for (int j = blockIdx.x * kIpmThreads + threadIdx.x; j < n; j += stride) {
    const double x = v.x[j], lo = v.xl[j], hi = v.xu[j];
    v.zl_x[j] = finite_bound(lo) ? mu / (x - lo) : 0.0;
    v.zu_x[j] = finite_bound(hi) ? mu / (hi - x) : 0.0;
  }
  for (int r = blockIdx.x * kIpmThreads + threadIdx.x; r < m; r += stride) {
    const double s = v.s[r], lo = v.sl[r], hi = v.su[r];
    v.y[r] = 0.0;
    v.ym[r] = 0.0;
    v.zl_s[r] = finite_bound(lo) ? mu / (s - lo) : 0.0;
    v.zu_s[r] = finite_bound(hi) ? mu / (hi - s) : 0.0;
  }
}

}  // namespace

int ipm_blocks(int sms) { return 4 * sms; }

cudaError_t launch_resto_slack(const double* cons, const double* lo_s, const double* hi_s, int m,
                               double* s, double* r, double* w, int blocks, double* part,
                               double* out, cudaStream_t st) {
  k_resto_slack<<<blocks, kIpmThreads, 0, st>>>(cons, lo_s, hi_s, m, s, r, w, part);
  k_ipm_final<2, 0><<<1, kIpmThreads, 0, st>>>(part, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_resto_grad(const DevStep& step, const double* jvals, const double* r,
                              const double* x, const double* xr, const double* xl,
                              const double* xu, double mu_r, double zeta, double* rhs,
                              double* sigma, int blocks, cudaStream_t s) {
  k_resto_grad<<<blocks, kIpmThreads, 0, s>>>(step, jvals, r, x, xr, xl, xu, mu_r, zeta, rhs,
                                              sigma);
  return cudaGetLastError();
}

cudaError_t launch_resto_dir(const double* x, const double* dx, const double* rhs,
                             const double* xr, const double* xl, const double* xu, int n,
                             double tau, int blocks, double* part, double* out, cudaStream_t s) {
  k_resto_dir<<<blocks, kIpmThreads, 0, s>>>(x, dx, rhs, xr, xl, xu, n, tau, part);
  k_ipm_final<4, 1><<<1, kIpmThreads, 0, s>>>(part, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_resto_trial(const double* x, const double* dx, const double* xr,
                               const double* xl, const double* xu, int n, double alpha,
                               double* xt, int blocks, double* part, double* out,
                               cudaStream_t s) {
  k_resto_trial<<<blocks, kIpmThreads, 0, s>>>(x, dx, xr, xl, xu, n, alpha, xt, part);
  k_ipm_final<2, 0><<<1, kIpmThreads, 0, s>>>(part, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_resto_duals(const IpmVec& v, int n, int m, double mu, int blocks,
                               cudaStream_t s) {
  k_resto_duals<<<blocks, kIpmThreads, 0, s>>>(v, n, m, mu);
  return cudaGetLastError();
}

cudaError_t launch_ipm_rhs(const DevStep& st, const IpmVec& v, double mu, int blocks,
                           cudaStream_t s) {
  k_ipm_rhs<<<blocks, kIpmThreads, 0, s>>>(st, v, mu);
  return cudaGetLastError();
}

cudaError_t launch_ipm_dir(const IpmVec& v, int n, int m, double tau, double mu, int blocks,
                           double* part, double* out, cudaStream_t s) {
  k_ipm_dir<<<blocks, kIpmThreads, 0, s>>>(v, n, m, tau, mu, part);
  k_ipm_final<4, 2><<<1, kIpmThreads, 0, s>>>(part, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_ipm_trial(const IpmVec& v, int n, int m, double alpha, int blocks,
                             cudaStream_t s) {
  k_ipm_trial<<<blocks, kIpmThreads, 0, s>>>(v, n, m, alpha);
  return cudaGetLastError();
}

cudaError_t launch_ipm_measure(const IpmVec& v, const double* x, const double* sv,
                               const double* cons, int n, int m, int blocks, double* part,
                               double* out, cudaStream_t s) {
  k_ipm_measure<<<blocks, kIpmThreads, 0, s>>>(v, x, sv, cons, n, m, part);
  k_ipm_final<2, 0><<<1, kIpmThreads, 0, s>>>(part, blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_soc_rhs(double* c, double* py, const double* cons, const double* sv,
                           const double* ct, const double* st, double a, int m, int blocks,
                           cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_soc_rhs<<<blocks, kIpmThreads, 0, s>>>(c, py, cons, sv, ct, st, a, m);
  return cudaGetLastError();
}

cudaError_t launch_ipm_accept(const IpmVec& v, int n, int m, double alpha, double alpha_z,
                              double mu, double kappa, int blocks, cudaStream_t s) {
  k_ipm_accept<<<blocks, kIpmThreads, 0, s>>>(v, n, m, alpha, alpha_z, mu, kappa);
  return cudaGetLastError();
}

}  // namespace acopf
