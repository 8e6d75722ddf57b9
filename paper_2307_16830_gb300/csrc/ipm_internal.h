// Device vectors of the interior-point iteration and the launchers of ipm_k.cu.
#pragma once

#include <cuda_runtime.h>

#include "acopf_internal.h"

namespace acopf {

// Every vector of one solve (device pointers): the iterate and its bounds,
// the callbacks' outputs at x, the Newton right-hand side, the step, the
// trial point.
struct IpmVec {
  double *x, *s, *y, *ym;  // ym = -y (the Hessian's multipliers)
  const double *xl, *xu, *sl, *su;
  double *zl_x, *zu_x, *zl_s, *zu_s;
  double *grad, *cons, *jvals;
  double *p_x, *p_s, *p_y, *p_zl_x, *p_zu_x, *p_zl_s, *p_zu_s;
  double *dx, *ds, *dy, *dzl_x, *dzu_x, *dzl_s, *dzu_s;
  double *xt, *st, *cons_t;
};

int ipm_blocks(int sms);
cudaError_t launch_ipm_rhs(const DevStep& st, const IpmVec& v, double mu, int blocks,
                           cudaStream_t s);
// out[0..3] = primal step bound, dual step bound, grad phi' d, sum of log gaps.
cudaError_t launch_ipm_dir(const IpmVec& v, int n, int m, double tau, double mu, int blocks,
                           double* part, double* out, cudaStream_t s);
cudaError_t launch_ipm_trial(const IpmVec& v, int n, int m, double alpha, int blocks,
                             cudaStream_t s);
// out[0..1] = sum |cons - s|, sum of log gaps at (x, s).
cudaError_t launch_ipm_measure(const IpmVec& v, const double* x, const double* sv,
                               const double* cons, int n, int m, int blocks, double* part,
                               double* out, cudaStream_t s);
cudaError_t launch_ipm_accept(const IpmVec& v, int n, int m, double alpha, double alpha_z,
                              double mu, double kappa, int blocks, cudaStream_t s);
// Second-order correction: c = a (cons - sv) + (ct - st) when cons is not
// NULL (the first correction), else c = a c + (ct - st); py = -c.
cudaError_t launch_soc_rhs(double* c, double* py, const double* cons, const double* sv,
                           const double* ct, const double* st, double a, int m, int blocks,
                           cudaStream_t s);

// Feasibility restoration.  s = clip(cons, lo_s, hi_s), r = cons - s, w = 1
// where r != 0 (r, w may be NULL); out[0..1] = sum |r|, sum r^2.
cudaError_t launch_resto_slack(const double* cons, const double* lo_s, const double* hi_s, int m,
                               double* s, double* r, double* w, int blocks, double* part,
                               double* out, cudaStream_t st);
// rhs = -(A'r + mu_r (1/(u-x) - 1/(x-l)) + zeta (x - xr)), sigma the
// barrier's curvature + zeta.
cudaError_t launch_resto_grad(const DevStep& step, const double* jvals, const double* r,
                              const double* x, const double* xr, const double* xl,
                              const double* xu, double mu_r, double zeta, double* rhs,
                              double* sigma, int blocks, cudaStream_t s);
// out[0..3] = fraction-to-boundary step, -rhs'dx, sum log gaps of x, ||x - xr||^2.
cudaError_t launch_resto_dir(const double* x, const double* dx, const double* rhs,
                             const double* xr, const double* xl, const double* xu, int n,
                             double tau, int blocks, double* part, double* out, cudaStream_t s);
// xt = x + alpha dx; out[0..1] = sum log gaps of xt, ||xt - xr||^2.
cudaError_t launch_resto_trial(const double* x, const double* dx, const double* xr,
                               const double* xl, const double* xu, int n, double alpha,
                               double* xt, int blocks, double* part, double* out,
                               cudaStream_t s);
// y = 0 and z = mu / gap at the finite bounds of the iterate.
cudaError_t launch_resto_duals(const IpmVec& v, int n, int m, double mu, int blocks,
                               cudaStream_t s);

}  // namespace acopf
