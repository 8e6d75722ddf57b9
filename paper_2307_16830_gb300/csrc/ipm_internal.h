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

}  // namespace acopf
