// sm_103a FP64 kernels of libacopf.
//
// One call of the fused unit of work (objective, gradient, constraints,
// Jacobian, Lagrangian Hessian and the condensed KKT matrix of Sec. IV.C)
// is two launches:
//
//   phase 1  one thread per branch: patterns 3-9 fused around one sincos per
//            branch, which values, Jacobian, the merged Hessian block and the
//            branch's KKT contributions all share.  The branch writes the
//            four arc rows of M_cond directly and leaves its contributions to
//            the bus rows in the slot scratch.
//   phase 2  one thread per bus (patterns 2, 10-15: balance rows summed over
//            the bus's generators and arcs in a fixed order, no atomics; the
//            bus rows of M_cond gathered from the slot partials staged in
//            shared memory), one thread per generator (pattern 1 and the
//            generator rows of M_cond), and one block that reduces the
//            objective in a fixed order.
//
// Phase 2 is launched with programmatic dependent launch: its blocks start
// while phase 1 drains and do all the work that reads only the call's inputs
// before waiting on the grid dependency; only the bus rows of M_cond wait.
//
// Every K entry has one owner thread that writes it (arc rows: branch
// threads; generator rows: generator threads; bus rows: bus threads), so the
// assembly is a gather: deterministic and free of atomics.  Row layouts are
// the ones model.cpp documents.
//
// FP64 throughput on this part is about 0.6 T FMA/s, far below what its
// memory bandwidth could feed, so the kernels are written to minimise FP64
// pipe instructions: the four flows share two trigonometric brackets, the
// Hessians of the four flow rows merge into one weighted bracket, the
// condensation factor is a plain copy when delta_w = delta_c = 0, KKT
// entries of the form D (+-1) J are copies, and stored negations flip the
// sign bit with an integer instruction instead of an FP64 one.
#include <cstdint>

#include "acopf_internal.h"

namespace acopf {
namespace {

__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

// -x with an integer sign-bit flip (keeps the negation off the FP64 pipe).
__device__ __forceinline__ double neg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ static_cast<long long>(0x8000000000000000ULL));
}

// D = (Sigma_s + delta_w) / (delta_c Sigma_s + 1 + delta_c delta_w)  (Sec. IV.C);
// without regularisation D = Sigma_s.
template <bool REG>
__device__ __forceinline__ double dcond(double ss, double dw, double dc) {
  if constexpr (REG) {
    return (ss + dw) / fma(dc, ss, fma(dc, dw, 1.0));
  } else {
    return ss;
  }
}
template <bool REG>
__device__ __forceinline__ double sxw(double sx, double dw) {
  if constexpr (REG) {
    return sx + dw;
  } else {
    return sx;
  }
}

// Fixed-order block sum (warp shuffle tree, then warp 0 over warp sums).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// Writes the four bus entries of an arc row in column order
// (va_lo, va_hi, vm_lo, vm_hi).
__device__ __forceinline__ void put4(double* __restrict__ K, int r0, bool f_lo, double e_vaf,
                                     double e_vat, double e_vmf, double e_vmt) {
  if (f_lo) {
    K[r0 + 0] = e_vaf;
    K[r0 + 1] = e_vat;
    K[r0 + 2] = e_vmf;
    K[r0 + 3] = e_vmt;
  } else {
    K[r0 + 0] = e_vat;
    K[r0 + 1] = e_vaf;
    K[r0 + 2] = e_vmt;
    K[r0 + 3] = e_vmf;
  }
}

// ===========================================================================
// Phase 1, fused path: branch thread.
// ===========================================================================
template <unsigned W, bool REG>
__device__ __forceinline__ void branch_fused(const DevModel& dm, const EvalArgs& a, int l) {
  const Layout& L = dm.L;
  const int nl = L.nl;
  const int f = ld(dm.f + l), t = ld(dm.t + l);
  const double* __restrict__ x = a.x;
  const int iPf = L.P + l, iPt = L.P + nl + l, iQf = L.Q + l, iQt = L.Q + nl + l;

  if constexpr ((W & OUT_GRAD) != 0) {
    a.grad[iPf] = 0.0;
    a.grad[iPt] = 0.0;
    a.grad[iQf] = 0.0;
    a.grad[iQt] = 0.0;
  }
  if constexpr ((W & OUT_JAC) != 0) {
    double* __restrict__ J = a.jvals;
    J[L.JPF + 5 * l] = 1.0;
    J[L.JQF + 5 * l] = 1.0;
    J[L.JPT + 5 * l] = 1.0;
    J[L.JQT + 5 * l] = 1.0;
    J[L.JANG + 2 * l] = 1.0;
    J[L.JANG + 2 * l + 1] = -1.0;
    J[L.JPBA + l] = 1.0;
    J[L.JPBA + nl + l] = 1.0;
    J[L.JQBA + l] = 1.0;
    J[L.JQBA + nl + l] = 1.0;
  }
  constexpr bool kNeedFlows = (W & (OUT_CONS | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  if constexpr (!kNeedFlows) {
    return;
  } else {
    const double va_f = ld(x + L.VA + f), va_t = ld(x + L.VA + t);
    const double vm_f = ld(x + L.VM + f), vm_t = ld(x + L.VM + t);
    const double* __restrict__ cf = dm.coef;
    const double g_ff = ld(cf + CG_FF * nl + l), b_ff = ld(cf + CB_FF * nl + l);
    const double g_ft = ld(cf + CG_FT * nl + l), b_ft = ld(cf + CB_FT * nl + l);
    const double g_tf = ld(cf + CG_TF * nl + l), b_tf = ld(cf + CB_TF * nl + l);
    const double g_tt = ld(cf + CG_TT * nl + l), b_tt = ld(cf + CB_TT * nl + l);

    const double th = va_f - va_t;
    double s, c;
    sincos(th, &s, &c);
    // Trigonometric brackets of the four flows F = a vm_f^2 + d vm_t^2 + V T(th):
    //   P_f: T = E_f,   T' = Ep_f      Q_f: T = -Ep_f, T' = E_f
    //   P_t: T = E_t,   T' = Ep_t      Q_t: T = Ep_t,  T' = -E_t
    const double E_f = fma(g_ft, c, b_ft * s);
    const double Ep_f = fma(b_ft, c, -(g_ft * s));
    const double E_t = fma(g_tf, c, -(b_tf * s));
    const double Ep_t = -fma(g_tf, s, b_tf * c);

    const double vtE_f = vm_t * E_f, vtEp_f = vm_t * Ep_f;
    const double vfE_t = vm_f * E_t, vfEp_t = vm_f * Ep_t;
    const double VE_f = vm_f * vtE_f, VEp_f = vm_f * vtEp_f;
    const double VE_t = vm_t * vfE_t, VEp_t = vm_t * vfEp_t;
    const double tvf = vm_f + vm_f, tvt = vm_t + vm_t;

    // dF/dth, dF/dvm_f, dF/dvm_t of each flow (th_qt = -VE_t is used negated).
    const double th_pf = VEp_f, th_qf = VE_f, th_pt = VEp_t;
    const double mf_pf = fma(g_ff, tvf, vtE_f), mt_pf = vm_f * E_f;
    const double mf_qf = fma(-b_ff, tvf, -vtEp_f), nmt_qf = vm_f * Ep_f;  // nmt_qf = -mt_qf
    const double mf_pt = vm_t * E_t, mt_pt = fma(g_tt, tvt, vfE_t);
    const double mf_qt = vm_t * Ep_t, mt_qt = fma(-b_tt, tvt, vfEp_t);

    const double p_f = ld(x + iPf), p_t = ld(x + iPt), q_f = ld(x + iQf), q_t = ld(x + iQt);
    if constexpr ((W & OUT_CONS) != 0) {
      const double vmf2 = vm_f * vm_f, vmt2 = vm_t * vm_t;
      // g = var - F
      double* __restrict__ g = a.cons;
      g[L.PF + l] = p_f - fma(g_ff, vmf2, VE_f);
      g[L.QF + l] = q_f + fma(b_ff, vmf2, VEp_f);
      g[L.PT + l] = p_t - fma(g_tt, vmt2, VE_t);
      g[L.QT + l] = q_t - fma(-b_tt, vmt2, VEp_t);
      g[L.ANG + l] = th;
      g[L.SF + l] = fma(p_f, p_f, q_f * q_f);
      g[L.ST + l] = fma(p_t, p_t, q_t * q_t);
    }
    const double jp_f = p_f + p_f, jq_f = q_f + q_f, jp_t = p_t + p_t, jq_t = q_t + q_t;
    if constexpr ((W & OUT_JAC) != 0) {
      // J row = [1, -dF/dth, dF/dth, -dF/dvm_f, -dF/dvm_t]
      double* __restrict__ J = a.jvals;
      double* jp = J + L.JPF + 5 * l;
      jp[1] = neg(th_pf);
      jp[2] = th_pf;
      jp[3] = neg(mf_pf);
      jp[4] = neg(mt_pf);
      jp = J + L.JQF + 5 * l;
      jp[1] = neg(th_qf);
      jp[2] = th_qf;
      jp[3] = neg(mf_qf);
      jp[4] = nmt_qf;
      jp = J + L.JPT + 5 * l;
      jp[1] = neg(th_pt);
      jp[2] = th_pt;
      jp[3] = neg(mf_pt);
      jp[4] = neg(mt_pt);
      jp = J + L.JQT + 5 * l;
      jp[1] = VE_t;
      jp[2] = neg(VE_t);
      jp[3] = neg(mf_qt);
      jp[4] = neg(mt_qt);
      J[L.JSF + 2 * l] = jp_f;
      J[L.JSF + 2 * l + 1] = jq_f;
      J[L.JST + 2 * l] = jp_t;
      J[L.JST + 2 * l + 1] = jq_t;
    }
    constexpr bool kNeedH = (W & (OUT_HESS | OUT_KKT)) != 0;
    if constexpr (kNeedH) {
      const double* __restrict__ y = a.y;
      const double y_pf = ld(y + L.PF + l), y_qf = ld(y + L.QF + l);
      const double y_pt = ld(y + L.PT + l), y_qt = ld(y + L.QT + l);
      const double y_sf = ld(y + L.SF + l), y_st = ld(y + L.ST + l);
      // Merged Hessian of the flow rows: with w_k = -y_k,
      //   TH = sum_k w_k T_k, TP = sum_k w_k T'_k, AF = sum_k w_k a_k, AT = sum_k w_k d_k;
      // nTH = -TH, nTP = -TP are computed.
      const double nTH = fma(y_pf, E_f, fma(-y_qf, Ep_f, fma(y_pt, E_t, y_qt * Ep_t)));
      const double nTP = fma(y_pf, Ep_f, fma(y_qf, E_f, fma(y_pt, Ep_t, -(y_qt * E_t))));
      const double AF = fma(-y_pf, g_ff, y_qf * b_ff);
      const double AT = fma(-y_pt, g_tt, y_qt * b_tt);
      const double V = vm_f * vm_t;
      const double VnTH = V * nTH;
      const double vtTP = vm_t * nTP, vfTP = vm_f * nTP;  // = -(vm TP)
      const double AF2 = AF + AF, AT2 = AT + AT;
      const double hs_f = y_sf + y_sf, hs_t = y_st + y_st;
      if constexpr ((W & OUT_HESS) != 0) {
        double* __restrict__ H = a.hvals + L.HBLK + 10 * l;
        H[0] = VnTH;
        H[1] = neg(VnTH);
        H[2] = VnTH;
        H[3] = neg(vtTP);
        H[4] = vtTP;
        H[5] = AF2;
        H[6] = neg(vfTP);
        H[7] = vfTP;
        H[8] = neg(nTH);
        H[9] = AT2;
        double* __restrict__ Ht = a.hvals + L.HTH + 4 * l;
        Ht[0] = hs_f;
        Ht[1] = hs_f;
        Ht[2] = hs_t;
        Ht[3] = hs_t;
      }
      if constexpr ((W & OUT_KKT) != 0) {
        const double* __restrict__ ss = a.sigma_s;
        const double* __restrict__ sx = a.sigma_x;
        const double dw = a.delta_w, dc = a.delta_c;
        const double D_pf = dcond<REG>(ld(ss + L.PF + l), dw, dc);
        const double D_qf = dcond<REG>(ld(ss + L.QF + l), dw, dc);
        const double D_pt = dcond<REG>(ld(ss + L.PT + l), dw, dc);
        const double D_qt = dcond<REG>(ld(ss + L.QT + l), dw, dc);
        const double D_an = dcond<REG>(ld(ss + L.ANG + l), dw, dc);
        const double D_sf = dcond<REG>(ld(ss + L.SF + l), dw, dc);
        const double D_st = dcond<REG>(ld(ss + L.ST + l), dw, dc);
        const double D_Pf = dcond<REG>(ld(ss + L.PB + f), dw, dc);
        const double D_Qf = dcond<REG>(ld(ss + L.QB + f), dw, dc);
        const double D_Pt = dcond<REG>(ld(ss + L.PB + t), dw, dc);
        const double D_Qt = dcond<REG>(ld(ss + L.QB + t), dw, dc);

        // D_k times dF_k/dth, dF_k/dvm_f, dF_k/dvm_t (th_qt = -VE_t folds into signs).
        const double A_pf = D_pf * th_pf, A_qf = D_qf * th_qf, A_pt = D_pt * th_pt,
                     nA_qt = D_qt * VE_t;
        const double B_pf = D_pf * mf_pf, B_qf = D_qf * mf_qf, B_pt = D_pt * mf_pt,
                     B_qt = D_qt * mf_qt;
        const double C_pf = D_pf * mt_pf, nC_qf = D_qf * nmt_qf, C_pt = D_pt * mt_pt,
                     C_qt = D_qt * mt_qt;
        // Block sums over the four flow rows: S1 = sum D th^2, S2 = sum D th mf,
        // S3 = sum D th mt, S4 = sum D mf^2, S5 = sum D mf mt, S6 = sum D mt^2.
        const double S1 = fma(A_pf, th_pf, fma(A_qf, th_qf, fma(A_pt, th_pt, nA_qt * VE_t)));
        const double S2 = fma(A_pf, mf_pf, fma(A_qf, mf_qf, fma(A_pt, mf_pt, -(nA_qt * mf_qt))));
        const double S3 = fma(A_pf, mt_pf, fma(-A_qf, nmt_qf, fma(A_pt, mt_pt, -(nA_qt * mt_qt))));
        const double S4 = fma(B_pf, mf_pf, fma(B_qf, mf_qf, fma(B_pt, mf_pt, B_qt * mf_qt)));
        const double S5 = fma(B_pf, mt_pf, fma(-B_qf, nmt_qf, fma(B_pt, mt_pt, B_qt * mt_qt)));
        const double S6 = fma(C_pf, mt_pf, fma(nC_qf, nmt_qf, fma(C_pt, mt_pt, C_qt * mt_qt)));
        // The branch's (va_f, va_t, vm_f, vm_t) block of W + A'DA over its
        // flow and angle rows:  (va_f,va_f) = (va_t,va_t) = aa = -(va_t,va_f),
        // (vm_f,va_f) = maf = -(vm_f,va_t), (vm_t,va_f) = mat = -(vm_t,va_t).
        const double aa = (S1 + D_an) + VnTH;
        const double maf = S2 - vtTP;
        const double mat = S3 - vfTP;
        const double mmf = S4 + AF2;
        const double mmt = S6 + AT2;
        const double ww = S5 - nTH;
        const double naa = neg(aa);
        dm.part_slot[ld(dm.slot_of_arc + l)] = SlotPart{aa, maf, mmf, neg(maf), naa, ww};
        dm.part_slot[ld(dm.slot_of_arc + nl + l)] = SlotPart{aa, neg(mat), mmt, mat, naa, ww};

        // Arc rows.  Balance-row coefficient of vm at the arc's bus:
        // Pbal: 2 Gs vm, Qbal: -2 Bs vm.
        const double jPv_f = ld(dm.Gs + f) * tvf, jQv_f = -(ld(dm.Bs + f) * tvf);
        const double jPv_t = ld(dm.Gs + t) * tvt, jQv_t = -(ld(dm.Bs + t) * tvt);
        const double Dsp_f = D_sf * jp_f, Dsp_t = D_st * jp_t;
        const int* __restrict__ rp = dm.krowptr;
        double* __restrict__ K = a.kvals;
        const bool f_lo = f < t;
        const int ngf = ld(dm.gen_ptr + f + 1) - ld(dm.gen_ptr + f);
        const int ngt = ld(dm.gen_ptr + t + 1) - ld(dm.gen_ptr + t);
        const double nD_Pf = neg(D_Pf), nD_Qf = neg(D_Qf), nD_Pt = neg(D_Pt), nD_Qt = neg(D_Qt);
        // row p_l (from arc, bus f)
        {
          const int r0 = ld(rp + iPf), r1 = ld(rp + iPf + 1);
          put4(K, r0, f_lo, neg(A_pf), A_pf, fma(D_Pf, jPv_f, -B_pf), neg(C_pf));
          int k = r0 + 4;
          for (int e = 0; e < ngf; ++e) K[k++] = nD_Pf;
          for (; k < r1 - 1; ++k) K[k] = D_Pf;
          K[r1 - 1] = sxw<REG>(ld(sx + iPf), dw) + hs_f + D_pf + fma(Dsp_f, jp_f, D_Pf);
        }
        // row q_l
        {
          const int r0 = ld(rp + iQf), r1 = ld(rp + iQf + 1);
          put4(K, r0, f_lo, neg(A_qf), A_qf, fma(D_Qf, jQv_f, -B_qf), nC_qf);
          int k = r0 + 4;
          for (int e = 0; e < ngf; ++e) K[k++] = nD_Qf;
          K[k++] = Dsp_f * jq_f;
          for (; k < r1 - 1; ++k) K[k] = D_Qf;
          K[r1 - 1] = sxw<REG>(ld(sx + iQf), dw) + hs_f + D_qf + fma(D_sf * jq_f, jq_f, D_Qf);
        }
        // row p_{nl+l} (to arc, bus t)
        {
          const int r0 = ld(rp + iPt), r1 = ld(rp + iPt + 1);
          put4(K, r0, f_lo, neg(A_pt), A_pt, neg(B_pt), fma(D_Pt, jPv_t, -C_pt));
          int k = r0 + 4;
          for (int e = 0; e < ngt; ++e) K[k++] = nD_Pt;
          for (; k < r1 - 1; ++k) K[k] = D_Pt;
          K[r1 - 1] = sxw<REG>(ld(sx + iPt), dw) + hs_t + D_pt + fma(Dsp_t, jp_t, D_Pt);
        }
        // row q_{nl+l}
        {
          const int r0 = ld(rp + iQt), r1 = ld(rp + iQt + 1);
          put4(K, r0, f_lo, nA_qt, neg(nA_qt), neg(B_qt), fma(D_Qt, jQv_t, -C_qt));
          int k = r0 + 4;
          for (int e = 0; e < ngt; ++e) K[k++] = nD_Qt;
          K[k++] = Dsp_t * jq_t;
          for (; k < r1 - 1; ++k) K[k] = D_Qt;
          K[r1 - 1] = sxw<REG>(ld(sx + iQt), dw) + hs_t + D_qt + fma(D_st * jq_t, jq_t, D_Qt);
        }
      }
    }
  }
}

template <unsigned W, bool REG>
__global__ void __launch_bounds__(kBranchThreads, 6) k_phase1(DevModel dm, EvalArgs a) {
  pdl_trigger();
  const int l = blockIdx.x * kBranchThreads + threadIdx.x;
  if (l < dm.L.nl) branch_fused<W, REG>(dm, a, l);
}

// ===========================================================================
// Phase 1 of the array-fed assembly (M_cond from given H and J values).
// ===========================================================================
template <bool REG>
__device__ __forceinline__ void branch_from_arrays(const DevModel& dm, const EvalArgs& a, int l) {
  const Layout& L = dm.L;
  const int nl = L.nl;
  const int f = ld(dm.f + l), t = ld(dm.t + l);
  const double* __restrict__ J = a.jvals_in;
  const double* __restrict__ Hv = a.hvals_in;
  const double* __restrict__ ss = a.sigma_s;
  const double* __restrict__ sx = a.sigma_x;
  const double dw = a.delta_w, dc = a.delta_c;
  const int base[4] = {L.JPF, L.JQF, L.JPT, L.JQT};
  const int crow[4] = {L.PF, L.QF, L.PT, L.QT};
  double j[4][5], D[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int e = 0; e < 5; ++e) j[q][e] = ld(J + base[q] + 5 * l + e);
    D[q] = dcond<REG>(ld(ss + crow[q] + l), dw, dc);
  }
  const double ja0 = ld(J + L.JANG + 2 * l), ja1 = ld(J + L.JANG + 2 * l + 1);
  const double D_an = dcond<REG>(ld(ss + L.ANG + l), dw, dc);
  // block over local (va_f, va_t, vm_f, vm_t) = Jacobian columns 1..4
  double blk[10];
  const int pu[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
  const int pv[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
#pragma unroll
  for (int e = 0; e < 10; ++e) {
    double acc = ld(Hv + L.HBLK + 10 * l + e);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc = fma(D[q] * j[q][1 + pu[e]], j[q][1 + pv[e]], acc);
    blk[e] = acc;
  }
  blk[0] = fma(D_an * ja0, ja0, blk[0]);
  blk[1] = fma(D_an * ja1, ja0, blk[1]);
  blk[2] = fma(D_an * ja1, ja1, blk[2]);
  // blk: 0 (va_f,va_f) 1 (va_t,va_f) 2 (va_t,va_t) 3 (vm_f,va_f) 4 (vm_f,va_t)
  //      5 (vm_f,vm_f) 6 (vm_t,va_f) 7 (vm_t,va_t) 8 (vm_t,vm_f) 9 (vm_t,vm_t)
  dm.part_slot[ld(dm.slot_of_arc + l)] = SlotPart{blk[0], blk[3], blk[5], blk[4], blk[1], blk[8]};
  dm.part_slot[ld(dm.slot_of_arc + nl + l)] =
      SlotPart{blk[2], blk[7], blk[9], blk[6], blk[1], blk[8]};

  // arc rows
  const double js_f0 = ld(J + L.JSF + 2 * l), js_f1 = ld(J + L.JSF + 2 * l + 1);
  const double js_t0 = ld(J + L.JST + 2 * l), js_t1 = ld(J + L.JST + 2 * l + 1);
  const double D_sf = dcond<REG>(ld(ss + L.SF + l), dw, dc);
  const double D_st = dcond<REG>(ld(ss + L.ST + l), dw, dc);
  const int* __restrict__ rp = dm.krowptr;
  double* __restrict__ K = a.kvals;
  const bool f_lo = f < t;
  // q = 0: p_l (bus f), 1: q_l (bus f), 2: p_{nl+l} (bus t), 3: q_{nl+l} (bus t)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool to = q >= 2, isq = (q & 1) != 0;
    const int bus = to ? t : f;
    const int arc = to ? nl + l : l;
    const int var = (isq ? L.Q : L.P) + arc;
    const int brow = (isq ? L.QB : L.PB) + bus;
    const double D_B = dcond<REG>(ld(ss + brow), dw, dc);
    const double jBa = ld(J + (isq ? L.JQBA : L.JPBA) + arc);  // arc var in balance row
    const double jBv = ld(J + (isq ? L.JQBV : L.JPBV) + bus);  // vm in balance row
    const double js0 = to ? js_t0 : js_f0, js1 = to ? js_t1 : js_f1;
    const double D_s = to ? D_st : D_sf;
    const double DBa = D_B * jBa;
    const double Dj0 = D[q] * j[q][0];
    double e_vaf = Dj0 * j[q][1], e_vat = Dj0 * j[q][2];
    double e_vmf = Dj0 * j[q][3], e_vmt = Dj0 * j[q][4];
    if (to)
      e_vmt = fma(DBa, jBv, e_vmt);
    else
      e_vmf = fma(DBa, jBv, e_vmf);
    const int r0 = ld(rp + var), r1 = ld(rp + var + 1);
    put4(K, r0, f_lo, e_vaf, e_vat, e_vmf, e_vmt);
    int k = r0 + 4;
    const int g0 = ld(dm.gen_ptr + bus), g1 = ld(dm.gen_ptr + bus + 1);
    const int gsec = isq ? L.JQBG : L.JPBG;
    for (int e = g0; e < g1; ++e) K[k++] = DBa * ld(J + gsec + ld(dm.gens_at + e));
    if (isq) K[k++] = D_s * js0 * js1;
    const int asec = isq ? L.JQBA : L.JPBA;
    const int a0 = ld(dm.arc_ptr + bus);
    for (int e = a0; k < r1 - 1; ++e) K[k++] = DBa * ld(J + asec + ld(dm.arcs_by_idx + e));
    const double jsv = isq ? js1 : js0;
    const double hth = ld(Hv + L.HTH + 4 * l + q);
    K[r1 - 1] =
        sxw<REG>(ld(sx + var), dw) + hth + fma(Dj0, j[q][0], fma(D_s * jsv, jsv, DBa * jBa));
  }
}

template <bool REG>
__global__ void __launch_bounds__(kBranchThreads) k_asm_phase1(DevModel dm, EvalArgs a) {
  pdl_trigger();
  const int l = blockIdx.x * kBranchThreads + threadIdx.x;
  if (l < dm.L.nl) branch_from_arrays<REG>(dm, a, l);
}

// ===========================================================================
// Phase 2: generator threads (no dependency on phase 1).
// ===========================================================================
template <unsigned W, bool REG>
__device__ __forceinline__ void gen_fused(const DevModel& dm, const EvalArgs& a, int g) {
  const Layout& L = dm.L;
  const double* __restrict__ x = a.x;
  if constexpr ((W & OUT_GRAD) != 0) {
    a.grad[L.PG + g] = fma(ld(dm.c2 + g) + ld(dm.c2 + g), ld(x + L.PG + g), ld(dm.c1 + g));
    a.grad[L.QG + g] = 0.0;
  }
  if constexpr ((W & OUT_JAC) != 0) {
    a.jvals[L.JPBG + g] = -1.0;
    a.jvals[L.JQBG + g] = -1.0;
  }
  if constexpr ((W & (OUT_HESS | OUT_KKT)) != 0) {
    const double c2 = ld(dm.c2 + g);
    const double hg = a.obj_weight * (c2 + c2);
    if constexpr ((W & OUT_HESS) != 0) a.hvals[L.HG + g] = hg;
    if constexpr ((W & OUT_KKT) != 0) {
      const int i = ld(dm.gbus + g);
      const double dw = a.delta_w, dc = a.delta_c;
      const double D_P = dcond<REG>(ld(a.sigma_s + L.PB + i), dw, dc);
      const double D_Q = dcond<REG>(ld(a.sigma_s + L.QB + i), dw, dc);
      const double tv = 2.0 * ld(x + L.VM + i);
      double* __restrict__ K = a.kvals;
      const int* __restrict__ rp = dm.krowptr;
      // row pg_g: (pg, vm_i) = D_P (-1)(2 Gs vm), earlier generators D_P, diagonal
      {
        const int r0 = ld(rp + L.PG + g), r1 = ld(rp + L.PG + g + 1);
        K[r0] = neg(D_P * (ld(dm.Gs + i) * tv));
        for (int k = r0 + 1; k < r1 - 1; ++k) K[k] = D_P;
        K[r1 - 1] = sxw<REG>(ld(a.sigma_x + L.PG + g), dw) + hg + D_P;
      }
      // row qg_g: (qg, vm_i) = D_Q (-1)(-2 Bs vm)
      {
        const int r0 = ld(rp + L.QG + g), r1 = ld(rp + L.QG + g + 1);
        K[r0] = D_Q * (ld(dm.Bs + i) * tv);
        for (int k = r0 + 1; k < r1 - 1; ++k) K[k] = D_Q;
        K[r1 - 1] = sxw<REG>(ld(a.sigma_x + L.QG + g), dw) + D_Q;
      }
    }
  }
}

template <bool REG>
__device__ __forceinline__ void gen_from_arrays(const DevModel& dm, const EvalArgs& a, int g) {
  const Layout& L = dm.L;
  const int i = ld(dm.gbus + g);
  const double* __restrict__ J = a.jvals_in;
  const double dw = a.delta_w, dc = a.delta_c;
  const double D_P = dcond<REG>(ld(a.sigma_s + L.PB + i), dw, dc);
  const double D_Q = dcond<REG>(ld(a.sigma_s + L.QB + i), dw, dc);
  const int* __restrict__ rp = dm.krowptr;
  double* __restrict__ K = a.kvals;
  const int g0 = ld(dm.gen_ptr + i);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double D_B = q ? D_Q : D_P;
    const int gsec = q ? L.JQBG : L.JPBG;
    const double jg = ld(J + gsec + g);
    const double jv = ld(J + (q ? L.JQBV : L.JPBV) + i);
    const int var = (q ? L.QG : L.PG) + g;
    const int r0 = ld(rp + var), r1 = ld(rp + var + 1);
    const double Dj = D_B * jg;
    K[r0] = Dj * jv;
    for (int k = r0 + 1, e = g0; k < r1 - 1; ++k, ++e) K[k] = Dj * ld(J + gsec + ld(dm.gens_at + e));
    const double hd = q ? 0.0 : ld(a.hvals_in + L.HG + g);
    K[r1 - 1] = sxw<REG>(ld(a.sigma_x + var), dw) + hd + Dj * jg;
  }
}

// ===========================================================================
// Phase 2: bus rows of M_cond from the slot partials.
// ===========================================================================
// sp / sn: the block's slot partials and neighbours (shared memory or
// global), indexed from the block's first slot s0.
__device__ __forceinline__ void bus_kkt_rows(const DevModel& dm, const EvalArgs& a, int i, int s0,
                                             const SlotPart* sp, const int* sn, double d_va,
                                             double d_vm) {
  const Layout& L = dm.L;
  const int* __restrict__ rp = dm.krowptr;
  double* __restrict__ K = a.kvals;
  const int bva = ld(rp + L.VA + i), eva = ld(rp + L.VA + i + 1);
  const int bvm = ld(rp + L.VM + i), evm = ld(rp + L.VM + i + 1);
  const int nlo = eva - bva - 1;  // distinct neighbours below i
  // Row va_i = [va_j (j < i) ..., va_i];
  // row vm_i = [va_j / va_i ascending (nu + 1)][vm_j (j < i)][vm_i], or just
  // [vm_i] for a bus without branches.
  const int nu = evm - bvm - nlo - 2;
  int pva = bva, pvmva = bvm, pvmvm = bvm + nu + 1;
  double aa = 0.0, ma = 0.0, mm = 0.0;
  double gv = 0.0, gx = 0.0, gw = 0.0;
  int cur = -1;
  const int k0 = ld(dm.arc_ptr + i) - s0, k1 = ld(dm.arc_ptr + i + 1) - s0;
  for (int k = k0; k < k1; ++k) {
    const int j = sn[k];
    const SlotPart p = sp[k];
    aa += p.aa;
    ma += p.ma;
    mm += p.mm;
    if (j != cur) {
      if (cur >= 0) {
        if (cur > i && pvmva == bvm + nlo) ++pvmva;  // skip the (vm_i, va_i) slot
        K[pvmva++] = gx;
        if (cur < i) {
          K[pva++] = gv;
          K[pvmvm++] = gw;
        }
      }
      cur = j;
      gv = p.vv;
      gx = p.mx;
      gw = p.ww;
    } else {
      gv += p.vv;
      gx += p.mx;
      gw += p.ww;
    }
  }
  if (cur >= 0) {
    if (cur > i && pvmva == bvm + nlo) ++pvmva;
    K[pvmva++] = gx;
    if (cur < i) {
      K[pva++] = gv;
      K[pvmvm++] = gw;
    }
  }
  K[bva + nlo] = d_va + aa;
  if (k1 > k0) K[bvm + nlo] = ma;  // (vm_i, va_i) exists only when bus i has a branch
  K[evm - 1] = d_vm + mm;
}

template <unsigned W, bool REG, bool ARRAYS>
__device__ __forceinline__ void bus_block(const DevModel& dm, const EvalArgs& a, int blk,
                                          double* smem) {
  const Layout& L = dm.L;
  const int i0 = blk * kBusThreads;
  const int i = i0 + threadIdx.x;
  const bool active = i < L.nb;
  const double* __restrict__ x = a.x;
  // Work that reads only the call's inputs.
  double d_va = 0.0, d_vm = 0.0;
  if (active) {
    const int r = ld(dm.ref_row + i);
    if constexpr (!ARRAYS) {
      const double vm = ld(x + L.VM + i);
      const double Gs = ld(dm.Gs + i), Bs = ld(dm.Bs + i);
      const double tv = vm + vm;
      const double jPv = Gs * tv, jQv = -(Bs * tv);
      if constexpr ((W & OUT_GRAD) != 0) {
        a.grad[L.VA + i] = 0.0;
        a.grad[L.VM + i] = 0.0;
      }
      if constexpr ((W & OUT_CONS) != 0) {
        if (r >= 0) a.cons[L.REF + r] = ld(x + L.VA + i);
        double P = fma(Gs * vm, vm, ld(dm.Pd + i));
        double Q = fma(-(Bs * vm), vm, ld(dm.Qd + i));
        const int g0 = ld(dm.gen_ptr + i), g1 = ld(dm.gen_ptr + i + 1);
        for (int k = g0; k < g1; ++k) {
          const int g = ld(dm.gens_at + k);
          P -= ld(x + L.PG + g);
          Q -= ld(x + L.QG + g);
        }
        const int k0 = ld(dm.arc_ptr + i), k1 = ld(dm.arc_ptr + i + 1);
        for (int k = k0; k < k1; ++k) {
          const int arc = ld(dm.arcs_by_idx + k);
          P += ld(x + L.P + arc);
          Q += ld(x + L.Q + arc);
        }
        a.cons[L.PB + i] = P;
        a.cons[L.QB + i] = Q;
      }
      if constexpr ((W & OUT_JAC) != 0) {
        if (r >= 0) a.jvals[L.JREF + r] = 1.0;
        a.jvals[L.JPBV + i] = jPv;
        a.jvals[L.JQBV + i] = jQv;
      }
      if constexpr ((W & (OUT_HESS | OUT_KKT)) != 0) {
        const double hb = fma(Gs + Gs, ld(a.y + L.PB + i), -((Bs + Bs) * ld(a.y + L.QB + i)));
        if constexpr ((W & OUT_HESS) != 0) a.hvals[L.HB + i] = hb;
        if constexpr ((W & OUT_KKT) != 0) {
          const double dw = a.delta_w, dc = a.delta_c;
          const double D_P = dcond<REG>(ld(a.sigma_s + L.PB + i), dw, dc);
          const double D_Q = dcond<REG>(ld(a.sigma_s + L.QB + i), dw, dc);
          d_va = sxw<REG>(ld(a.sigma_x + L.VA + i), dw);
          if (r >= 0) d_va += dcond<REG>(ld(a.sigma_s + L.REF + r), dw, dc);
          d_vm = sxw<REG>(ld(a.sigma_x + L.VM + i), dw) + hb +
                 fma(D_P * jPv, jPv, D_Q * jQv * jQv);
        }
      }
    } else {
      const double* __restrict__ J = a.jvals_in;
      const double dw = a.delta_w, dc = a.delta_c;
      const double jPv = ld(J + L.JPBV + i), jQv = ld(J + L.JQBV + i);
      const double D_P = dcond<REG>(ld(a.sigma_s + L.PB + i), dw, dc);
      const double D_Q = dcond<REG>(ld(a.sigma_s + L.QB + i), dw, dc);
      d_va = sxw<REG>(ld(a.sigma_x + L.VA + i), dw);
      if (r >= 0) {
        const double jr = ld(J + L.JREF + r);
        d_va += dcond<REG>(ld(a.sigma_s + L.REF + r), dw, dc) * jr * jr;
      }
      d_vm = sxw<REG>(ld(a.sigma_x + L.VM + i), dw) + ld(a.hvals_in + L.HB + i) +
             fma(D_P * jPv, jPv, D_Q * jQv * jQv);
    }
  }
  if constexpr ((W & OUT_KKT) != 0) {
    pdl_wait();
    const int i1 = min(i0 + kBusThreads, L.nb);
    const int s0 = ld(dm.arc_ptr + i0), s1 = ld(dm.arc_ptr + i1);
    const int ns = s1 - s0;
    const SlotPart* sp = dm.part_slot + s0;
    const int* sn = dm.slot_nbr + s0;
    if (ns <= dm.slot_cap) {
      // Stage the block's slot partials (contiguous in global memory) in shared memory.
      double2* d2 = reinterpret_cast<double2*>(smem);
      const double2* g2 = reinterpret_cast<const double2*>(dm.part_slot + s0);
      for (int k = threadIdx.x; k < 3 * ns; k += kBusThreads) d2[k] = g2[k];
      int* si = reinterpret_cast<int*>(smem + 6 * dm.slot_cap);
      for (int k = threadIdx.x; k < ns; k += kBusThreads) si[k] = ld(dm.slot_nbr + s0 + k);
      __syncthreads();
      sp = reinterpret_cast<const SlotPart*>(smem);
      sn = si;
    }
    if (active) bus_kkt_rows(dm, a, i, s0, sp, sn, d_va, d_vm);
  }
}

// Block roles: [0, nbus) bus blocks, [nbus, nbus + ngen) generator blocks,
// then one objective block when W has OUT_OBJ.
template <unsigned W, bool REG, bool ARRAYS>
__global__ void __launch_bounds__(kBusThreads) k_phase2(DevModel dm, EvalArgs a, int nbus,
                                                       int ngen) {
  extern __shared__ double smem[];
  const int b = blockIdx.x;
  if (b < nbus) {
    bus_block<W, REG, ARRAYS>(dm, a, b, smem);
  } else if (b < nbus + ngen) {
    const int g = (b - nbus) * kGenThreads + threadIdx.x;
    if (g < dm.L.ng) {
      if constexpr (ARRAYS)
        gen_from_arrays<REG>(dm, a, g);
      else
        gen_fused<W, REG>(dm, a, g);
    }
  } else if constexpr ((W & OUT_OBJ) != 0) {
    // objective: fixed-order sum over all generators
    const Layout& L = dm.L;
    double s = 0.0;
    for (int g = threadIdx.x; g < L.ng; g += kGenThreads)
      s += fma(fma(ld(dm.c2 + g), ld(a.x + L.PG + g), ld(dm.c1 + g)), ld(a.x + L.PG + g),
               ld(dm.c0 + g));
    s = block_sum<kGenThreads>(s, smem);
    if (threadIdx.x == 0) *a.f = s;
  }
}

// FP64 FMA throughput probe: 8 independent dependent chains per thread.
__global__ void k_fp64_probe(double* out, int iters) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  const double m = 0.9999999, c = 1e-7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, m, c);
    x1 = fma(x1, m, c);
    x2 = fma(x2, m, c);
    x3 = fma(x3, m, c);
    x4 = fma(x4, m, c);
    x5 = fma(x5, m, c);
    x6 = fma(x6, m, c);
    x7 = fma(x7, m, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename Kern, typename... Args>
cudaError_t launch_ex(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

size_t phase2_smem(const DevModel& dm) {
  const size_t b = size_t(dm.slot_cap) * kSlotBytes;
  return b < 64 ? 64 : (b + 15) / 16 * 16;
}

template <unsigned W, bool REG, bool ARRAYS>
cudaError_t launch_phase2(const DevModel& dm, const EvalArgs& a, cudaStream_t s, bool pdl) {
  const Layout& L = dm.L;
  constexpr bool kBus = (W & (OUT_GRAD | OUT_CONS | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  constexpr bool kGen = (W & (OUT_GRAD | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  const int nbus = kBus ? ceil_div(L.nb, kBusThreads) : 0;
  const int ngen = kGen ? ceil_div(L.ng, kGenThreads) : 0;
  const int nobj = (W & OUT_OBJ) != 0 ? 1 : 0;
  const int blocks = nbus + ngen + nobj;
  if (blocks == 0) return cudaSuccess;
  return launch_ex(k_phase2<W, REG, ARRAYS>, dim3(blocks), dim3(kBusThreads), phase2_smem(dm), s,
                   pdl, dm, a, nbus, ngen);
}

template <unsigned W, bool REG>
cudaError_t launch_eval_t(const DevModel& dm, const EvalArgs& a, cudaStream_t s,
                          cudaEvent_t mid) {
  const Layout& L = dm.L;
  constexpr bool kBranch = (W & (OUT_GRAD | OUT_CONS | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  const int nbb = kBranch ? ceil_div(L.nl, kBranchThreads) : 0;
  if (nbb > 0) {
    k_phase1<W, REG><<<nbb, kBranchThreads, 0, s>>>(dm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (mid) {
    cudaError_t e = cudaEventRecord(mid, s);
    if (e != cudaSuccess) return e;
  }
  return launch_phase2<W, REG, false>(dm, a, s, nbb > 0 && !mid);
}

template <unsigned W>
cudaError_t launch_eval_w(const DevModel& dm, const EvalArgs& a, cudaStream_t s, cudaEvent_t mid) {
  const bool reg = (W & OUT_KKT) != 0 && (a.delta_w != 0.0 || a.delta_c != 0.0);
  return reg ? launch_eval_t<W, true>(dm, a, s, mid) : launch_eval_t<W, false>(dm, a, s, mid);
}

}  // namespace

cudaError_t launch_eval(const DevModel& dm, unsigned what, const EvalArgs& a, cudaStream_t s,
                        cudaEvent_t mid) {
  switch (what) {
    case OUT_ALL:
      return launch_eval_w<OUT_ALL>(dm, a, s, mid);
    case OUT_OBJ:
      return launch_eval_w<OUT_OBJ>(dm, a, s, mid);
    case OUT_GRAD:
      return launch_eval_w<OUT_GRAD>(dm, a, s, mid);
    case OUT_CONS:
      return launch_eval_w<OUT_CONS>(dm, a, s, mid);
    case OUT_JAC:
      return launch_eval_w<OUT_JAC>(dm, a, s, mid);
    case OUT_HESS:
      return launch_eval_w<OUT_HESS>(dm, a, s, mid);
    default:
      return cudaErrorInvalidValue;
  }
}

int launches_for(unsigned what) {
  switch (what) {
    case OUT_OBJ:
      return 1;
    case OUT_ALL:
    case OUT_GRAD:
    case OUT_CONS:
    case OUT_JAC:
    case OUT_HESS:
    case OUT_KKT:
      return 2;
    default:
      return -1;
  }
}

cudaError_t launch_assemble(const DevModel& dm, const EvalArgs& a, cudaStream_t s) {
  const Layout& L = dm.L;
  const bool reg = a.delta_w != 0.0 || a.delta_c != 0.0;
  const int nbb = ceil_div(L.nl, kBranchThreads);
  if (nbb > 0) {
    if (reg)
      k_asm_phase1<true><<<nbb, kBranchThreads, 0, s>>>(dm, a);
    else
      k_asm_phase1<false><<<nbb, kBranchThreads, 0, s>>>(dm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (reg) return launch_phase2<OUT_KKT, true, true>(dm, a, s, nbb > 0);
  return launch_phase2<OUT_KKT, false, true>(dm, a, s, nbb > 0);
}

cudaError_t launch_fp64_probe(double* out, int blocks, int iters, cudaStream_t s) {
  k_fp64_probe<<<blocks, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

}  // namespace acopf
