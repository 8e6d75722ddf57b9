// sm_103a FP64 kernels of libacopf.
//
// One call of the fused unit of work (objective, gradient, constraints,
// Jacobian, Lagrangian Hessian and the condensed KKT matrix of Sec. IV.C)
// is two launches:
//
//   phase 1  branch blocks, one thread per branch: patterns 3-9 fused around
//            one sincos per branch, which values, Jacobian, the merged
//            Hessian block and the branch's KKT contributions all share; the
//            branch writes the four arc rows of M_cond directly and leaves its
//            contributions to the bus rows in the slot scratch.
//            Bus-input blocks, one thread per bus: patterns 2, 10-15 (balance
//            rows summed over the bus's generators and arcs in a fixed order,
//            no atomics) and the bus's own diagonal terms of M_cond.
//            Generator blocks, one thread per generator: pattern 1, the
//            generator rows of M_cond, and the objective reduced in a fixed
//            order.  The bus and generator blocks depend on nothing the
//            branch blocks write; they run behind them and fill the tail.
//   phase 2  one thread per bus: the bus rows of M_cond, gathered from the
//            slot partials of its incident branches.
//
// Calls that do not assemble M_cond are the single phase-1 launch.  Phase 2
// is launched with programmatic dependent launch: its blocks load the
// structure they need while phase 1 drains and wait on the grid dependency
// before reading phase 1's partial sums.
//
// Every K entry has one owner thread that writes it (arc rows: branch
// threads; generator rows: generator threads; bus rows: bus threads), so the
// assembly is a gather: deterministic and free of atomics.  Row layouts are
// the ones model.cpp documents.
//
// FP64 throughput on this part is about 0.6 T FMA/s, far below what its
// memory bandwidth could feed, and an FP64 warp instruction occupies the
// SM's FP64 unit for the same time however many of its lanes are active.
// So the kernels minimise FP64 warp instructions: the four flows share two
// trigonometric brackets, the Hessians of the four flow rows merge into one
// weighted bracket, the condensation factor is a plain copy when
// delta_w = delta_c = 0, KKT entries of the form D (+-1) J are copies,
// stored negations and exact doublings use integer instructions, and the
// buses are processed in an order that gives every warp loops of one length.
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

__device__ __noinline__ double twice_slow(double x) { return x + x; }

// 2x.  For a normal x whose double does not overflow this adds one to the
// exponent field with an integer instruction (exact, and off the FP64 pipe);
// zeros, subnormals, infinities and NaNs take x + x.
__device__ __forceinline__ double twice(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned e = static_cast<unsigned>(b >> 52) & 0x7FFu;
  if (e - 1u < 0x7FDu) return __longlong_as_double(b + (1LL << 52));
  return twice_slow(x);
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

// Writes one arc row of M_cond from position k of `out`: the four bus
// entries, ng generator entries vg, the optional entry vx (the p_a column of
// row q_a), rk earlier-arc entries vr and the diagonal vd.
__device__ __forceinline__ void row_write(double* out, int k, bool f_lo, double e_vaf, double e_vat,
                                          double e_vmf, double e_vmt, int ng, double vg, bool hasx,
                                          double vx, int rk, double vr, double vd) {
  put4(out, k, f_lo, e_vaf, e_vat, e_vmf, e_vmt);
  k += 4;
  for (int e = 0; e < ng; ++e) out[k++] = vg;
  if (hasx) out[k++] = vx;
  for (int e = 0; e < rk; ++e) out[k++] = vr;
  out[k] = vd;
}

// Per-warp staging capacity for the arc rows (doubles): the branch blocks
// reuse the bus-input blocks' shared buffer, kBalCap double2 per warp.
constexpr int kRowStageCap = 2 * kBalCap;

// One arc row per lane, rows r0 of the warp's 32 branches being consecutive
// rows of the CSR (so the warp's rows tile one contiguous range of K).
// With a staging buffer (a full warp) the rows are assembled in shared
// memory and the range is written with coalesced stores; without one, or
// when the range exceeds the buffer, each lane stores its own row.
__device__ __forceinline__ void arc_row(double* __restrict__ K, double* stage, int r0, bool f_lo,
                                        double e_vaf, double e_vat, double e_vmf, double e_vmt,
                                        int ng, double vg, bool hasx, double vx, int rk, double vr,
                                        double vd) {
  if (stage != nullptr) {  // uniform over the warp: all 32 lanes are here
    const int len = 5 + ng + (hasx ? 1 : 0) + rk;
    const int base = __shfl_sync(0xffffffffu, r0, 0);
    const int n = __shfl_sync(0xffffffffu, r0 + len, 31) - base;
    if (n <= kRowStageCap) {
      row_write(stage, r0 - base, f_lo, e_vaf, e_vat, e_vmf, e_vmt, ng, vg, hasx, vx, rk, vr, vd);
      __syncwarp();
      for (int i = threadIdx.x & 31; i < n; i += 32) K[base + i] = stage[i];
      __syncwarp();
      return;
    }
  }
  row_write(K, r0, f_lo, e_vaf, e_vat, e_vmf, e_vmt, ng, vg, hasx, vx, rk, vr, vd);
}

// ===========================================================================
// Phase 1, fused path: branch thread.
// ===========================================================================
// SHUNT = false: every bus has Gs = Bs = 0, so the balance rows' vm
// coefficients 2 Gs vm and -2 Bs vm vanish from the arc rows of M_cond.
// `stage`: the warp's slice of the block's shared buffer when all 32 lanes
// of the warp run a branch (nullptr otherwise); used for the arc rows.
template <unsigned W, bool REG, bool SHUNT>
__device__ __forceinline__ void branch_fused(const DevModel& dm, const EvalArgs& a, int l,
                                             double* stage) {
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
    J[L.JPF + l] = 1.0;
    J[L.JQF + l] = 1.0;
    J[L.JPT + l] = 1.0;
    J[L.JQT + l] = 1.0;
    J[L.JANG + l] = 1.0;
    J[L.JANG + nl + l] = -1.0;
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
    const double tvf = twice(vm_f), tvt = twice(vm_t);

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
    const double jp_f = twice(p_f), jq_f = twice(q_f), jp_t = twice(p_t), jq_t = twice(q_t);
    if constexpr ((W & OUT_JAC) != 0) {
      // J row = [1, -dF/dth, dF/dth, -dF/dvm_f, -dF/dvm_t], entry k of every
      // branch's row stored contiguously (section + k nl + l).
      double* __restrict__ J = a.jvals;
      double* jp = J + L.JPF + l;
      jp[nl] = neg(th_pf);
      jp[2 * nl] = th_pf;
      jp[3 * nl] = neg(mf_pf);
      jp[4 * nl] = neg(mt_pf);
      jp = J + L.JQF + l;
      jp[nl] = neg(th_qf);
      jp[2 * nl] = th_qf;
      jp[3 * nl] = neg(mf_qf);
      jp[4 * nl] = nmt_qf;
      jp = J + L.JPT + l;
      jp[nl] = neg(th_pt);
      jp[2 * nl] = th_pt;
      jp[3 * nl] = neg(mf_pt);
      jp[4 * nl] = neg(mt_pt);
      jp = J + L.JQT + l;
      jp[nl] = VE_t;
      jp[2 * nl] = neg(VE_t);
      jp[3 * nl] = neg(mf_qt);
      jp[4 * nl] = neg(mt_qt);
      J[L.JSF + l] = jp_f;
      J[L.JSF + nl + l] = jq_f;
      J[L.JST + l] = jp_t;
      J[L.JST + nl + l] = jq_t;
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
      const double AF2 = twice(AF), AT2 = twice(AT);
      const double hs_f = twice(y_sf), hs_t = twice(y_st);
      if constexpr ((W & OUT_HESS) != 0) {
        double* __restrict__ H = a.hvals + L.HBLK + l;
        H[0] = VnTH;
        H[nl] = neg(VnTH);
        H[2 * nl] = VnTH;
        H[3 * nl] = neg(vtTP);
        H[4 * nl] = vtTP;
        H[5 * nl] = AF2;
        H[6 * nl] = neg(vfTP);
        H[7 * nl] = vfTP;
        H[8 * nl] = neg(nTH);
        H[9 * nl] = AT2;
        double* __restrict__ Ht = a.hvals + L.HTH + l;
        Ht[0] = hs_f;
        Ht[nl] = hs_f;
        Ht[2 * nl] = hs_t;
        Ht[3 * nl] = hs_t;
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
        double e_Pf = neg(B_pf), e_Qf = neg(B_qf), e_Pt = neg(C_pt), e_Qt = neg(C_qt);
        if constexpr (SHUNT) {
          const double jPv_f = ld(dm.Gs + f) * tvf, jQv_f = -(ld(dm.Bs + f) * tvf);
          const double jPv_t = ld(dm.Gs + t) * tvt, jQv_t = -(ld(dm.Bs + t) * tvt);
          e_Pf = fma(D_Pf, jPv_f, -B_pf);
          e_Qf = fma(D_Qf, jQv_f, -B_qf);
          e_Pt = fma(D_Pt, jPv_t, -C_pt);
          e_Qt = fma(D_Qt, jQv_t, -C_qt);
        }
        const double Dsp_f = D_sf * jp_f, Dsp_t = D_st * jp_t;
        double* __restrict__ K = a.kvals;
        const bool f_lo = f < t;
        // Row starts and, per bus, generator count and arc rank (row
        // p_a = [4 bus entries][generators][earlier arcs][diagonal],
        // row q_a = [4 bus entries][generators][p_a][earlier arcs][diagonal]).
        const int4 rs = ld(dm.brow + l);
        const uint32_t cnt = ld(dm.bcnt + l);
        int ngf, rkf, ngt, rkt;
        if (cnt != kCountsWide) {
          ngf = cnt & 0xFF;
          rkf = (cnt >> 8) & 0xFF;
          ngt = (cnt >> 16) & 0xFF;
          rkt = cnt >> 24;
        } else {
          const int* __restrict__ rp = dm.krowptr;
          ngf = ld(dm.gen_ptr + f + 1) - ld(dm.gen_ptr + f);
          ngt = ld(dm.gen_ptr + t + 1) - ld(dm.gen_ptr + t);
          rkf = ld(rp + iPf + 1) - rs.x - 5 - ngf;
          rkt = ld(rp + iPt + 1) - rs.z - 5 - ngt;
        }
        // row p_l (from arc, bus f)
        arc_row(K, stage, rs.x, f_lo, neg(A_pf), A_pf, e_Pf, neg(C_pf), ngf, neg(D_Pf), false, 0.0,
                rkf, D_Pf, sxw<REG>(ld(sx + iPf), dw) + hs_f + D_pf + fma(Dsp_f, jp_f, D_Pf));
        // row q_l
        arc_row(K, stage, rs.y, f_lo, neg(A_qf), A_qf, e_Qf, nC_qf, ngf, neg(D_Qf), true,
                Dsp_f * jq_f, rkf, D_Qf,
                sxw<REG>(ld(sx + iQf), dw) + hs_f + D_qf + fma(D_sf * jq_f, jq_f, D_Qf));
        // row p_{nl+l} (to arc, bus t)
        arc_row(K, stage, rs.z, f_lo, neg(A_pt), A_pt, neg(B_pt), e_Pt, ngt, neg(D_Pt), false, 0.0,
                rkt, D_Pt, sxw<REG>(ld(sx + iPt), dw) + hs_t + D_pt + fma(Dsp_t, jp_t, D_Pt));
        // row q_{nl+l}
        arc_row(K, stage, rs.w, f_lo, nA_qt, neg(nA_qt), neg(B_qt), e_Qt, ngt, neg(D_Qt), true,
                Dsp_t * jq_t, rkt, D_Qt,
                sxw<REG>(ld(sx + iQt), dw) + hs_t + D_qt + fma(D_st * jq_t, jq_t, D_Qt));
      }
    }
  }
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
    for (int e = 0; e < 5; ++e) j[q][e] = ld(J + base[q] + e * nl + l);
    D[q] = dcond<REG>(ld(ss + crow[q] + l), dw, dc);
  }
  const double ja0 = ld(J + L.JANG + l), ja1 = ld(J + L.JANG + nl + l);
  const double D_an = dcond<REG>(ld(ss + L.ANG + l), dw, dc);
  // block over local (va_f, va_t, vm_f, vm_t) = Jacobian columns 1..4
  double blk[10];
  const int pu[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
  const int pv[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};
#pragma unroll
  for (int e = 0; e < 10; ++e) {
    double acc = ld(Hv + L.HBLK + e * nl + l);
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
  const double js_f0 = ld(J + L.JSF + l), js_f1 = ld(J + L.JSF + nl + l);
  const double js_t0 = ld(J + L.JST + l), js_t1 = ld(J + L.JST + nl + l);
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
    const double hth = ld(Hv + L.HTH + q * nl + l);
    K[r1 - 1] =
        sxw<REG>(ld(sx + var), dw) + hth + fma(Dj0, j[q][0], fma(D_s * jsv, jsv, DBa * jBa));
  }
}

// ===========================================================================
// Generator threads (no dependency on the branch threads).
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
// Bus-input blocks (phase 1): everything about a bus that reads only the
// call's inputs.  Buses are taken in the processing order, so the 32 buses
// of a warp have equal arc and generator counts and run loops of equal
// length.  Leaves the bus's diagonal terms of M_cond for phase 2.
// ===========================================================================
// Warp w of bus block blk (of nblk) takes the buses at processing positions
// [32 g, 32 g + 32) with g = w * nblk + (nblk - 1 - blk): every block gets
// one warp from each quarter of the degree-sorted order, and block 0, which
// starts first, the heaviest ones.
__device__ __forceinline__ int bus_warp_base(int blk, int nblk) {
  const int w = threadIdx.x >> 5;
  return 32 * (w * nblk + (nblk - 1 - blk));
}

// One warp: the 32 buses at processing positions [pw0, pw0 + 32), with
// `buf` the warp's shared staging buffer (kBalCap double2).
template <unsigned W, bool REG, bool ARRAYS, bool SHUNT>
__device__ __forceinline__ void bus_input_warp(const DevModel& dm, const EvalArgs& a, int pw0,
                                               double2* buf) {
  const Layout& L = dm.L;
  const int p = pw0 + (threadIdx.x & 31);
  const bool active = p < L.nb;
  const int i = active ? ld(dm.porder + p) : 0;
  const double* __restrict__ x = a.x;
  if constexpr (!ARRAYS && (W & OUT_CONS) != 0) {
    // Balance rows.  The warp's buses own a contiguous range of the term list
    // (generators then arcs of each bus); lanes fetch the terms together with
    // all loads in flight at once, stage them in shared memory, and each lane
    // then sums its own bus's terms in list order.
    const int lane = threadIdx.x & 31;
    if (pw0 < L.nb) {
      const int pw1 = min(pw0 + 32, L.nb);
      const int e0 = ld(dm.pbal_ptr + pw0), e1 = ld(dm.pbal_ptr + pw1);
      const int ne = e1 - e0;
      const bool staged = ne <= kBalCap;
      if (staged) {
        constexpr int R = kBalCap / 32;
        int idx[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int k = lane + 32 * r;
          idx[r] = k < ne ? ld(dm.bal_idx + e0 + k) : -1;
        }
        double vp[R], vq[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (idx[r] >= 0) {
            const int off = idx[r] < L.P ? L.ng : 2 * L.nl;  // pg -> qg, p_a -> q_a
            vp[r] = ld(x + idx[r]);
            vq[r] = ld(x + idx[r] + off);
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (idx[r] >= 0) {
            const bool gen = idx[r] < L.P;  // generators enter with a minus sign
            buf[lane + 32 * r] = gen ? make_double2(neg(vp[r]), neg(vq[r])) : make_double2(vp[r], vq[r]);
          }
        }
        __syncwarp();
      }
      if (active) {
        double P = ld(dm.Pd + i), Q = ld(dm.Qd + i);
        if constexpr (SHUNT) {
          const double vm = ld(x + L.VM + i);
          P = fma(ld(dm.Gs + i) * vm, vm, P);
          Q = fma(-(ld(dm.Bs + i) * vm), vm, Q);
        }
        const int k0 = ld(dm.pbal_ptr + p) - e0, k1 = ld(dm.pbal_ptr + p + 1) - e0;
        for (int k = k0; k < k1; ++k) {
          double2 v;
          if (staged) {
            v = buf[k];
          } else {
            const int id = ld(dm.bal_idx + e0 + k);
            const bool gen = id < L.P;
            const double vp = ld(x + id), vq = ld(x + id + (gen ? L.ng : 2 * L.nl));
            v = gen ? make_double2(neg(vp), neg(vq)) : make_double2(vp, vq);
          }
          P += v.x;
          Q += v.y;
        }
        a.cons[L.PB + i] = P;
        a.cons[L.QB + i] = Q;
      }
    }
  }
  if (!active) return;
  const int r = ld(dm.ref_row + i);
  double d_va = 0.0, d_vm = 0.0;
  if constexpr (!ARRAYS) {
    double jPv = 0.0, jQv = 0.0, hb = 0.0;
    if constexpr (SHUNT) {
      const double vm = ld(x + L.VM + i);
      const double Gs = ld(dm.Gs + i), Bs = ld(dm.Bs + i);
      const double tv = vm + vm;
      jPv = Gs * tv;
      jQv = -(Bs * tv);
      if constexpr ((W & (OUT_HESS | OUT_KKT)) != 0)
        hb = fma(Gs + Gs, ld(a.y + L.PB + i), -((Bs + Bs) * ld(a.y + L.QB + i)));
    }
    if constexpr ((W & OUT_GRAD) != 0) {
      a.grad[L.VA + i] = 0.0;
      a.grad[L.VM + i] = 0.0;
    }
    if constexpr ((W & OUT_CONS) != 0) {
      if (r >= 0) a.cons[L.REF + r] = ld(x + L.VA + i);
    }
    if constexpr ((W & OUT_JAC) != 0) {
      if (r >= 0) a.jvals[L.JREF + r] = 1.0;
      a.jvals[L.JPBV + i] = jPv;
      a.jvals[L.JQBV + i] = jQv;
    }
    if constexpr ((W & OUT_HESS) != 0) a.hvals[L.HB + i] = hb;
    if constexpr ((W & OUT_KKT) != 0) {
      const double dw = a.delta_w, dc = a.delta_c;
      d_va = sxw<REG>(ld(a.sigma_x + L.VA + i), dw);
      if (r >= 0) d_va += dcond<REG>(ld(a.sigma_s + L.REF + r), dw, dc);
      d_vm = sxw<REG>(ld(a.sigma_x + L.VM + i), dw);
      if constexpr (SHUNT) {
        const double D_P = dcond<REG>(ld(a.sigma_s + L.PB + i), dw, dc);
        const double D_Q = dcond<REG>(ld(a.sigma_s + L.QB + i), dw, dc);
        d_vm += hb + fma(D_P * jPv, jPv, D_Q * jQv * jQv);
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
  if constexpr ((W & OUT_KKT) != 0) dm.bus_diag[p] = BusDiag{d_va, d_vm};
}

// Bus-input block blk of nblk: its four warps (bus_warp_base interleaving).
template <unsigned W, bool REG, bool ARRAYS, bool SHUNT>
__device__ __forceinline__ void bus_input_block(const DevModel& dm, const EvalArgs& a, int blk,
                                                int nblk, double* smem) {
  bus_input_warp<W, REG, ARRAYS, SHUNT>(
      dm, a, bus_warp_base(blk, nblk), reinterpret_cast<double2*>(smem) + (threadIdx.x >> 5) * kBalCap);
}

// Generator warp gw of ngw: generator rows, and the objective.  Each warp
// reduces its generators' cost terms in a fixed shuffle order; the last
// warp to arrive (an arrival counter, not an accumulation) adds the warp
// sums in warp order, so the result does not depend on scheduling.
template <unsigned W, bool REG, bool ARRAYS>
__device__ __forceinline__ void gen_warp(const DevModel& dm, const EvalArgs& a, int gw, int ngw) {
  const Layout& L = dm.L;
  const int lane = threadIdx.x & 31;
  const int g = gw * 32 + lane;
  if (g < L.ng) {
    if constexpr (ARRAYS)
      gen_from_arrays<REG>(dm, a, g);
    else
      gen_fused<W, REG>(dm, a, g);
  }
  if constexpr (!ARRAYS && (W & OUT_OBJ) != 0) {
    double v = 0.0;
    if (g < L.ng) {
      const double pg = ld(a.x + L.PG + g);
      v = fma(fma(ld(dm.c2 + g), pg, ld(dm.c1 + g)), pg, ld(dm.c0 + g));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int last = 0;
    if (lane == 0) {
      dm.obj_part[gw] = v;
      __threadfence();
      last = atomicAdd(dm.obj_ticket, 1u) == static_cast<unsigned int>(ngw - 1);
    }
    if (__shfl_sync(0xffffffffu, last, 0)) {
      __threadfence();
      double r = 0.0;
      for (int k = lane; k < ngw; k += 32) r += __ldcg(dm.obj_part + k);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
      if (lane == 0) {
        *a.f = r;
        *dm.obj_ticket = 0u;
      }
    }
  }
}

// Generator warps of ng generators (at least one when the objective is
// evaluated, so that a model without generators still writes f = 0).
__device__ __forceinline__ int gen_warps(int ng) { return ng > 0 ? (ng + 31) / 32 : 1; }

// Generator block gb: its four warps.
template <unsigned W, bool REG, bool ARRAYS>
__device__ __forceinline__ void gen_block(const DevModel& dm, const EvalArgs& a, int gb) {
  const int ngw = gen_warps(dm.L.ng);
  const int gw = gb * (kGenThreads / 32) + (threadIdx.x >> 5);
  if (gw < ngw) gen_warp<W, REG, ARRAYS>(dm, a, gw, ngw);
}

// Phase 1: block roles [0, nbb) branch blocks, [nbb, nbb + nbi) bus-input
// blocks, then ngb generator blocks.
template <unsigned W, bool REG, bool SHUNT>
__global__ void __launch_bounds__(kBranchThreads, 6) k_phase1(DevModel dm, EvalArgs a, int nbb,
                                                             int nbi, int ngb) {
  pdl_trigger();
  __shared__ __align__(16) double smem[(kBranchThreads / 32) * kBalCap * 2];  // read as double2
  const int b = blockIdx.x;
  if (b < nbb) {
    const int l = b * kBranchThreads + threadIdx.x;
    const bool full = (l | 31) < dm.L.nl;  // the whole warp has branches
    if (l < dm.L.nl)
      branch_fused<W, REG, SHUNT>(dm, a, l, full ? smem + (threadIdx.x >> 5) * kRowStageCap : nullptr);
  } else if (b < nbb + nbi) {
    bus_input_block<W, REG, false, SHUNT>(dm, a, b - nbb, nbi, smem);
  } else {
    gen_block<W, REG, false>(dm, a, b - nbb - nbi);
  }
}

// Phase 1 of the array-fed assembly (M_cond from given H and J values).
template <bool REG>
__global__ void __launch_bounds__(kBranchThreads) k_asm_phase1(DevModel dm, EvalArgs a, int nbb,
                                                              int nbi, int ngb) {
  pdl_trigger();
  __shared__ double smem[8];
  const int b = blockIdx.x;
  if (b < nbb) {
    const int l = b * kBranchThreads + threadIdx.x;
    if (l < dm.L.nl) branch_from_arrays<REG>(dm, a, l);
  } else if (b < nbb + nbi) {
    bus_input_block<OUT_KKT, REG, true, true>(dm, a, b - nbb, nbi, smem);
  } else {
    gen_block<OUT_KKT, REG, true>(dm, a, b - nbb - nbi);
  }
}

// ===========================================================================
// Phase 2: the bus rows of M_cond, gathered from the slot partials.
// ===========================================================================
// Row va_i = [va_j (j < i) ..., va_i]; row vm_i = [va_j / va_i ascending
// (nu + 1)][vm_j (j < i)][vm_i], or just [vm_i] for a bus without branches.
// The bus's slots run over its arcs by (other end, arc id), so parallel
// branches (equal other end) are adjacent and their entries are summed.
// Each lane runs one row chunk (DevModel::rchunk): about kRowChunk slots of
// one bus, all their loads in flight at once; it writes the chunk's
// off-diagonal entries from the row positions the chunk records and keeps
// its part of the three diagonal sums.  The bus's last chunk lane adds the
// chunks' parts in chunk order (shuffles within the warp) and writes the
// diagonal entries: a bus with many branches costs one round of loads.
// Warp w of block blk (of nblk) runs chunk warp w nblk + (nblk - 1 - blk),
// so every block gets one warp from each quarter of the degree order and
// block 0, which starts first, the heaviest.
__device__ __forceinline__ void bus_rows_block(const DevModel& dm, const EvalArgs& a, int blk,
                                               int nblk) {
  const Layout& L = dm.L;
  const int lane = threadIdx.x & 31;
  const int g = (threadIdx.x >> 5) * nblk + (nblk - 1 - blk);
  int4 A = make_int4(-1, 0, 0, 0), B = make_int4(0, 0, 0, 0);
  if (32 * g < L.nrc) {  // structure only: independent of phase 1
    A = ld(dm.rchunk + 2 * (32 * g + lane));
    B = ld(dm.rchunk + 2 * (32 * g + lane) + 1);
  }
  const int i = A.x;
  int bva = 0, eva = 0, bvm = 0, evm = 0;
  if (i >= 0) {
    const int* __restrict__ rp = dm.krowptr;
    bva = ld(rp + L.VA + i);
    eva = ld(rp + L.VA + i + 1);
    bvm = ld(rp + L.VM + i);
    evm = ld(rp + L.VM + i + 1);
  }
  pdl_wait();
  if (__all_sync(0xffffffffu, i < 0)) return;
  double* __restrict__ K = a.kvals;
  const int nlo = eva - bva - 1;  // distinct neighbours below i
  double aa = 0.0, ma = 0.0, mm = 0.0;
  if (i >= 0) {
    int pva = B.x, pvmva = B.y, pvmvm = B.z;
    double gv = 0.0, gx = 0.0, gw = 0.0;
    int cur = -1;
    constexpr int U = kRowChunk;  // slots fetched per round, all loads in flight together
    for (int k = A.z; k < A.w; k += U) {
      double2 q0[U], q1[U], q2[U];
      int jj[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k + u < A.w) {
          const double2* src = reinterpret_cast<const double2*>(dm.part_slot + k + u);
          q0[u] = __ldcg(src);
          q1[u] = __ldcg(src + 1);
          q2[u] = __ldcg(src + 2);
          jj[u] = ld(dm.slot_nbr + k + u);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (k + u < A.w) {
          // SlotPart {aa, ma | mm, mx | vv, ww}
          aa += q0[u].x;
          ma += q0[u].y;
          mm += q1[u].x;
          const int j = jj[u];
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
            gv = q2[u].x;
            gx = q1[u].y;
            gw = q2[u].y;
          } else {  // parallel branches between i and j
            gv += q2[u].x;
            gx += q1[u].y;
            gw += q2[u].y;
          }
        }
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
  }
  // the bus's chunks' diagonal parts, added in chunk order by its last chunk
  const int first = B.w & 31, nch = B.w >> 5;  // nch = 0 on an idle lane
  double ta = __shfl_sync(0xffffffffu, aa, first), tm = __shfl_sync(0xffffffffu, ma, first),
         tmm = __shfl_sync(0xffffffffu, mm, first);
  const int maxn = __reduce_max_sync(0xffffffffu, static_cast<unsigned>(nch));
  for (int q = 1; q < maxn; ++q) {
    const int src = first + min(q, max(nch - 1, 0));
    const double va = __shfl_sync(0xffffffffu, aa, src), vb = __shfl_sync(0xffffffffu, ma, src),
                 vc = __shfl_sync(0xffffffffu, mm, src);
    if (q < nch) {
      ta += va;
      tm += vb;
      tmm += vc;
    }
  }
  if (i >= 0 && lane == first + nch - 1) {
    const double2 dd = __ldcg(reinterpret_cast<const double2*>(dm.bus_diag + A.y));
    K[bva + nlo] = dd.x + ta;
    if (A.w > A.z) K[bvm + nlo] = tm;  // (vm_i, va_i) exists only when bus i has a branch
    K[evm - 1] = dd.y + tmm;
  }
}

__global__ void __launch_bounds__(kBusThreads, 5) k_bus_rows(DevModel dm, EvalArgs a) {
  bus_rows_block(dm, a, blockIdx.x, gridDim.x);
}

// ===========================================================================
// Batched evaluation: many instances in one launch per phase.  Work item
// {instance, role, block, blocks of that role in the instance}; roles 0
// branch, 1 bus input, 2 generators (phase 1); phase 2 items are bus-row
// blocks.  Each block runs items[b], items[b + gridDim.x], ... (one item per
// block when the grid covers the list; fewer, persistent blocks otherwise).
// Per item the instance's model view and arguments are copied to shared
// memory.  Phase 1 is compiled per code variant (regularised or not, shunts
// or not) and launched once per variant present, over the items of the
// instances of that variant: each instance runs the variant its own call
// takes, so its results are bit-identical to those of that call.
// ===========================================================================
template <typename Fn>
__device__ __forceinline__ void for_items(const DevModel* __restrict__ models,
                                          const EvalArgs* __restrict__ ios,
                                          const int4* __restrict__ items, int n, DevModel& sdm,
                                          EvalArgs& sa, Fn fn) {
  static_assert(sizeof(DevModel) % 8 == 0 && sizeof(EvalArgs) % 8 == 0, "copied as 8-byte words");
  constexpr int kM = sizeof(DevModel) / 8, kA = sizeof(EvalArgs) / 8;
  static_assert(kM <= 64 && 64 + kA <= kBranchThreads && 64 + kA <= kBusThreads, "copy layout");
  int cur = -1;
  for (int b = blockIdx.x; b < n; b += gridDim.x) {
    const int4 it = items[b];
    if (it.x != cur) {  // uniform over the block
      __syncthreads();  // every thread is done with the previous instance
      // Word-parallel copy: threads 0.. the model view, threads 64.. the arguments.
      const int t = threadIdx.x;
      if (t < kM) {
        reinterpret_cast<unsigned long long*>(&sdm)[t] =
            __ldg(reinterpret_cast<const unsigned long long*>(models + it.x) + t);
      } else if (t >= 64 && t < 64 + kA) {
        reinterpret_cast<unsigned long long*>(&sa)[t - 64] =
            __ldg(reinterpret_cast<const unsigned long long*>(ios + it.x) + (t - 64));
      }
      cur = it.x;
    }
    __syncthreads();
    fn(it);
  }
}

template <bool REG, bool SHUNT>
__global__ void __launch_bounds__(kBranchThreads, 6) k_batch_phase1(
    const DevModel* __restrict__ models, const EvalArgs* __restrict__ ios,
    const int4* __restrict__ items, int n) {
  // Raw storage (the views are trivially copied in; no constructor runs).
  __shared__ alignas(8) unsigned char sdm_raw[sizeof(DevModel)];
  __shared__ alignas(8) unsigned char sa_raw[sizeof(EvalArgs)];
  DevModel& sdm = *reinterpret_cast<DevModel*>(sdm_raw);
  EvalArgs& sa = *reinterpret_cast<EvalArgs*>(sa_raw);
  __shared__ __align__(16) double smem[(kBranchThreads / 32) * kBalCap * 2];  // read as double2
  pdl_trigger();
  for_items(models, ios, items, n, sdm, sa, [&](const int4& it) {
    if (it.y == 0) {
      const int l = it.z * kBranchThreads + threadIdx.x;
      const bool full = (l | 31) < sdm.L.nl;  // the whole warp has branches
      if (l < sdm.L.nl)
        branch_fused<OUT_ALL, REG, SHUNT>(sdm, sa, l,
                                          full ? smem + (threadIdx.x >> 5) * kRowStageCap : nullptr);
    } else if (it.y == 1) {
      bus_input_block<OUT_ALL, REG, false, SHUNT>(sdm, sa, it.z, it.w, smem);
    } else {
      gen_block<OUT_ALL, REG, false>(sdm, sa, it.z);
    }
  });
}

__global__ void __launch_bounds__(kBusThreads, 5) k_batch_bus_rows(
    const DevModel* __restrict__ models, const EvalArgs* __restrict__ ios,
    const int4* __restrict__ items, int n) {
  // Raw storage (the views are trivially copied in; no constructor runs).
  __shared__ alignas(8) unsigned char sdm_raw[sizeof(DevModel)];
  __shared__ alignas(8) unsigned char sa_raw[sizeof(EvalArgs)];
  DevModel& sdm = *reinterpret_cast<DevModel*>(sdm_raw);
  EvalArgs& sa = *reinterpret_cast<EvalArgs*>(sa_raw);
  for_items(models, ios, items, n, sdm, sa,
            [&](const int4& it) { bus_rows_block(sdm, sa, it.z, it.w); });
}

// FP64 throughput probe: 8 independent dependent chains per thread of one
// operation (0 fma, 1 add, 2 mul); the operands a, b are kernel arguments.
template <int OP>
__global__ void k_fp64_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    if constexpr (OP == 0) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    } else if constexpr (OP == 1) {
      x0 = x0 + b; x1 = x1 + b; x2 = x2 + b; x3 = x3 + b;
      x4 = x4 + b; x5 = x5 + b; x6 = x6 + b; x7 = x7 + b;
    } else {
      x0 = x0 * a; x1 = x1 * a; x2 = x2 * a; x3 = x3 * a;
      x4 = x4 * a; x5 = x5 * a; x6 = x6 * a; x7 = x7 * a;
    }
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

template <unsigned W, bool REG>
cudaError_t launch_eval_t(const DevModel& dm, const EvalArgs& a, cudaStream_t s,
                          cudaEvent_t mid) {
  const Layout& L = dm.L;
  constexpr bool kBranch = (W & (OUT_GRAD | OUT_CONS | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  constexpr bool kBus = kBranch;
  constexpr bool kGen = (W & (OUT_OBJ | OUT_GRAD | OUT_JAC | OUT_HESS | OUT_KKT)) != 0;
  const int nbb = kBranch ? ceil_div(L.nl, kBranchThreads) : 0;
  const int nbi = kBus ? ceil_div(L.nb, kBusThreads) : 0;
  int ngb = kGen ? ceil_div(L.ng, kGenThreads) : 0;
  if ((W & OUT_OBJ) != 0 && ngb == 0) ngb = 1;  // the objective of a model without generators
  const int blocks = nbb + nbi + ngb;
  if (blocks > 0) {
    if ((W & OUT_KKT) == 0 || dm.has_shunt)
      k_phase1<W, REG, true><<<blocks, kBranchThreads, 0, s>>>(dm, a, nbb, nbi, ngb);
    else
      k_phase1<W, REG, false><<<blocks, kBranchThreads, 0, s>>>(dm, a, nbb, nbi, ngb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if constexpr ((W & OUT_KKT) == 0) {
    return cudaSuccess;
  } else {
    if (mid) {
      cudaError_t e = cudaEventRecord(mid, s);
      if (e != cudaSuccess) return e;
    }
    return launch_ex(k_bus_rows, dim3(ceil_div(L.nrc, kBusThreads)), dim3(kBusThreads), 0, s,
                     blocks > 0 && !mid && dm.pdl, dm, a);
  }
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
    case OUT_ALL:
    case OUT_KKT:
      return 2;
    case OUT_OBJ:
    case OUT_GRAD:
    case OUT_CONS:
    case OUT_JAC:
    case OUT_HESS:
      return 1;
    default:
      return -1;
  }
}

cudaError_t launch_assemble(const DevModel& dm, const EvalArgs& a, cudaStream_t s) {
  const Layout& L = dm.L;
  const bool reg = a.delta_w != 0.0 || a.delta_c != 0.0;
  const int nbb = ceil_div(L.nl, kBranchThreads);
  const int nbi = ceil_div(L.nb, kBusThreads);
  const int ngb = ceil_div(L.ng, kGenThreads);
  const int blocks = nbb + nbi + ngb;
  if (reg)
    k_asm_phase1<true><<<blocks, kBranchThreads, 0, s>>>(dm, a, nbb, nbi, ngb);
  else
    k_asm_phase1<false><<<blocks, kBranchThreads, 0, s>>>(dm, a, nbb, nbi, ngb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_ex(k_bus_rows, dim3(ceil_div(L.nrc, kBusThreads)), dim3(kBusThreads), 0, s,
                   dm.pdl != 0, dm, a);
}

cudaError_t launch_batch(const DevModel* models, const EvalArgs* ios, const int4* items1,
                         const int64_t* seg1, int64_t cap1, const int4* items2, int n2, int grid2,
                         bool pdl, cudaStream_t s) {
  bool any1 = false;
  for (int c = 0; c < 4; ++c) {
    const int n = static_cast<int>(seg1[c + 1] - seg1[c]);
    if (n == 0) continue;
    const int grid = static_cast<int>(n < cap1 ? n : cap1);
    const int4* it = items1 + seg1[c];
    switch (c) {
      case 0: k_batch_phase1<false, false><<<grid, kBranchThreads, 0, s>>>(models, ios, it, n); break;
      case 1: k_batch_phase1<false, true><<<grid, kBranchThreads, 0, s>>>(models, ios, it, n); break;
      case 2: k_batch_phase1<true, false><<<grid, kBranchThreads, 0, s>>>(models, ios, it, n); break;
      default: k_batch_phase1<true, true><<<grid, kBranchThreads, 0, s>>>(models, ios, it, n); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    any1 = true;
  }
  if (n2 == 0) return cudaSuccess;
  return launch_ex(k_batch_bus_rows, dim3(grid2), dim3(kBusThreads), 0, s, pdl && any1, models,
                   ios, items2, n2);
}

cudaError_t batch_occupancy(int* phase1, int* phase2) {
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(phase1, k_batch_phase1<false, false>,
                                                    kBranchThreads, 0);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(phase2, k_batch_bus_rows, kBusThreads, 0);
}

cudaError_t launch_fp64_probe(int op, double* out, int blocks, int iters, cudaStream_t s) {
  if (op == 0)
    k_fp64_probe<0><<<blocks, 256, 0, s>>>(out, iters, 0.9999999, 1e-7);
  else if (op == 1)
    k_fp64_probe<1><<<blocks, 256, 0, s>>>(out, iters, 0.9999999, 1e-7);
  else
    k_fp64_probe<2><<<blocks, 256, 0, s>>>(out, iters, 0.9999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace acopf
