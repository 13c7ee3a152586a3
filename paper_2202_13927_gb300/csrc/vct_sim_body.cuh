// vct_sim_body.cuh -- the closed-loop Monte Carlo kernel (Sec. III, Eq. 1-3).
// Included by the vct_sim_*.cu files, which instantiate its variants.
//
// One thread integrates PPT patients of one scenario over the requested
// period range, keeping every state, controller variable and running
// indicator in registers.  Per control period t_k (Sec. III-B):
//   1. bin G(t_k) = Q1 / (V_G BW) into the five ranges of Sec. IV-A (edges
//      54, 70, 180, 250 mg/dL = those / 18 mmol/L, lower-closed) and update
//      the running indicators (Sec. III-C);
//   2. CGM sample y_k = Gsc(t_k) + v_k (Eq. 1d);
//   3. PID on y_k and the announced meal bolus (Eq. 3);
//   4. m Euler-Maruyama steps of the Hovorka 2004 model with u_k and d_k held
//      (Eq. 1b, Eq. 2), additive noise on Q1, Q1 clamped at zero.
// With GLU the two s.c. glucagon compartments Z1, Z2 (Sec. IV-B) join the
// state, EGP gains EGP0 s_gg Z2, and a scenario with glucagon mode switches
// the controller to glucagon microboli with no insulin while y_k is below its
// threshold (Sec. IV-C).  A scenario without glucagon mode runs bit-identically
// in the GLU and the plain variants (its Z1, Z2 stay exactly zero).
// The Euler step x + h f(x) is evaluated in the factorised form x a + b with
// per-patient coefficients a = 1 - h/tau etc. precomputed once; every product
// of the model is still evaluated at x_n.  Along the linear chains of the
// model (D1 -> D2, S1 -> S2 -> I -> x1, x2, x3, G -> Gsc) each variable is
// held divided by its input coefficient (D2 / (h/tau_D), I / (c_I h/tau_S),
// ...), an exact change of variables of the same Euler recursion that makes
// every chain update a single fma; the coefficients of the variables' uses
// carry the scale instead.
//
// Real = double: the plain FP64 form.  Real = float: the fast form -- FP32
// state and arithmetic, FP32 Box-Muller from the same Philox words, FP64 for
// the initial state (computed by the population kernel) and for the
// long-horizon sums, which take FP32 partials folded into FP64 once per day.
// The FP64 sums and other data touched at most once per day live in shared
// memory, the rest in registers.
//
// Work items are (scenario, block of B*PPT patients), enumerated longest
// horizon first; with `persistent` a grid of resident CTAs pulls items from an
// atomic counter, otherwise one CTA runs one item.
#pragma once
#include <cuda_fp16.h>

#include <type_traits>

#include "vct_internal.cuh"
#include "vct_rng.cuh"

namespace vct {
namespace {

// BG range edges in mmol/L (mg/dL / 18)
constexpr double kEdge0 = 54.0 / 18.0, kEdge1 = 70.0 / 18.0, kEdge2 = 180.0 / 18.0,
                 kEdge3 = 250.0 / 18.0;
constexpr int kMaxBlock = 256;

// Per-patient data read or written at most once per day (shared memory).
struct Cold {
  double S1, S2, B, BOL;  // long-horizon sums: G - G_sp, (G - G_sp)^2, basal rate, bolus U
  float tdd500;           // bolus units per gram of carbohydrate (FP32 path)
  double tdd500d;         // same in FP64
  uint32_t pid, status;
  uint32_t valid;
  double bw;              // body weight (protocol meals are per kg)
  double GG;              // glucagon delivered, ug
  double BOLd;            // bolus of the current day, U (daily doses)
};

template <typename Real>
struct Hot {
  // factorised Euler coefficients (chain variables held scaled, see state_scales)
  Real aD, gD, aS, aI, a1, a2, a3, e1, e2, e3, f45, q45, q9, q0, hk12, omhk12, hAG, aC, cC,
      inv_vg_bw;
  // glucagon compartments (GLU variants), EGP effect h EGP0 s_gg Z2, day partial
  Real Z1, Z2, cGg, ggd;
  // controller
  Real ubh, kp, ki, kd;
  // state
  Real x[VCT_NSTATE];
  Real integ, y_prev;
  // running indicators since the last fold
  Real s1, s2, bas, gmin, gmax;
  uint32_t cge0, cge1, cge2, cge3, hypo, clamps, n;
  bool prev_low, alive;
  // Philox words after round 1 for (patient, stream)
  uint32_t w0, w1;
};

// Smallest scale of a chain variable: a link whose input coefficient is zero
// (a zero rate or sensitivity) keeps a tiny one, so that its variable stays
// finite; its input then differs from zero by that scale times the upstream
// variable, far below rounding for any physiological value.
constexpr double kMinScale = 1e-30;

// Scale of each state in the kernel's representation x_j / s_j (1 for the
// states that are not chain links): D2 by h/tau_D, S2 by h/tau_S, I by
// c_I h/tau_S with c_I = h/(tau_S V_I BW), x_i by b_i s_I with b_i = h k_ai S_i,
// Gsc by c_C = h/(tau_CGM V_G BW) (Gsc as a multiple of Q1).
__device__ __forceinline__ void state_scales(const double *p, double h, double s[VCT_NSTATE]) {
  const double bw = p[VCT_P_BW];
  const double hD = h / p[VCT_P_TAUD], hS = h / p[VCT_P_TAUS];
  const double cI = h / (p[VCT_P_TAUS] * p[VCT_P_VI] * bw);
  const double sI = fmax(cI * hS, kMinScale);
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) s[j] = 1.0;
  s[1] = fmax(hD, kMinScale);
  s[3] = fmax(hS, kMinScale);
  s[4] = sI;
  s[5] = fmax(h * p[VCT_P_KA1] * p[VCT_P_SIT] * sI, kMinScale);
  s[6] = fmax(h * p[VCT_P_KA2] * p[VCT_P_SID] * sI, kMinScale);
  s[7] = fmax(h * p[VCT_P_KA3] * p[VCT_P_SIE] * sI, kMinScale);
  s[10] = fmax(h / p[VCT_P_TAUCGM] / (p[VCT_P_VG] * bw), kMinScale);
}

template <typename Real>
__device__ __forceinline__ void load_patient(Hot<Real> &P, Cold &C, const SimArgs &a,
                                             const ScenDev &sc, uint32_t i, bool valid, double h) {
  const PopDev &pop = a.pop;
  const uint32_t ii = valid ? i : 0u;
  const int64_t np = pop.n_pad;
  double p[VCT_NROW];
#pragma unroll
  for (int j = 0; j < VCT_NROW; ++j) p[j] = pop.rows[j * np + ii];
  const double ub = pop.ub[ii];
  C.valid = valid;
  C.status = valid ? (pop.status[ii] & VCT_PATIENT_REJECTED) : VCT_PATIENT_REJECTED;
  C.pid = (uint32_t)(pop.first + ii);

  const double bw = p[VCT_P_BW];
  const double vgbw = p[VCT_P_VG] * bw;
  double sc_x[VCT_NSTATE];
  state_scales(p, h, sc_x);
  C.bw = bw;
  const double hD = h / p[VCT_P_TAUD];
  P.aD = (Real)(1.0 - hD);
  P.gD = (Real)(hD * sc_x[1]);  // U_G h = (h/tau_D) D2 = (h/tau_D) s_D2 (D2 / s_D2)
  P.aS = (Real)(1.0 - h / p[VCT_P_TAUS]);
  P.aI = (Real)(1.0 - h * p[VCT_P_KE]);
  P.a1 = (Real)(1.0 - h * p[VCT_P_KA1]);
  P.a2 = (Real)(1.0 - h * p[VCT_P_KA2]);
  P.a3 = (Real)(1.0 - h * p[VCT_P_KA3]);
  P.e1 = (Real)(h * sc_x[5]);                       // h x1
  P.e2 = (Real)(h * sc_x[6]);                       // h x2
  P.e3 = (Real)(h * p[VCT_P_EGP0] * bw * sc_x[7]);  // h EGP0 BW x3
  // h F01c = h F01 BW min(1, G/4.5) = f45 min(Q1, q45), q45 = 4.5 V_G BW;
  // h F_R = 0.003 h max(Q1 - q9, 0) = 0.003 h max(Q1, q9) - 0.003 h q9, q9 = 9 V_G BW,
  // whose constant joins h EGP0 BW in q0, the constant part of the Q1 step
  P.q45 = (Real)(4.5 * vgbw);
  P.f45 = (Real)(h * p[VCT_P_F01] * bw / (4.5 * vgbw));
  P.q9 = (Real)(9.0 * vgbw);
  P.q0 = (Real)(h * p[VCT_P_EGP0] * bw + h * 0.003 * 9.0 * vgbw);
  P.hk12 = (Real)(h * p[VCT_P_K12]);
  P.omhk12 = (Real)(1.0 - h * p[VCT_P_K12]);
  P.hAG = (Real)(h * p[VCT_P_AG]);
  P.aC = (Real)(1.0 - h / p[VCT_P_TAUCGM]);
  P.cC = (Real)sc_x[10];  // Gsc = c_C (Gsc / c_C), the CGM lag's input gain on Q1
  P.inv_vg_bw = (Real)(1.0 / vgbw);
  // Z2 is held divided by h/tau_gg (its input coefficient) when the model is on
  const double hG = pop.tau_gg > 0.0 ? h / pop.tau_gg : 0.0;
  P.cGg = (Real)(h * p[VCT_P_EGP0] * pop.s_gg * (hG > 0.0 ? hG : 1.0));
  P.Z1 = P.Z2 = P.ggd = Real(0);
  C.GG = 0.0;
  C.BOLd = 0.0;

  const double ubh = sc.basal_scale * ub;
  const double kpn = sc.kp_per_ub * ubh;
  P.ubh = (Real)ubh;
  P.kp = (Real)(sc.kp_mult * kpn);
  P.ki = (Real)(sc.ki_mult * kpn / sc.ti);
  P.kd = (Real)(sc.kd_mult * kpn * sc.td);
  C.tdd500d = 2.0 * 24.0 * (ubh * 60.0 / 1000.0) / 500.0;
  C.tdd500 = (float)C.tdd500d;

  bool finite = true;
#pragma unroll
  for (int j = 0; j < VCT_NROW; ++j) finite = finite && isfinite(p[j]);
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) {
    const double v = pop.x0[j * np + ii];
    finite = finite && isfinite(v);
    P.x[j] = (Real)(v / sc_x[j]);
  }
  P.integ = Real(0);
  P.y_prev = Real(0);
  P.s1 = P.s2 = P.bas = Real(0);
  C.S1 = C.S2 = C.B = C.BOL = 0.0;
  P.gmin = Real(INFINITY);
  P.gmax = Real(-INFINITY);
  P.cge0 = P.cge1 = P.cge2 = P.cge3 = P.hypo = P.clamps = P.n = 0;
  P.prev_low = false;
  P.alive = finite && C.status == 0;
  if (!finite && C.status == 0) C.status = VCT_PATIENT_NONFINITE;
}

template <typename Real, bool GLU>
__device__ __forceinline__ void load_state(Hot<Real> &P, Cold &C, const SimArgs &a, int64_t slot) {
  const int64_t S = a.state_stride;
  const double *d = a.state_in_d;
  const uint32_t *w = a.state_in_w;
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) P.x[j] = (Real)d[j * S + slot];
  P.integ = (Real)d[11 * S + slot];
  P.y_prev = (Real)d[12 * S + slot];
  P.s1 = (Real)d[13 * S + slot];
  P.s2 = (Real)d[14 * S + slot];
  P.bas = (Real)d[15 * S + slot];
  C.S1 = d[16 * S + slot];
  C.S2 = d[17 * S + slot];
  C.B = d[18 * S + slot];
  C.BOL = d[19 * S + slot];
  P.gmin = (Real)d[20 * S + slot];
  P.gmax = (Real)d[21 * S + slot];
  P.cge0 = w[0 * S + slot];
  P.cge1 = w[1 * S + slot];
  P.cge2 = w[2 * S + slot];
  P.cge3 = w[3 * S + slot];
  P.hypo = w[4 * S + slot];
  P.clamps = w[5 * S + slot];
  P.n = w[6 * S + slot];
  const uint32_t f = w[7 * S + slot];
  P.prev_low = (f & 1u) != 0;
  P.alive = (f & 2u) != 0;
  C.status = f >> 8;
  if (GLU) {
    P.Z1 = (Real)d[22 * S + slot];
    P.Z2 = (Real)d[23 * S + slot];
    P.ggd = (Real)d[24 * S + slot];
  }
  C.GG = d[25 * S + slot];
  C.BOLd = d[26 * S + slot];
}

template <typename Real, bool GLU>
__device__ __forceinline__ void store_state(const Hot<Real> &P, const Cold &C, const SimArgs &a,
                                            int64_t slot) {
  const int64_t S = a.state_stride;
  double *d = a.state_out_d;
  uint32_t *w = a.state_out_w;
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) d[j * S + slot] = (double)P.x[j];
  d[11 * S + slot] = (double)P.integ;
  d[12 * S + slot] = (double)P.y_prev;
  d[13 * S + slot] = (double)P.s1;
  d[14 * S + slot] = (double)P.s2;
  d[15 * S + slot] = (double)P.bas;
  d[16 * S + slot] = C.S1;
  d[17 * S + slot] = C.S2;
  d[18 * S + slot] = C.B;
  d[19 * S + slot] = C.BOL;
  d[20 * S + slot] = (double)P.gmin;
  d[21 * S + slot] = (double)P.gmax;
  w[0 * S + slot] = P.cge0;
  w[1 * S + slot] = P.cge1;
  w[2 * S + slot] = P.cge2;
  w[3 * S + slot] = P.cge3;
  w[4 * S + slot] = P.hypo;
  w[5 * S + slot] = P.clamps;
  w[6 * S + slot] = P.n;
  w[7 * S + slot] = (P.prev_low ? 1u : 0u) | (P.alive ? 2u : 0u) | (C.status << 8);
  d[22 * S + slot] = GLU ? (double)P.Z1 : 0.0;
  d[23 * S + slot] = GLU ? (double)P.Z2 : 0.0;
  d[24 * S + slot] = GLU ? (double)P.ggd : 0.0;
  d[25 * S + slot] = C.GG;
  d[26 * S + slot] = C.BOLd;
}

template <typename Real, bool GLU>
__device__ __forceinline__ void fold(Hot<Real> &P, Cold &C) {
  C.S1 += (double)P.s1;
  C.S2 += (double)P.s2;
  C.B += (double)P.bas;
  if (GLU) C.GG += (double)P.ggd;
  P.s1 = P.s2 = P.bas = P.ggd = Real(0);
}

// The per-period test for a non-finite state.  FP64: exact (some state
// infinite or NaN, the oracle's test), on the exponent fields in integer
// arithmetic, off the FP64 pipe that bounds that form.  FP32: the sum of the
// states is not finite -- true whenever a state is infinite or NaN, and
// otherwise only for finite states whose sum overflows (above 1.7e38, a
// patient already diverging); the exact test costs the issue-bound FP32
// kernel 0.85 %.
template <typename Real, bool GLU>
__device__ __forceinline__ bool state_nonfinite(const Hot<Real> &p) {
  if constexpr (sizeof(Real) == 8) {
    uint32_t e = 0u;
#pragma unroll
    for (int j = 0; j < VCT_NSTATE; ++j) e = max(e, (uint32_t)__double2hiint((double)p.x[j]) & 0x7FF00000u);
    if (GLU) {
      e = max(e, (uint32_t)__double2hiint((double)p.Z1) & 0x7FF00000u);
      e = max(e, (uint32_t)__double2hiint((double)p.Z2) & 0x7FF00000u);
    }
    return e == 0x7FF00000u;
  } else {
    Real sum = p.x[0];
#pragma unroll
    for (int j = 1; j < VCT_NSTATE; ++j) sum += p.x[j];
    if (GLU) sum += p.Z1 + p.Z2;
    return !isfinite(sum);
  }
}

// Daily doses (Fig. 5): at the end of a day, one count per dose to the bins of
// the day's basal (U), bolus (U) and glucagon (ug), if the patient is alive.
template <typename Real>
__device__ __forceinline__ void bin_day(const Hot<Real> &P, Cold &C, double ts, uint32_t *dose) {
  if (P.alive) {
    const double v[3] = {(double)P.bas * ts / 1000.0, C.BOLd, (double)P.ggd};
    const double w[3] = {VCT_DOSE_BASAL_BIN, VCT_DOSE_BOLUS_BIN, VCT_DOSE_GLUCAGON_BIN};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double b = floor(v[j] / w[j]);  // doses are >= 0
      atomicAdd(&dose[j * VCT_DOSE_BINS + (b < (double)(VCT_DOSE_BINS - 1) ? (int)b : VCT_DOSE_BINS - 1)], 1u);
    }
  }
  C.BOLd = 0.0;
}

// Step 1: indicators on G(t_k).
template <typename Real>
__device__ __forceinline__ void measure(Hot<Real> &P, Real g, Real gsp, uint32_t *hist) {
  if (!P.alive) return;
  if (hist) atomicAdd(&hist[min((int)(g * Real(10)), VCT_BG_BINS - 1)], 1u);  // g >= 0: truncation = floor
  P.cge0 += g >= Real(kEdge0);
  P.cge1 += g >= Real(kEdge1);
  P.cge2 += g >= Real(kEdge2);
  P.cge3 += g >= Real(kEdge3);
  const bool low = g < Real(kEdge1);
  P.hypo += (low && !P.prev_low);
  P.prev_low = low;
  const Real dev = g - gsp;
  P.s1 += dev;
  P.s2 = fma(dev, dev, P.s2);
  P.gmin = fmin(P.gmin, g);
  P.gmax = fmax(P.gmax, g);
  P.n += 1;
}

// The glucagon compartments' Euler coefficient, the same for every patient:
// aG = 1 - h/tau_gg (1 when the model is off; Z1, Z2 then stay zero).  Z2 is
// held divided by h/tau_gg, so its input coefficient is 1.
template <typename Real>
struct GgCoef {
  Real aG;
};

// One Euler-Maruyama step of the Hovorka model; hu = h u_k, bD = h A_G d_k,
// hR = 0.003 h is uniform; nz = sigma sqrt(h) z + q0 carries the step's noise
// and the constant part of the Q1 step; hg = h u_gg (GLU).
template <typename Real, bool GLU>
__device__ __forceinline__ void em_step(Hot<Real> &P, Real hu, Real bD, Real hR, Real nz, Real hg,
                                        GgCoef<Real> gc) {
  Real *x = P.x;
  const Real D1 = x[0], D2 = x[1], S1 = x[2], S2 = x[3], I = x[4];
  const Real X1 = x[5], X2 = x[6], X3 = x[7], Q1 = x[8], Q2 = x[9], GSC = x[10];
  // (D2, S2, I, X1-X3, GSC: the scaled chain variables, each update one fma)
  // gut: D1' = A_G d - D1/tau_D, D2' = (D1 - D2)/tau_D, U_G = D2/tau_D
  x[0] = fma(D1, P.aD, bD);
  x[1] = fma(D2, P.aD, D1);
  // s.c. insulin and plasma insulin
  x[2] = fma(S1, P.aS, hu);
  x[3] = fma(S2, P.aS, S1);
  x[4] = fma(I, P.aI, S2);
  // insulin action
  x[5] = fma(X1, P.a1, I);
  x[6] = fma(X2, P.a2, I);
  x[7] = fma(X3, P.a3, I);
  // glucose: Q1' = -F01c - F_R - x1 Q1 + k12 Q2 + U_G + EGP0 BW (1 - x3), with
  // F01c = F01 BW min(1, G/4.5) and F_R = 0.003 (G - 9) V_G BW above 9 mmol/L
  // (the terms free of Q1 are summed off Q1's dependency chain)
  const Real hx1 = P.e1 * X1;
  Real c = fma(P.hk12, Q2, nz);
  c = fma(D2, P.gD, c);
  c = fma(-P.e3, X3, c);
  if (GLU) c = fma(P.cGg, P.Z2, c);
  Real q = fma(-P.f45, fmin(Q1, P.q45), c);
  const Real r = fma(-hx1, Q1, Q1);
  q = fma(-hR, fmax(Q1, P.q9), q);
  q = q + r;
  // Q2' = x1 Q1 - (k12 + x2) Q2
  x[9] = fma(Q2, fma(-P.e2, X2, P.omhk12), hx1 * Q1);
  // CGM lag: Gsc' = (G - Gsc)/tau_CGM
  x[10] = fma(GSC, P.aC, Q1);
  const bool neg = q < Real(0);
  x[8] = neg ? Real(0) : q;
  P.clamps += neg;
  if (GLU) {
    // s.c. glucagon: Z1' = u_gg - Z1/tau_gg, Z2' = (Z1 - Z2)/tau_gg
    const Real Z1 = P.Z1;
    P.Z1 = fma(Z1, gc.aG, hg);
    P.Z2 = fma(P.Z2, gc.aG, Z1);  // Z2 / (h/tau_gg)
  }
}

template <typename Real>
__device__ __forceinline__ void store_trace(const SimArgs &a, int64_t off, Real v) {
  switch (a.trace_dtype) {
    case VCT_TRACE_F16: ((__half *)a.trace)[off] = __float2half_rn((float)v); break;
    case VCT_TRACE_F32: ((float *)a.trace)[off] = (float)v; break;
    case VCT_TRACE_F64: ((double *)a.trace)[off] = (double)v; break;
    default: break;
  }
}

struct Smem {
  int item;
  int n_slots;
  int meal_kd[VCT_MAX_MEALS];
  int meal_cnt[VCT_MAX_MEALS];
  int meal_j[VCT_MAX_MEALS * VCT_MAX_MEALS];
};

// The end of a work item for one patient: the resumable state if asked, and,
// when the run reached the horizon, its indicator record.
template <typename Real, bool GLU>
__device__ __forceinline__ void finish_patient(const SimArgs &a, Hot<Real> &p, Cold &C, int64_t gslot,
                                               bool stopped_early) {
  const PopDev &pop = a.pop;
  {
    if (!C.valid) return;
    if (a.state_out_d) store_state<Real, GLU>(p, C, a, gslot);
    if (stopped_early) return;  // state only
    fold<Real, GLU>(p, C);
    vct_patient_stats o;
    const uint32_t n = p.n;
    o.tir[0] = n - p.cge0;
    o.tir[1] = p.cge0 - p.cge1;
    o.tir[2] = p.cge1 - p.cge2;
    o.tir[3] = p.cge2 - p.cge3;
    o.tir[4] = p.cge3;
    o.hypo_episodes = p.hypo;
    o.q1_clamps = p.clamps;
    o.status = C.status;
    o.n_samples = n;
    o.reserved = 0;
    if (n > 0) {
      const double md = C.S1 / (double)n;
      o.g_mean = pop.g_sp + md;
      o.g_var = fmax(C.S2 / (double)n - md * md, 0.0);
      o.g_min = (double)p.gmin;
      o.g_max = (double)p.gmax;
    } else {
      o.g_mean = o.g_var = o.g_min = o.g_max = 0.0;
    }
    o.basal_u = C.B * a.ts / 1000.0;
    o.bolus_u = C.BOL;
    o.glucagon_ug = C.GG;
    a.out[gslot] = o;
  }
}

template <typename Real, int MS, int PPT, bool GLU, int LEAN>
__device__ __forceinline__ void run_item(const SimArgs &a, int s, int b, const Smem &sm,
                                         Cold *cold, uint32_t *hist, uint32_t *dose) {
  const ScenDev &sc = a.scen[s];
  const int B = blockDim.x;
  const PopDev &pop = a.pop;
  const int m = MS > 0 ? MS : a.m;
  const double hd = a.ts / (double)m;
  const Real h = (Real)hd, hR = (Real)(hd * 0.003);
  const Real sig = (Real)(pop.sigma_q1 * sqrt(hd));
  const Real gsp = (Real)pop.g_sp;
  const Real cgm_sd = (Real)pop.cgm_sd;
  const Real ts = (Real)a.ts;
  const Real inv_ts = (Real)(1.0 / a.ts);
  const Real c_mmol = (Real)(1000.0 / 180.16 / a.ts);  // g -> mmol/min over one period
  const Real bolus_rate = (Real)(1000.0 / a.ts);        // U -> mU/min over one period
  // glucagon mode (GLU variants): threshold, microbolus gain and cap, and h / Ts
  // (a microbolus of gg ug over one period enters Z1 as h gg / Ts per step)
  const bool glu_on = GLU && sc.glucagon != 0;
  const Real gg_thr = (Real)sc.gg_thr, gg_gain = (Real)sc.gg_gain, gg_max = (Real)sc.gg_max;
  const Real h_per_ts = (Real)(hd / a.ts);
  const bool gg_model = pop.tau_gg > 0.0;  // else Z1, Z2 stay zero (no scenario uses them)
  const GgCoef<Real> gc{(Real)(gg_model ? 1.0 - hd / pop.tau_gg : 1.0)};
  const Real imax = (Real)sc.i_max;
  const Real meal_mean = (Real)sc.meal_mean, meal_sd = (Real)sc.meal_sd;
  const bool bolus_on = sc.bolus != 0;
  const uint32_t per_day = (uint32_t)llround(1440.0 / a.ts);
  const uint32_t horizon = (uint32_t)sc.horizon;
  const uint32_t k_begin = (uint32_t)a.period_begin;
  const uint32_t k_end = (a.period_end > 0 && a.period_end < sc.horizon) ? (uint32_t)a.period_end : horizon;
  const bool noise = pop.sigma_q1 != 0.0;
  const uint64_t seed = pop.key;  // a kernel parameter: uniform, round keys stay off the data path
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
  const uint32_t *rk = pop.rk;  // round keys in the kernel parameter: constant operands
  const uint32_t stream = sc.stream_id;
  const uint32_t n_meals = (uint32_t)sc.n_meals;
  const uint32_t base = (uint32_t)b * (uint32_t)(B * PPT) + threadIdx.x;
  const bool tracing = LEAN != 1 && a.trace != nullptr;
  const uint32_t n_trace = (uint32_t)a.trace_patients;
  const bool trace_bg = a.trace_kind == VCT_TRACE_BG;

  Hot<Real> P[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const uint32_t i = base + (uint32_t)(q * B);
    const bool valid = (int64_t)i < pop.n;
    Cold &C = cold[q * B + threadIdx.x];
    load_patient(P[q], C, a, sc, i, valid, hd);
    if (a.state_in_d && valid) load_state<Real, GLU>(P[q], C, a, (int64_t)s * pop.n + i);
    const uint32_t pid = C.pid;
    P[q].w0 = __umulhi(kPhiloxM1, stream) ^ pid ^ key0;
    P[q].w1 = kPhiloxM1 * stream;
  }

  uint32_t day = k_begin / per_day;
  uint32_t kd = k_begin % per_day;
  int slot = 0;  // next meal slot within the day
  while (slot < sm.n_slots && (uint32_t)sm.meal_kd[slot] < kd) ++slot;
  // protocol (Sec. II-B): the day's plan, the next meal's index, period and size
  const bool use_plan = !LEAN && sc.plan != nullptr;
  const vct_day_plan *dp = use_plan ? sc.plan + (day % (uint32_t)sc.plan_days) : nullptr;
  int pm = 0;
  uint32_t plan_kd = 0xFFFFFFFFu;
  float plan_gkg = 0.0f;
  const Real meal_cv = (Real)sc.meal_cv;
  const double ts_d = a.ts;
  auto next_plan_meal = [&]() {
    plan_kd = 0xFFFFFFFFu;
    if (pm < dp->n_meals) {
      plan_kd = (uint32_t)llround((double)dp->minute[pm] / ts_d);
      plan_gkg = dp->g_per_kg[pm];
    }
  };
  if (use_plan) {
    next_plan_meal();
    while (plan_kd < kd) {
      ++pm;
      next_plan_meal();
    }
  }

  // The first Philox call of period k + 1 is drawn during period k's Euler
  // steps (software pipelining: it depends on the period index only).
  Words4 wnext[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q)
    wnext[q] = PhiloxLaneRk{P[q].w0, P[q].w1, rk}.call(__umulhi(kPhiloxM0, k_begin),
                                                      kPhiloxM0 * k_begin, kTagSde);

  // within-day period of the next meal (0xFFFFFFFF: no more meals today)
  uint32_t meal_kd = use_plan ? plan_kd : (slot < sm.n_slots ? (uint32_t)sm.meal_kd[slot] : 0xFFFFFFFFu);

  uint32_t k = k_begin;
  // One control period, the meal code compiled in only where a meal falls
  // (MEAL): the periods between meals run without it.
  auto period = [&](auto meal_tag) {
    constexpr bool MEAL = decltype(meal_tag)::value;
      const uint32_t c0_hi = __umulhi(kPhiloxM0, k), c0_lo = kPhiloxM0 * k;
      Real hu[PPT], bD[PPT], hg[PPT];
      Real n0[PPT], n1[PPT], n2[PPT];  // scaled normals 1, 2, 3 of the period (Euler steps 0-2)
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        Hot<Real> &p = P[q];
        const Real g = p.x[8] * p.inv_vg_bw;
        measure(p, g, gsp, hist);
        // the period's first Philox call: normal 0 is the CGM noise, 1-3 drive steps 0-2
        const Words4 wc = wnext[q];
        Real zc, z1;
        box_muller<Real>(wc.a, wc.b, zc, z1);
        n0[q] = fma(sig, z1, p.q0);
        if (MS != 1) box_muller_axpb(wc.c, wc.d, sig, p.q0, n1[q], n2[q]);
        // CGM measurement and PID
        const Real y = fma(p.cC, p.x[10], cgm_sd * zc);
        const Real e = y - gsp;
        p.integ = fmin(fmax(fma(e, ts, p.integ), -imax), imax);
        const Real deriv = k == 0 ? Real(0) : (y - p.y_prev) * inv_ts;
        p.y_prev = y;
        Real u = fmax(fma(p.kd, deriv, fma(p.ki, p.integ, fma(p.kp, e, p.ubh))), Real(0));
        // glucagon mode: no insulin, a microbolus proportional to the distance below
        // the threshold (the PID state above still advances)
        bool gmode = false;
        Real gg = Real(0);
        if (GLU) {
          gmode = glu_on && y < gg_thr;
          gg = gmode ? fmin(gg_gain * (gg_thr - y), gg_max) : Real(0);
          u = gmode ? Real(0) : u;
          p.ggd += gg;
        }
        p.bas += u;
        Real dist = Real(0);
        if (MEAL) {
          Cold &C = cold[q * B + threadIdx.x];
          Real bol = Real(0);
          const Real tdd500 = sizeof(Real) == 8 ? (Real)C.tdd500d : (Real)C.tdd500;
          if (use_plan) {
            const uint32_t midx = day * (uint32_t)VCT_MAX_MEALS + (uint32_t)pm;
            const Words4 wm = philox4x32_10(Words4{midx, C.pid, stream, kTagMeal}, key0, key1);
            const Real amount = (Real)((double)plan_gkg * C.bw);
            const Real carbs =
                fmax(amount * fma(meal_cv, box_muller_first(wm.a, wm.b, Real(0)), Real(1)), Real(0));
            dist += carbs * c_mmol;
            if (bolus_on && !gmode) bol = fma(carbs, tdd500, bol);
          } else {
            for (int jj = 0; jj < sm.meal_cnt[slot]; ++jj) {
              const uint32_t midx = day * n_meals + (uint32_t)sm.meal_j[slot * VCT_MAX_MEALS + jj];
              const Words4 wm = philox4x32_10(Words4{midx, C.pid, stream, kTagMeal}, key0, key1);
              const Real carbs =
                  fmax(fma(meal_sd, box_muller_first(wm.a, wm.b, Real(0)), meal_mean), Real(0));
              dist += carbs * c_mmol;
              if (bolus_on && !gmode) bol = fma(carbs, tdd500, bol);
            }
          }
          C.BOL += (double)bol;
          C.BOLd += (double)bol;
          u = fma(bol, bolus_rate, u);
        }
        if (tracing) {
          const uint32_t i = base + (uint32_t)(q * B);
          if (i < n_trace)
            store_trace(a, sc.trace_offset + (int64_t)k * n_trace + i, trace_bg ? g : y);
        }
        hu[q] = h * u;
        bD[q] = p.hAG * dist;
        hg[q] = gg * h_per_ts;
      }

      {
        const uint32_t k1 = k + 1u;
        const uint32_t c1_hi = __umulhi(kPhiloxM0, k1), c1_lo = kPhiloxM0 * k1;
#pragma unroll
        for (int q = 0; q < PPT; ++q)
          wnext[q] = PhiloxLaneRk{P[q].w0, P[q].w1, rk}.call(c1_hi, c1_lo, kTagSde);
      }

      // m Euler-Maruyama steps; normal 1 + s of the period drives step s.  Steps
      // 0-2 use the first call's normals, later calls are drawn as they are used.
      if (MS > 0) {
#pragma unroll
        for (int q = 0; q < PPT; ++q) em_step<Real, GLU>(P[q], hu[q], bD[q], hR, n0[q], hg[q], gc);
        if (MS > 1) {
#pragma unroll
          for (int q = 0; q < PPT; ++q) em_step<Real, GLU>(P[q], hu[q], bD[q], hR, n1[q], hg[q], gc);
        }
        if (MS > 2) {
#pragma unroll
          for (int q = 0; q < PPT; ++q) em_step<Real, GLU>(P[q], hu[q], bD[q], hR, n2[q], hg[q], gc);
        }
#pragma unroll
        for (int c = 1; 4 * c <= MS; ++c) {
          Real z[PPT][4];
#pragma unroll
          for (int q = 0; q < PPT; ++q) {
            const PhiloxLaneRk lane{P[q].w0, P[q].w1, rk};
            const Words4 w = lane.call(c0_hi, c0_lo, kTagSde | ((uint32_t)c << 8));
            box_muller_axpb(w.a, w.b, sig, P[q].q0, z[q][0], z[q][1]);
            if (4 * c + 1 < MS) box_muller_axpb(w.c, w.d, sig, P[q].q0, z[q][2], z[q][3]);
            else z[q][2] = z[q][3] = P[q].q0;
          }
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (4 * c - 1 + t < MS) {
#pragma unroll
              for (int q = 0; q < PPT; ++q) em_step<Real, GLU>(P[q], hu[q], bD[q], hR, z[q][t], hg[q], gc);
            }
          }
        }
      } else {
        // any m: call c holds normals 4c .. 4c+3, i.e. steps 4c-1 .. 4c+2
        for (int c = 0; 4 * c <= m; ++c) {
          Real z[PPT][4];
#pragma unroll
          for (int q = 0; q < PPT; ++q) {
            if (c == 0) {
              z[q][1] = n0[q];
              z[q][2] = n1[q];
              z[q][3] = n2[q];
            } else if (noise) {
              const PhiloxLaneRk lane{P[q].w0, P[q].w1, rk};
              const Words4 w = lane.call(c0_hi, c0_lo, kTagSde | ((uint32_t)c << 8));
              box_muller_axpb(w.a, w.b, sig, P[q].q0, z[q][0], z[q][1]);
              box_muller_axpb(w.c, w.d, sig, P[q].q0, z[q][2], z[q][3]);
            } else {
              z[q][0] = z[q][1] = z[q][2] = z[q][3] = P[q].q0;
            }
          }
          for (int t = (c == 0 ? 1 : 0); t < 4; ++t) {
            if (4 * c - 1 + t >= m) break;
#pragma unroll
            for (int q = 0; q < PPT; ++q) em_step<Real, GLU>(P[q], hu[q], bD[q], hR, z[q][t], hg[q], gc);
          }
        }
      }

      // a patient whose state turned non-finite stops being binned
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        Hot<Real> &p = P[q];
        // the test first and unconditionally: with `alive` tested first (the
        // test then under a branch) the FP32 kernel measured 2 % slower
        const bool bad = state_nonfinite<Real, GLU>(p);
        if (bad && p.alive) {
          p.alive = false;
          cold[q * B + threadIdx.x].status |= VCT_PATIENT_NONFINITE;
#pragma unroll
          for (int j = 0; j < VCT_NSTATE; ++j) p.x[j] = Real(NAN);
        }
      }

  };

  while (k < k_end) {
    // the periods up to the end of this day (or of the run), then the day's end
    const uint32_t k_stop = k_end - k < per_day - kd ? k_end : k + (per_day - kd);
    while (k < k_stop) {
      // up to the next meal (or the day's end) no period has one
      const uint32_t k_meal =
          (meal_kd != 0xFFFFFFFFu && meal_kd - kd < k_stop - k) ? k + (meal_kd - kd) : k_stop;
      for (; k < k_meal; ++k, ++kd) period(std::false_type());
      if (k < k_stop) {
        period(std::true_type());
        ++k;
        ++kd;
        if (use_plan) {
          ++pm;
          next_plan_meal();
          meal_kd = plan_kd;
        } else {
          ++slot;
          meal_kd = slot < sm.n_slots ? (uint32_t)sm.meal_kd[slot] : 0xFFFFFFFFu;
        }
      }
    }
    if (kd == per_day) {
      kd = 0;
      ++day;
      slot = 0;
      if (use_plan) {
        dp = sc.plan + (day % (uint32_t)sc.plan_days);
        pm = 0;
        next_plan_meal();
      }
      meal_kd = use_plan ? plan_kd : (sm.n_slots > 0 ? (uint32_t)sm.meal_kd[0] : 0xFFFFFFFFu);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        if (dose) bin_day(P[q], cold[q * B + threadIdx.x], a.ts, dose);
        fold<Real, GLU>(P[q], cold[q * B + threadIdx.x]);
      }
    }
  }

#pragma unroll
  for (int q = 0; q < PPT; ++q)
    finish_patient<Real, GLU>(a, P[q], cold[q * B + threadIdx.x], (int64_t)s * pop.n + base + (uint32_t)(q * B),
                              k_end < horizon);
}

}  // namespace
}  // namespace vct

#include "vct_sim_pk2.cuh"

namespace vct {
namespace {

// The kernel loop: a persistent CTA pulls work items from the queue, a
// non-persistent one runs blockIdx.x.  PK: two patients per thread in packed
// FP32 pairs (run_item_pk2; FP32, m = 10, lean, PPT = 2).
template <typename Real, int MS, int PPT, bool GLU, int LEAN, bool PK>
__device__ __forceinline__ void sim_body(const SimArgs &a) {
  __shared__ Smem sm;
  __shared__ uint32_t sh_hist[VCT_BG_BINS];  // BG histogram of this CTA's current item
  extern __shared__ Cold cold[];  // [PPT][blockDim.x], then the daily-dose histograms if asked
  uint32_t *sh_dose = reinterpret_cast<uint32_t *>(cold + PPT * blockDim.x);
  if (a.bg_hist)
    for (int j = threadIdx.x; j < VCT_BG_BINS; j += blockDim.x) sh_hist[j] = 0u;
  if (a.dose_hist)
    for (int j = threadIdx.x; j < 3 * VCT_DOSE_BINS; j += blockDim.x) sh_dose[j] = 0u;
  int64_t item = blockIdx.x;
  for (;;) {
    if (a.persistent) {
      __syncthreads();
      if (threadIdx.x == 0) sm.item = atomicAdd(a.queue, 1);
      __syncthreads();
      item = sm.item;
    }
    if (item >= a.n_items) break;
    const int rank = (int)(item / a.blocks_per_scen);
    const int b = (int)(item % a.blocks_per_scen);
    const int s = a.order[rank];
    // stage this scenario's meal slots: distinct within-day periods, ascending,
    // with the meals (by scenario index, the noise counter) that fall on each
    if (threadIdx.x == 0) {
      const ScenDev &sc = a.scen[s];
      sm.n_slots = sc.n_meal_slots;
      for (int t = 0; t < sc.n_meal_slots; ++t) {
        sm.meal_kd[t] = sc.meal_kd[t];
        int c = 0;
        for (int j = 0; j < sc.n_meals; ++j)
          if (sc.meal_slot[j] == t) sm.meal_j[t * VCT_MAX_MEALS + c++] = j;
        sm.meal_cnt[t] = c;
      }
    }
    __syncthreads();
    if constexpr (PK)
      run_item_pk2(a, s, b, sm, cold, a.dose_hist ? sh_dose : nullptr);
    else
      run_item<Real, MS, PPT, GLU, LEAN>(a, s, b, sm, cold, (!LEAN && a.bg_hist) ? sh_hist : nullptr,
                                         a.dose_hist ? sh_dose : nullptr);
    if (a.bg_hist || a.dose_hist) __syncthreads();
    if (a.bg_hist) {
      for (int j = threadIdx.x; j < VCT_BG_BINS; j += blockDim.x) {
        if (sh_hist[j]) atomicAdd(&a.bg_hist[(int64_t)s * VCT_BG_BINS + j], sh_hist[j]);
        sh_hist[j] = 0u;
      }
    }
    if (a.dose_hist) {
      for (int j = threadIdx.x; j < 3 * VCT_DOSE_BINS; j += blockDim.x) {
        if (sh_dose[j]) atomicAdd(&a.dose_hist[(int64_t)s * 3 * VCT_DOSE_BINS + j], sh_dose[j]);
        sh_dose[j] = 0u;
      }
    }
    if (!a.persistent) break;
  }
}

// Natural register allocation (up to 255 per thread for blocks of <= 256).
template <typename Real, int MS, int PPT, bool GLU>
__global__ void __launch_bounds__(kMaxBlock) sim_kernel(const __grid_constant__ SimArgs a) {
  sim_body<Real, MS, PPT, GLU, false, false>(a);
}

// Capped register allocation: more resident warps, possibly a few spills.
// LEAN 1: a run with no trace, no BG histogram and fixed daily meals (no
// protocol); those branches are compiled out.  LEAN 2: the same with the trace
// branch kept (a traced run that asks for nothing else).  LEAN 0: every
// branch.  PK: the packed two-patient form.
template <typename Real, int MS, int PPT, int REG, bool GLU, int LEAN, bool PK>
__global__ void __maxnreg__(REG) sim_kernel_r(const __grid_constant__ SimArgs a) {
  sim_body<Real, MS, PPT, GLU, LEAN, PK>(a);
}

// Dynamic shared memory: the Cold records, then (with a daily-dose histogram)
// 3 x VCT_DOSE_BINS counters.  Above the default 48 KB the kernel opts in.
template <typename Real, int MS, int PPT, int REG, bool GLU, int LEAN, bool PK>
struct SimVariant {
  static_assert(!LEAN || REG != 0, "the lean variants have a register cap");
  static_assert(!PK || (LEAN == 1 && PPT == 2 && MS == 10 && !GLU), "the packed form is lean, m = 10, two patients");
  static const void *fn() {
    if constexpr (REG == 0)
      return (const void *)sim_kernel<Real, MS, PPT, GLU>;
    else
      return (const void *)sim_kernel_r<Real, MS, PPT, REG, GLU, LEAN, PK>;
  }
  static size_t smem(int block, bool dose) {
    return sizeof(Cold) * PPT * block + (dose ? sizeof(uint32_t) * 3 * VCT_DOSE_BINS : 0);
  }
  static cudaError_t opt_in(size_t bytes) {
    return bytes > (48u << 10)
               ? cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
               : cudaSuccess;
  }
  static cudaError_t launch(const SimArgs &a, int block, int grid, cudaStream_t st) {
    const size_t bytes = smem(block, a.dose_hist != nullptr);
    cudaError_t e = opt_in(bytes);
    if (e != cudaSuccess) return e;
    if constexpr (REG == 0)
      sim_kernel<Real, MS, PPT, GLU><<<grid, block, bytes, st>>>(a);
    else
      sim_kernel_r<Real, MS, PPT, REG, GLU, LEAN, PK><<<grid, block, bytes, st>>>(a);
    return cudaGetLastError();
  }
  // resident blocks per SM, counted with the daily-dose histogram (the larger case)
  static int occupancy(int block) {
    int nb = 0;
    const size_t bytes = smem(block, true);
    if (opt_in(bytes) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn(), block, bytes) != cudaSuccess) return 0;
    return nb;
  }
};

}  // namespace
}  // namespace vct

namespace vct {
namespace {
// op 0: launch (returns the cudaError_t), op 1: resident blocks per SM.
template <typename Real, int MS, int PPT, int REG, bool GLU = false, int LEAN = 0, bool PK = false>
int run_variant(int op, const SimArgs *a, int block, int grid, cudaStream_t st) {
  using V = SimVariant<Real, MS, PPT, REG, GLU, LEAN, PK>;
  return op == 0 ? (int)V::launch(*a, block, grid, st) : V::occupancy(block);
}
}  // namespace
}  // namespace vct
