// vct_sim_pk2.cuh -- the closed-loop kernel with two patients per thread in
// packed FP32 pairs (included by vct_sim_body.cuh).
//
// The FP32 fast form, m = 10, fixed daily meals, no trace, BG histogram or
// glucagon (the lean configuration of the paper-scale trial): every state,
// coefficient and running sum of the thread's two patients is a pair of floats,
// and every add, multiply and fma of the method is one packed instruction
// (add/sub/mul/fma.rn.f32x2) for both.  Each lane rounds exactly as the scalar
// instruction does, so the two patients get bit for bit the results of the
// one-patient kernel: the same operations in the same order per patient, the
// sign of a negated operand folded into a negated constant (exact).  What has
// no packed form runs per lane: Philox (integer), the hardware approximations
// of Box-Muller, minima and maxima, comparisons, the indicators' counters, and
// a patient whose state turned non-finite (it leaves the packed path: its
// partner's sums go on alone).
#pragma once

namespace vct {
namespace {

struct alignas(8) F2 {
  float x, y;
};

__device__ __forceinline__ unsigned long long pk(F2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ F2 up(unsigned long long r) {
  F2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ F2 both(float v) { return F2{v, v}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return up(d);
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return up(d);
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return up(d);
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return up(d);
}
__device__ __forceinline__ F2 fmin2(F2 a, F2 b) { return F2{fminf(a.x, b.x), fminf(a.y, b.y)}; }
__device__ __forceinline__ F2 fmax2(F2 a, F2 b) { return F2{fmaxf(a.x, b.x), fmaxf(a.y, b.y)}; }
__device__ __forceinline__ float lane(F2 v, int q) { return q == 0 ? v.x : v.y; }
__device__ __forceinline__ void set_lane(F2 &v, int q, float f) {
  if (q == 0) v.x = f;
  else v.y = f;
}

// The two patients' hot data (the packed counterpart of Hot<float>).  The
// coefficients the scalar form uses negated are held negated.
struct Hot2 {
  F2 aD, gD, aS, aI, a1, a2, a3, e1, ne1, ne2, ne3, nf45, q45, q9, q0, hk12, omhk12, hAG, aC, cC,
      inv_vg_bw;
  F2 ubh, kp, ki, kd;
  F2 x[VCT_NSTATE];
  F2 integ, y_prev;
  F2 s1, s2, bas, gmin, gmax;
  uint32_t cge0[2], cge1[2], cge2[2], cge3[2], hypo[2], clamps[2], n[2];
  bool prev_low[2], alive[2];
  uint32_t w0[2], w1[2];
};

#define VCT_PK_FIELD(f) d.f = F2{p0.f, p1.f}
__device__ __forceinline__ void pack(Hot2 &d, const Hot<float> &p0, const Hot<float> &p1) {
  VCT_PK_FIELD(aD); VCT_PK_FIELD(gD); VCT_PK_FIELD(aS); VCT_PK_FIELD(aI); VCT_PK_FIELD(a1);
  VCT_PK_FIELD(a2); VCT_PK_FIELD(a3); VCT_PK_FIELD(e1); VCT_PK_FIELD(q45); VCT_PK_FIELD(q9);
  VCT_PK_FIELD(q0); VCT_PK_FIELD(hk12); VCT_PK_FIELD(omhk12); VCT_PK_FIELD(hAG); VCT_PK_FIELD(aC);
  VCT_PK_FIELD(cC); VCT_PK_FIELD(inv_vg_bw); VCT_PK_FIELD(ubh); VCT_PK_FIELD(kp); VCT_PK_FIELD(ki);
  VCT_PK_FIELD(kd); VCT_PK_FIELD(integ); VCT_PK_FIELD(y_prev); VCT_PK_FIELD(s1); VCT_PK_FIELD(s2);
  VCT_PK_FIELD(bas); VCT_PK_FIELD(gmin); VCT_PK_FIELD(gmax);
  d.ne1 = F2{-p0.e1, -p1.e1};
  d.ne2 = F2{-p0.e2, -p1.e2};
  d.ne3 = F2{-p0.e3, -p1.e3};
  d.nf45 = F2{-p0.f45, -p1.f45};
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) d.x[j] = F2{p0.x[j], p1.x[j]};
  const Hot<float> *p[2] = {&p0, &p1};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    d.cge0[q] = p[q]->cge0;
    d.cge1[q] = p[q]->cge1;
    d.cge2[q] = p[q]->cge2;
    d.cge3[q] = p[q]->cge3;
    d.hypo[q] = p[q]->hypo;
    d.clamps[q] = p[q]->clamps;
    d.n[q] = p[q]->n;
    d.prev_low[q] = p[q]->prev_low;
    d.alive[q] = p[q]->alive;
    d.w0[q] = p[q]->w0;
    d.w1[q] = p[q]->w1;
  }
}
#undef VCT_PK_FIELD

// Back into the scalar form (the fields the end of the item and the state blob
// read; the coefficients are not needed any more).
__device__ __forceinline__ void unpack(const Hot2 &d, int q, Hot<float> &p) {
#pragma unroll
  for (int j = 0; j < VCT_NSTATE; ++j) p.x[j] = lane(d.x[j], q);
  p.integ = lane(d.integ, q);
  p.y_prev = lane(d.y_prev, q);
  p.s1 = lane(d.s1, q);
  p.s2 = lane(d.s2, q);
  p.bas = lane(d.bas, q);
  p.gmin = lane(d.gmin, q);
  p.gmax = lane(d.gmax, q);
  p.cge0 = d.cge0[q];
  p.cge1 = d.cge1[q];
  p.cge2 = d.cge2[q];
  p.cge3 = d.cge3[q];
  p.hypo = d.hypo[q];
  p.clamps = d.clamps[q];
  p.n = d.n[q];
  p.prev_low = d.prev_low[q];
  p.alive = d.alive[q];
  p.Z1 = p.Z2 = p.ggd = 0.0f;
}

// Step 1 of a period for both patients (measure() of the scalar form).
__device__ __forceinline__ void measure2(Hot2 &P, F2 g, float gsp) {
  const float e0 = (float)kEdge0, e1 = (float)kEdge1, e2 = (float)kEdge2, e3 = (float)kEdge3;
  const float gq[2] = {g.x, g.y};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!P.alive[q]) continue;
    const float v = gq[q];
    P.cge0[q] += v >= e0;
    P.cge1[q] += v >= e1;
    P.cge2[q] += v >= e2;
    P.cge3[q] += v >= e3;
    const bool low = v < e1;
    P.hypo[q] += (low && !P.prev_low[q]);
    P.prev_low[q] = low;
    P.n[q] += 1;
  }
  if (P.alive[0] && P.alive[1]) {
    const F2 dev = add2(g, both(-gsp));
    P.s1 = add2(P.s1, dev);
    P.s2 = fma2(dev, dev, P.s2);
    P.gmin = fmin2(P.gmin, g);
    P.gmax = fmax2(P.gmax, g);
  } else {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!P.alive[q]) continue;
      const float v = gq[q], dev = v - gsp;
      set_lane(P.s1, q, lane(P.s1, q) + dev);
      set_lane(P.s2, q, fmaf(dev, dev, lane(P.s2, q)));
      set_lane(P.gmin, q, fminf(lane(P.gmin, q), v));
      set_lane(P.gmax, q, fmaxf(lane(P.gmax, q), v));
    }
  }
}

// Box-Muller of one word pair per lane, as box_muller_f32 / box_muller_axpb
// compute it: returns t = r (cos, sin) of the shifted angle, i.e. the negated
// normals (the callers fold the sign into their constants).
__device__ __forceinline__ void box_muller2_t(const uint32_t w0[2], const uint32_t w1[2], F2 &tc, F2 &ts) {
  const F2 two_m32 = both(2.3283064365386963e-10f), two_m33 = both(1.1641532182693481e-10f);
  const F2 u0 = fma2(F2{__uint2float_rz(w0[0]), __uint2float_rz(w0[1])}, two_m32, two_m33);
  const F2 l = mul2(both(-2.0f), F2{__logf(u0.x), __logf(u0.y)});
  const F2 r2 = fmax2(l, both(1e-30f));
  const F2 r = mul2(r2, F2{rsqrtf(r2.x), rsqrtf(r2.y)});
  const F2 ang = fma2(F2{__uint2float_rz(w1[0]), __uint2float_rz(w1[1])}, both(1.4629180792671596e-09f),
                      both(7.3145904e-10f - 3.14159265358979f));
  float s0, c0, s1, c1;
  __sincosf(ang.x, &s0, &c0);
  __sincosf(ang.y, &s1, &c1);
  tc = mul2(r, F2{c0, c1});
  ts = mul2(r, F2{s0, s1});
}

// The axpb form: n_i = scale z_i + offset with rs = -(r scale) formed once.
__device__ __forceinline__ void box_muller2_axpb(const uint32_t w0[2], const uint32_t w1[2], F2 nscale,
                                                 F2 offset, F2 &n0, F2 &n1) {
  const F2 two_m32 = both(2.3283064365386963e-10f), two_m33 = both(1.1641532182693481e-10f);
  const F2 u0 = fma2(F2{__uint2float_rz(w0[0]), __uint2float_rz(w0[1])}, two_m32, two_m33);
  const F2 r2 = fmax2(mul2(both(-2.0f), F2{__logf(u0.x), __logf(u0.y)}), both(1e-30f));
  const F2 rs = mul2(mul2(r2, F2{rsqrtf(r2.x), rsqrtf(r2.y)}), nscale);  // -(r scale)
  const F2 ang = fma2(F2{__uint2float_rz(w1[0]), __uint2float_rz(w1[1])}, both(1.4629180792671596e-09f),
                      both(7.3145904e-10f - 3.14159265358979f));
  float s0, c0, s1, c1;
  __sincosf(ang.x, &s0, &c0);
  __sincosf(ang.y, &s1, &c1);
  n0 = fma2(rs, F2{c0, c1}, offset);
  n1 = fma2(rs, F2{s0, s1}, offset);
}

// One Euler-Maruyama step for both patients (em_step of the scalar form).
__device__ __forceinline__ void em_step2(Hot2 &P, F2 hu, F2 bD, F2 nhR, F2 nz) {
  F2 *x = P.x;
  const F2 D1 = x[0], D2 = x[1], S1 = x[2], S2 = x[3], I = x[4];
  const F2 X1 = x[5], X2 = x[6], X3 = x[7], Q1 = x[8], Q2 = x[9], GSC = x[10];
  x[0] = fma2(D1, P.aD, bD);
  x[1] = fma2(D2, P.aD, D1);
  x[2] = fma2(S1, P.aS, hu);
  x[3] = fma2(S2, P.aS, S1);
  x[4] = fma2(I, P.aI, S2);
  x[5] = fma2(X1, P.a1, I);
  x[6] = fma2(X2, P.a2, I);
  x[7] = fma2(X3, P.a3, I);
  const F2 hx1 = mul2(P.e1, X1), nhx1 = mul2(P.ne1, X1);
  F2 c = fma2(P.hk12, Q2, nz);
  c = fma2(D2, P.gD, c);
  c = fma2(P.ne3, X3, c);
  F2 q = fma2(P.nf45, fmin2(Q1, P.q45), c);
  const F2 r = fma2(nhx1, Q1, Q1);
  q = fma2(nhR, fmax2(Q1, P.q9), q);
  q = add2(q, r);
  x[9] = fma2(Q2, fma2(P.ne2, X2, P.omhk12), mul2(hx1, Q1));
  x[10] = fma2(GSC, P.aC, Q1);
  const bool neg0 = q.x < 0.0f, neg1 = q.y < 0.0f;
  x[8] = F2{neg0 ? 0.0f : q.x, neg1 ? 0.0f : q.y};
  P.clamps[0] += neg0;
  P.clamps[1] += neg1;
}

// A work item of the packed form: 2 B patients, lanes i and i + B of thread i.
__device__ __forceinline__ void run_item_pk2(const SimArgs &a, int s, int b, const Smem &sm, Cold *cold,
                                             uint32_t *dose) {
  const ScenDev &sc = a.scen[s];
  const int B = blockDim.x;
  const PopDev &pop = a.pop;
  constexpr int MS = 10;
  const double hd = a.ts / (double)MS;
  const F2 h = both((float)hd), nhR = both(-(float)(hd * 0.003));
  const float sigf = (float)(pop.sigma_q1 * sqrt(hd));
  const F2 nsig = both(-sigf);
  const float gsp = (float)pop.g_sp;
  const F2 ncgm_sd = both(-(float)pop.cgm_sd);
  const F2 ts = both((float)a.ts);
  const F2 inv_ts = both((float)(1.0 / a.ts));
  const float c_mmol = (float)(1000.0 / 180.16 / a.ts);
  const F2 bolus_rate = both((float)(1000.0 / a.ts));
  const float imaxf = (float)sc.i_max;
  const float meal_mean = (float)sc.meal_mean, meal_sd = (float)sc.meal_sd;
  const bool bolus_on = sc.bolus != 0;
  const uint32_t per_day = (uint32_t)llround(1440.0 / a.ts);
  const uint32_t horizon = (uint32_t)sc.horizon;
  const uint32_t k_begin = (uint32_t)a.period_begin;
  const uint32_t k_end = (a.period_end > 0 && a.period_end < sc.horizon) ? (uint32_t)a.period_end : horizon;
  const uint64_t seed = pop.key;
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
  const uint32_t *rk = pop.rk;
  const uint32_t stream = sc.stream_id;
  const uint32_t n_meals = (uint32_t)sc.n_meals;
  const uint32_t base = (uint32_t)b * (uint32_t)(B * 2) + threadIdx.x;

  Hot2 P;
  {
    Hot<float> T[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t i = base + (uint32_t)(q * B);
      const bool valid = (int64_t)i < pop.n;
      Cold &C = cold[q * B + threadIdx.x];
      load_patient(T[q], C, a, sc, i, valid, hd);
      if (a.state_in_d && valid) load_state<float, false>(T[q], C, a, (int64_t)s * pop.n + i);
      T[q].w0 = __umulhi(kPhiloxM1, stream) ^ C.pid ^ key0;
      T[q].w1 = kPhiloxM1 * stream;
    }
    pack(P, T[0], T[1]);
  }

  uint32_t day = k_begin / per_day;
  uint32_t kd = k_begin % per_day;
  int slot = 0;
  while (slot < sm.n_slots && (uint32_t)sm.meal_kd[slot] < kd) ++slot;

  Words4 wnext[2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
    wnext[q] = PhiloxLaneRk{P.w0[q], P.w1[q], rk}.call(__umulhi(kPhiloxM0, k_begin), kPhiloxM0 * k_begin,
                                                      kTagSde);
  uint32_t meal_kd = slot < sm.n_slots ? (uint32_t)sm.meal_kd[slot] : 0xFFFFFFFFu;

  uint32_t k = k_begin;
  auto period = [&](auto meal_tag) {
    constexpr bool MEAL = decltype(meal_tag)::value;
    const uint32_t c0_hi = __umulhi(kPhiloxM0, k), c0_lo = kPhiloxM0 * k;
    const F2 g = mul2(P.x[8], P.inv_vg_bw);
    measure2(P, g, gsp);
    // the period's first Philox call: normal 0 is the CGM noise, 1-3 drive steps 0-2
    const uint32_t wa[2] = {wnext[0].a, wnext[1].a}, wb[2] = {wnext[0].b, wnext[1].b};
    const uint32_t wc[2] = {wnext[0].c, wnext[1].c}, wd[2] = {wnext[0].d, wnext[1].d};
    F2 tc, t1;
    box_muller2_t(wa, wb, tc, t1);
    const F2 n0 = fma2(nsig, t1, P.q0);            // sig z1 + q0, z1 = -t1
    F2 n1, n2;
    box_muller2_axpb(wc, wd, nsig, P.q0, n1, n2);
    // CGM measurement and PID
    const F2 y = fma2(P.cC, P.x[10], mul2(ncgm_sd, tc));   // cgm_sd zc, zc = -tc
    const F2 e = add2(y, both(-gsp));
    P.integ = fmin2(fmax2(fma2(e, ts, P.integ), both(-imaxf)), both(imaxf));
    const F2 deriv = k == 0 ? both(0.0f) : mul2(sub2(y, P.y_prev), inv_ts);
    P.y_prev = y;
    F2 u = fmax2(fma2(P.kd, deriv, fma2(P.ki, P.integ, fma2(P.kp, e, P.ubh))), both(0.0f));
    P.bas = add2(P.bas, u);
    F2 dist = both(0.0f);
    if (MEAL) {
      F2 bol = both(0.0f);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        Cold &C = cold[q * B + threadIdx.x];
        float d = 0.0f, bq = 0.0f;
        for (int jj = 0; jj < sm.meal_cnt[slot]; ++jj) {
          const uint32_t midx = day * n_meals + (uint32_t)sm.meal_j[slot * VCT_MAX_MEALS + jj];
          const Words4 wm = philox4x32_10(Words4{midx, C.pid, stream, kTagMeal}, key0, key1);
          const float carbs = fmaxf(fmaf(meal_sd, box_muller_first(wm.a, wm.b, 0.0f), meal_mean), 0.0f);
          d += carbs * c_mmol;
          if (bolus_on) bq = fmaf(carbs, C.tdd500, bq);
        }
        C.BOL += (double)bq;
        C.BOLd += (double)bq;
        set_lane(dist, q, d);
        set_lane(bol, q, bq);
      }
      u = fma2(bol, bolus_rate, u);
    }
    const F2 hu = mul2(h, u);
    const F2 bD = mul2(P.hAG, dist);

    {
      const uint32_t k1 = k + 1u;
      const uint32_t c1_hi = __umulhi(kPhiloxM0, k1), c1_lo = kPhiloxM0 * k1;
#pragma unroll
      for (int q = 0; q < 2; ++q) wnext[q] = PhiloxLaneRk{P.w0[q], P.w1[q], rk}.call(c1_hi, c1_lo, kTagSde);
    }

    em_step2(P, hu, bD, nhR, n0);
    em_step2(P, hu, bD, nhR, n1);
    em_step2(P, hu, bD, nhR, n2);
#pragma unroll
    for (int c = 1; 4 * c <= MS; ++c) {
      F2 z[4];
      Words4 w[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) w[q] = PhiloxLaneRk{P.w0[q], P.w1[q], rk}.call(c0_hi, c0_lo, kTagSde | ((uint32_t)c << 8));
      const uint32_t xa[2] = {w[0].a, w[1].a}, xb[2] = {w[0].b, w[1].b};
      const uint32_t xc[2] = {w[0].c, w[1].c}, xd[2] = {w[0].d, w[1].d};
      box_muller2_axpb(xa, xb, nsig, P.q0, z[0], z[1]);
      if (4 * c + 1 < MS) box_muller2_axpb(xc, xd, nsig, P.q0, z[2], z[3]);
      else z[2] = z[3] = P.q0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * c - 1 + t < MS) em_step2(P, hu, bD, nhR, z[t]);
    }

    // a patient whose state turned non-finite stops being binned
    F2 sum = P.x[0];
#pragma unroll
    for (int j = 1; j < VCT_NSTATE; ++j) sum = add2(sum, P.x[j]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!isfinite(lane(sum, q)) && P.alive[q]) {
        P.alive[q] = false;
        cold[q * B + threadIdx.x].status |= VCT_PATIENT_NONFINITE;
#pragma unroll
        for (int j = 0; j < VCT_NSTATE; ++j) set_lane(P.x[j], q, NAN);
      }
    }
  };

  while (k < k_end) {
    const uint32_t k_stop = k_end - k < per_day - kd ? k_end : k + (per_day - kd);
    while (k < k_stop) {
      const uint32_t k_meal =
          (meal_kd != 0xFFFFFFFFu && meal_kd - kd < k_stop - k) ? k + (meal_kd - kd) : k_stop;
      for (; k < k_meal; ++k, ++kd) period(std::false_type());
      if (k < k_stop) {
        period(std::true_type());
        ++k;
        ++kd;
        ++slot;
        meal_kd = slot < sm.n_slots ? (uint32_t)sm.meal_kd[slot] : 0xFFFFFFFFu;
      }
    }
    if (kd == per_day) {
      kd = 0;
      ++day;
      slot = 0;
      meal_kd = sm.n_slots > 0 ? (uint32_t)sm.meal_kd[0] : 0xFFFFFFFFu;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        Cold &C = cold[q * B + threadIdx.x];
        // bin_day and fold of the scalar form, on this lane
        if (dose && P.alive[q]) {
          const double v[3] = {(double)lane(P.bas, q) * a.ts / 1000.0, C.BOLd, 0.0};
          const double wbin[3] = {VCT_DOSE_BASAL_BIN, VCT_DOSE_BOLUS_BIN, VCT_DOSE_GLUCAGON_BIN};
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double bb = floor(v[j] / wbin[j]);
            atomicAdd(&dose[j * VCT_DOSE_BINS + (bb < (double)(VCT_DOSE_BINS - 1) ? (int)bb : VCT_DOSE_BINS - 1)], 1u);
          }
        }
        if (dose) C.BOLd = 0.0;
        C.S1 += (double)lane(P.s1, q);
        C.S2 += (double)lane(P.s2, q);
        C.B += (double)lane(P.bas, q);
      }
      P.s1 = P.s2 = P.bas = both(0.0f);
    }
  }

#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Hot<float> T;
    unpack(P, q, T);
    finish_patient<float, false>(a, T, cold[q * B + threadIdx.x], (int64_t)s * pop.n + base + (uint32_t)(q * B),
                                 k_end < horizon);
  }
}

}  // namespace
}  // namespace vct
