/*
 * vct_oracle.c -- plain FP64 CPU oracle of the closed-loop Monte Carlo path.
 *
 * TEST INFRASTRUCTURE ONLY (see vct_oracle.h).  Slow and obvious on purpose:
 * one patient at a time, the drift written term by term as the model states
 * it, x_{n+1} = x_n + h f(x_n) + sigma sqrt(h) xi_n with no rearrangement,
 * mean and variance of the binned glucose by the two-pass definition over the
 * stored per-patient samples.  Built with -ffp-contract=off so that x86 and
 * Arm give the same numbers.
 */
#include "vct_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Philox4x32-10, as published by Salmon, Moraes, Dror and Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64
 * multiplies; between rounds the two key words are bumped by the Weyl
 * constants.  The paper under study names no generator; using a counter-based
 * one makes every draw a function of (seed, counter) alone.
 * ------------------------------------------------------------------------- */
void vcto_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): (w + 1/2) 2^-32, exact in FP64.  Box-Muller on the word
 * pairs (0,1) and (2,3): z0 = r cos(2 pi u1), z1 = r sin(2 pi u1) with
 * r = sqrt(-2 ln u0), and the same for words 2 and 3. */
static double uniform_open(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

void vcto_box_muller(uint32_t w0, uint32_t w1, double z[2]) {
  const double two_pi = 6.283185307179586476925286766559;
  double u0 = uniform_open(w0);
  double u1 = uniform_open(w1);
  double r = sqrt(-2.0 * log(u0));
  z[0] = r * cos(two_pi * u1);
  z[1] = r * sin(two_pi * u1);
}

void vcto_normals4(const uint32_t ctr[4], const uint32_t key[2], double z[4]) {
  uint32_t w[4];
  vcto_philox4x32_10(ctr, key, w);
  vcto_box_muller(w[0], w[1], z);
  vcto_box_muller(w[2], w[3], z + 2);
}

/* Stream tags (fourth counter word, low byte). */
enum { TAG_PERIOD = 0, TAG_MEAL = 2, TAG_PARAM = 3 };

static void seed_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32);
}

/* The q-th standard normal of control period k: call q/4 of counter
 * (k, patient, stream, PERIOD | call << 8), slot q%4.  Normal 0 is the CGM
 * noise of the period; normal 1 + j drives the j-th Euler step (j on the
 * finest grid when the noise is refined), so the CGM draw does not depend on
 * the step size. */
static double period_normal(const uint32_t key[2], uint32_t k, uint32_t pid, uint32_t stream,
                            uint32_t q) {
  uint32_t ctr[4] = {k, pid, stream, (uint32_t)TAG_PERIOD | ((q / 4u) << 8)};
  double z[4];
  vcto_normals4(ctr, key, z);
  return z[q % 4u];
}

static double sde_normal(const uint32_t key[2], uint32_t k, uint32_t pid, uint32_t stream,
                         uint32_t j) {
  return period_normal(key, k, pid, stream, 1u + j);
}

static double cgm_normal(const uint32_t key[2], uint32_t k, uint32_t pid, uint32_t stream) {
  return period_normal(key, k, pid, stream, 0u);
}

static double meal_normal(const uint32_t key[2], uint32_t idx, uint32_t pid, uint32_t stream) {
  uint32_t ctr[4] = {idx, pid, stream, (uint32_t)TAG_MEAL};
  double z[4];
  vcto_normals4(ctr, key, z);
  return z[0];
}

/* ---------------------------------------------------------------------------
 * Patient model (Sec. IV-B): the Hovorka et al. 2004 glucose-insulin model
 * plus a one-state CGM lag.  Units: time min, glucose masses mmol, G mmol/L,
 * insulin infusion u mU/min, plasma insulin I mU/L, meal input d mmol/min.
 *   D1' = A_G d - D1/tau_D          D2' = D1/tau_D - D2/tau_D,  U_G = D2/tau_D
 *   S1' = u - S1/tau_S              S2' = S1/tau_S - S2/tau_S
 *   I'  = S2/(tau_S V_I BW) - k_e I
 *   x_i' = -k_ai x_i + k_ai S_i I   (S_1,2,3 = S_IT, S_ID, S_IE)
 *   Q1' = -F01c - F_R - x1 Q1 + k12 Q2 + U_G + EGP0 BW (1 - x3)
 *   Q2' = x1 Q1 - (k12 + x2) Q2,    G = Q1/(V_G BW)
 *   F01c = F01 BW min(1, G/4.5),    F_R = 0.003 (G - 9) V_G BW if G > 9 else 0
 *   Gsc' = (G - Gsc)/tau_CGM
 * ------------------------------------------------------------------------- */
void vcto_drift(const double *p, const double *x, double u, double d, double *f) {
  double bw = p[VO_BW];
  double g = x[XO_Q1] / (p[VO_VG] * bw);
  double u_g = x[XO_D2] / p[VO_TAUD];
  double f01c = g >= 4.5 ? p[VO_F01] * bw : p[VO_F01] * bw * g / 4.5;
  double f_r = g > 9.0 ? 0.003 * (g - 9.0) * p[VO_VG] * bw : 0.0;

  f[XO_D1] = p[VO_AG] * d - x[XO_D1] / p[VO_TAUD];
  f[XO_D2] = x[XO_D1] / p[VO_TAUD] - x[XO_D2] / p[VO_TAUD];
  f[XO_S1] = u - x[XO_S1] / p[VO_TAUS];
  f[XO_S2] = x[XO_S1] / p[VO_TAUS] - x[XO_S2] / p[VO_TAUS];
  f[XO_I] = x[XO_S2] / (p[VO_TAUS] * p[VO_VI] * bw) - p[VO_KE] * x[XO_I];
  f[XO_X1] = -p[VO_KA1] * x[XO_X1] + p[VO_KA1] * p[VO_SIT] * x[XO_I];
  f[XO_X2] = -p[VO_KA2] * x[XO_X2] + p[VO_KA2] * p[VO_SID] * x[XO_I];
  f[XO_X3] = -p[VO_KA3] * x[XO_X3] + p[VO_KA3] * p[VO_SIE] * x[XO_I];
  f[XO_Q1] = -f01c - f_r - x[XO_X1] * x[XO_Q1] + p[VO_K12] * x[XO_Q2] + u_g +
             p[VO_EGP0] * bw * (1.0 - x[XO_X3]);
  f[XO_Q2] = x[XO_X1] * x[XO_Q1] - (p[VO_K12] + x[XO_X2]) * x[XO_Q2];
  f[XO_GSC] = (g - x[XO_GSC]) / p[VO_TAUCGM];
}

/* ---------------------------------------------------------------------------
 * Basal steady state.  With no meal and u = u_b held, setting every derivative
 * to zero at G = G_sp gives I = u_b/(V_I BW k_e), x_i = S_i I,
 * Q2 = x1 Q1/(k12 + x2), and, eliminating Q2 from the Q1 equation, one scalar
 * equation for I:
 *   r(I) = EGP0 BW (1 - S_IE I) - F01c(G_sp) - F_R(G_sp)
 *          - Q1_sp S_IT I S_ID I / (k12 + S_ID I) = 0,   Q1_sp = G_sp V_G BW,
 * strictly decreasing on I >= 0, with r(1/S_IE) < 0.  Bisection on
 * [0, 1/S_IE] until the midpoint stops moving.  The paper's trial B (basal
 * 50 % low) presupposes this "correct basal" per patient.
 * ------------------------------------------------------------------------- */
static double basal_residual(const double *p, double g_sp, double i) {
  double bw = p[VO_BW];
  double q1 = g_sp * p[VO_VG] * bw;
  double f01c = g_sp >= 4.5 ? p[VO_F01] * bw : p[VO_F01] * bw * g_sp / 4.5;
  double f_r = g_sp > 9.0 ? 0.003 * (g_sp - 9.0) * p[VO_VG] * bw : 0.0;
  double x1 = p[VO_SIT] * i, x2 = p[VO_SID] * i, x3 = p[VO_SIE] * i;
  return p[VO_EGP0] * bw * (1.0 - x3) - f01c - f_r - q1 * x1 * x2 / (p[VO_K12] + x2);
}

int vcto_basal(const double *p, double g_sp, double *u_b, double *x0) {
  for (int j = 0; j < VCTO_NROW; ++j)
    if (!isfinite(p[j])) return 1;
  if (!(p[VO_SIE] > 0.0)) return 1;
  double lo = 0.0, hi = 1.0 / p[VO_SIE];
  if (!(basal_residual(p, g_sp, lo) > 0.0)) return 1;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (basal_residual(p, g_sp, mid) > 0.0)
      lo = mid;
    else
      hi = mid;
  }
  double i_ss = 0.5 * (lo + hi);
  double bw = p[VO_BW];
  double ub = i_ss * p[VO_VI] * bw * p[VO_KE];
  double q1 = g_sp * p[VO_VG] * bw;
  double x1 = p[VO_SIT] * i_ss, x2 = p[VO_SID] * i_ss, x3 = p[VO_SIE] * i_ss;
  *u_b = ub;
  x0[XO_D1] = 0.0;
  x0[XO_D2] = 0.0;
  x0[XO_S1] = ub * p[VO_TAUS];
  x0[XO_S2] = ub * p[VO_TAUS];
  x0[XO_I] = i_ss;
  x0[XO_X1] = x1;
  x0[XO_X2] = x2;
  x0[XO_X3] = x3;
  x0[XO_Q1] = q1;
  x0[XO_Q2] = x1 * q1 / (p[VO_K12] + x2);
  x0[XO_GSC] = g_sp;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Population draw (Sec. IV-B acceptance rule).  Reading: every parameter with
 * sd > 0 is N(mean, sd); a draw is kept only if |z| <= 1 (within one SD) and
 * the value is nonnegative, else the next normal of its own sequence is tried
 * (at most 64).  Because parameters are independent this per-parameter
 * rejection equals rejecting whole sets on those box constraints.  The set
 * is then rejected as a whole, and drawn again with the next set-attempt
 * counter, if the basal steady state does not exist or u_b < min_basal.
 * Counter of draw t of slot j in set attempt s: (s, patient, j*256 + t/4,
 * PARAM), normal t%4.
 * ------------------------------------------------------------------------- */
static int draw_set(const vcto_pop_desc *d, const uint32_t key[2], uint32_t pid, uint32_t s,
                    double *row) {
  for (int j = 0; j < VCTO_NROW; ++j) {
    double mean = j < VCTO_NPAR ? d->p_mean[j] : d->bw_mean;
    double sd = j < VCTO_NPAR ? d->p_sd[j] : d->bw_sd;
    if (sd == 0.0) {
      row[j] = mean;
      continue;
    }
    int ok = 0;
    for (uint32_t t = 0; t < 64 && !ok; ++t) {
      uint32_t ctr[4] = {s, pid, (uint32_t)j * 256u + t / 4u, (uint32_t)TAG_PARAM};
      double z[4];
      vcto_normals4(ctr, key, z);
      double zt = z[t % 4u];
      double v = mean + sd * zt;
      if (fabs(zt) <= 1.0 && v >= 0.0) {
        row[j] = v;
        ok = 1;
      }
    }
    if (!ok) return 0;
  }
  return 1;
}

static void create_one(const vcto_pop_desc *d, uint32_t pid, double *row, double *ub,
                       double *x0, int32_t *status, int32_t *attempts) {
  uint32_t key[2];
  seed_key(d->seed, key);
  *status = 1;
  *attempts = d->max_attempts;
  for (int s = 0; s < d->max_attempts; ++s) {
    if (!draw_set(d, key, pid, (uint32_t)s, row)) continue;
    double u;
    if (vcto_basal(row, d->g_sp, &u, x0) != 0) continue;
    if (u * 60.0 / 1000.0 < d->min_basal_u_per_h) continue;
    *ub = u;
    *status = 0;
    *attempts = s + 1;
    return;
  }
  /* rejected: keep the last row drawn, mark the patient */
  *ub = 0.0;
  for (int i = 0; i < VCTO_NX; ++i) x0[i] = 0.0;
}

/* ---------------------------------------------------------------------------
 * One closed-loop patient run.
 * Each control period k (t_k = k Ts, Sec. III-B):
 *   1. bin G(t_k) = Q1/(V_G BW) into the five ranges (Sec. IV-A), edges
 *      54/70/180/250 mg/dL = those values / 18 mmol/L, lower-closed;
 *   2. y_k = Gsc(t_k) + v_k, v_k ~ N(0, cgm_sd^2)            (Eq. 1d);
 *   3. PID on e_k = y_k - G_sp (reading of Eq. 3):
 *        integral += e_k Ts, clamped to +-i_max; deriv = (y_k - y_{k-1})/Ts
 *        (0 at k = 0); u_pid = max(0, ub_hat + Kp e + Ki integral + Kd deriv),
 *        ub_hat = basal_scale u_b, Kp = kp_mult kp_per_ub ub_hat,
 *        Ki = ki_mult kp_per_ub ub_hat / Ti, Kd = kd_mult kp_per_ub ub_hat Td;
 *   4. meal at this period: carbs = max(0, mean + sd z); d_k = carbs (1000/180.16)
 *      / Ts mmol/min over this one period; bolus = carbs TDD/500 U with
 *      TDD = 48 ub_hat[U/h], delivered over this period;
 *   5. m steps of Euler-Maruyama with u_k, d_k held (Eq. 2), noise on Q1 only,
 *      Q1 clamped at zero afterwards (counted).
 *
 * Glucagon (Sec. IV-B: a two-state model of s.c. glucagon; Sec. IV-C: the AP
 * switches to a glucagon mode in which no insulin is given and only glucagon
 * microboli are).  Reading, with the glucagon parameters shared by all
 * patients as Sec. IV-B states:
 *   Z1' = u_gg - Z1/tau_gg,   Z2' = (Z1 - Z2)/tau_gg          (ug, ug/min)
 *   EGP = EGP0 BW (1 - x3 + s_gg Z2/BW), i.e. Q1' gains EGP0 s_gg Z2;
 *   Z1 = Z2 = 0 at the basal state (no glucagon at rest);
 *   with the scenario's glucagon flag, a period whose CGM value y_k lies below
 *   gg_threshold is in glucagon mode: u_pid and the meal bolus are withheld
 *   (the PID state still advances), and min(gg_gain (gg_threshold - y_k),
 *   gg_max) ug of glucagon is given over the period (u_gg = that / Ts).
 * ------------------------------------------------------------------------- */
typedef struct {
  const vcto_pop_desc *d;
  const vcto_scenario *sc;
  const vcto_opts *o;
  int64_t first;
  const double *rows, *ub, *x0;
  vcto_stats *out;
  double *trace_g, *trace_y, *trace_u, *trace_x, *trace_z, *day_doses;
  int64_t begin, end;
} sim_job;

static void rk4_step(const double *p, double *x, double u, double d, double h) {
  double k1[VCTO_NX], k2[VCTO_NX], k3[VCTO_NX], k4[VCTO_NX], t[VCTO_NX];
  vcto_drift(p, x, u, d, k1);
  for (int i = 0; i < VCTO_NX; ++i) t[i] = x[i] + 0.5 * h * k1[i];
  vcto_drift(p, t, u, d, k2);
  for (int i = 0; i < VCTO_NX; ++i) t[i] = x[i] + 0.5 * h * k2[i];
  vcto_drift(p, t, u, d, k3);
  for (int i = 0; i < VCTO_NX; ++i) t[i] = x[i] + h * k3[i];
  vcto_drift(p, t, u, d, k4);
  for (int i = 0; i < VCTO_NX; ++i)
    x[i] = x[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

static void simulate_one(const sim_job *job, int64_t i, double *gbuf) {
  const vcto_pop_desc *d = job->d;
  const vcto_scenario *sc = job->sc;
  const vcto_opts *o = job->o;
  const double *p = job->rows + i * VCTO_NROW;
  vcto_stats *st = job->out + i;
  const int64_t horizon = sc->horizon;
  uint32_t pid = (uint32_t)(job->first + i);
  uint32_t key[2];
  seed_key(d->seed, key);

  memset(st, 0, sizeof(*st));
  double x[VCTO_NX];
  for (int j = 0; j < VCTO_NX; ++j) x[j] = job->x0[i * VCTO_NX + j];
  int finite = 1;
  for (int j = 0; j < VCTO_NX; ++j) finite = finite && isfinite(x[j]);
  for (int j = 0; j < VCTO_NROW; ++j) finite = finite && isfinite(p[j]);

  const double ts = o->ts_min;
  const int m = o->substeps;
  const int refine = o->noise_refine > 1 ? o->noise_refine : 1;
  const double h = ts / (double)m;
  const int64_t per_day = (int64_t)llround(1440.0 / ts);
  const double edges[4] = {54.0 / 18.0, 70.0 / 18.0, 180.0 / 18.0, 250.0 / 18.0};

  const double ub_hat = sc->basal_scale * job->ub[i];
  const double kp_nom = sc->kp_per_ub * ub_hat;
  const double kp = sc->kp_mult * kp_nom;
  const double ki = sc->ki_mult * kp_nom / sc->ti_min;
  const double kd = sc->kd_mult * kp_nom * sc->td_min;
  const double tdd = 2.0 * 24.0 * (ub_hat * 60.0 / 1000.0);
  const double sig_sqrt_h = d->sigma_q1 * sqrt(h);

  double integral = 0.0, y_prev = 0.0, g_prev = 0.0;
  double z1 = 0.0, z2 = 0.0;  /* s.c. glucagon compartments, ug */
  /* Fig. 5: insulin and glucagon delivered per whole day */
  const int64_t n_days = horizon / per_day;
  double day_basal = 0.0, day_bolus = 0.0, day_gg = 0.0;
  if (job->day_doses)
    for (int64_t j = 0; j < n_days * 3; ++j) job->day_doses[i * n_days * 3 + j] = NAN;
  const double tau_gg = d->tau_gg_min;
  int64_t n = 0;
  double gmin = 0.0, gmax = 0.0;

  for (int64_t k = 0; k < horizon && finite; ++k) {
    /* 1. measures on plasma glucose at t_k */
    double g = x[XO_Q1] / (p[VO_VG] * p[VO_BW]);
    int b = 0;
    for (int e = 0; e < 4; ++e)
      if (g >= edges[e]) b++;
    st->tir[b]++;
    for (int w = 0; w < 2; ++w)
      for (int e = 0; e < 4; ++e)
        if (fabs(g - edges[e]) <= o->edge_band[w][e]) st->near_edge[w][e]++;
    if (g < edges[1] && (k == 0 || g_prev >= edges[1])) st->hypo_episodes++;
    g_prev = g;
    if (n == 0 || g < gmin) gmin = g;
    if (n == 0 || g > gmax) gmax = g;
    gbuf[n++] = g;

    /* 2. CGM measurement */
    double y = x[XO_GSC] + d->cgm_sd * cgm_normal(key, (uint32_t)k, pid, sc->stream_id);

    /* 3. PID */
    double e_k = y - d->g_sp;
    integral += e_k * ts;
    if (integral > sc->i_max) integral = sc->i_max;
    if (integral < -sc->i_max) integral = -sc->i_max;
    double deriv = k == 0 ? 0.0 : (y - y_prev) / ts;
    y_prev = y;
    double u_pid = ub_hat + kp * e_k + ki * integral + kd * deriv;
    if (u_pid < 0.0) u_pid = 0.0;

    /* glucagon mode: no insulin, a glucagon microbolus */
    int glucagon_mode = sc->glucagon && y < sc->gg_threshold;
    double gg = 0.0;
    if (glucagon_mode) {
      gg = sc->gg_gain * (sc->gg_threshold - y);
      if (gg > sc->gg_max_ug) gg = sc->gg_max_ug;
      u_pid = 0.0;
    }

    /* 4. meals and the announced bolus */
    double dist = 0.0, bolus_u = 0.0;
    int64_t day = k / per_day, kd_in_day = k % per_day;
    /* protocol days (Sec. II-B, Table II): meal j of day d has g_per_kg BW
     * (1 + cv z) g, clipped at 0, z from meal counter d * 8 + j */
    if (sc->day_plans) {
      const vcto_day_plan *dp = &sc->day_plans[day % sc->n_day_plans];
      for (int j = 0; j < dp->n_meals; ++j) {
        int64_t meal_k = (int64_t)llround((double)dp->minute[j] / ts);
        if (meal_k != kd_in_day) continue;
        uint32_t idx = (uint32_t)(day * VCTO_MAXMEALS + j);
        double grams = (double)dp->g_per_kg[j] * p[VO_BW];
        double carbs = grams * (1.0 + (double)sc->meal_cv * meal_normal(key, idx, pid, sc->stream_id));
        if (carbs < 0.0) carbs = 0.0;
        dist += carbs * (1000.0 / 180.16) / ts;
        if (sc->bolus) bolus_u += carbs * tdd / 500.0;
      }
    }
    for (int j = 0; j < (sc->day_plans ? 0 : sc->n_meals); ++j) {
      int64_t meal_k = (int64_t)llround(sc->meal_minute[j] / ts);
      if (meal_k != kd_in_day) continue;
      uint32_t idx = (uint32_t)(day * sc->n_meals + j);
      double carbs = sc->meal_mean_g + sc->meal_sd_g * meal_normal(key, idx, pid, sc->stream_id);
      if (carbs < 0.0) carbs = 0.0;
      dist += carbs * (1000.0 / 180.16) / ts;
      if (sc->bolus) bolus_u += carbs * tdd / 500.0;
    }
    if (glucagon_mode) bolus_u = 0.0;
    double u = u_pid + bolus_u * 1000.0 / ts;
    st->basal_u += u_pid * ts / 1000.0;
    st->bolus_u += bolus_u;
    st->glucagon_ug += gg;
    day_basal += u_pid * ts / 1000.0;
    day_bolus += bolus_u;
    day_gg += gg;
    double u_gg = gg / ts;

    if (job->trace_g) job->trace_g[i * horizon + k] = g;
    if (job->trace_y) job->trace_y[i * horizon + k] = y;
    if (job->trace_u) job->trace_u[i * horizon + k] = u;
    if (job->trace_x)
      for (int j = 0; j < VCTO_NX; ++j) job->trace_x[(i * horizon + k) * VCTO_NX + j] = x[j];
    if (job->trace_z) {
      job->trace_z[(i * horizon + k) * 2] = z1;
      job->trace_z[(i * horizon + k) * 2 + 1] = z2;
    }

    /* 5. integrate over [t_k, t_k+1) */
    for (int s = 0; s < m; ++s) {
      if (o->integrator == 1) {
        rk4_step(p, x, u, dist, h);
      } else {
        double f[VCTO_NX];
        vcto_drift(p, x, u, dist, f);
        double xi = 0.0;
        if (d->sigma_q1 != 0.0) {
          for (int r = 0; r < refine; ++r)
            xi += sde_normal(key, (uint32_t)k, pid, sc->stream_id, (uint32_t)(s * refine + r));
          xi /= sqrt((double)refine);
        }
        /* glucagon compartments and their effect on EGP, at x_n */
        double fz1 = 0.0, fz2 = 0.0;
        if (sc->glucagon) {
          f[XO_Q1] += p[VO_EGP0] * d->s_gg * z2;
          fz1 = u_gg - z1 / tau_gg;
          fz2 = (z1 - z2) / tau_gg;
        }
        for (int j = 0; j < VCTO_NX; ++j) x[j] = x[j] + h * f[j];
        z1 += h * fz1;
        z2 += h * fz2;
        x[XO_Q1] += sig_sqrt_h * xi;
      }
      if (x[XO_Q1] < 0.0) {
        x[XO_Q1] = 0.0;
        st->q1_clamps++;
      }
    }
    for (int j = 0; j < VCTO_NX; ++j) finite = finite && isfinite(x[j]);
    finite = finite && isfinite(z1) && isfinite(z2);
    if ((k + 1) % per_day == 0) {  /* the day ends with this period */
      if (job->day_doses && finite) {
        double *dd = job->day_doses + (i * n_days + k / per_day) * 3;
        dd[0] = day_basal;
        dd[1] = day_bolus;
        dd[2] = day_gg;
      }
      day_basal = day_bolus = day_gg = 0.0;
    }
  }
  if (!finite) st->status |= 1u;

  st->n_samples = (uint32_t)n;
  if (n > 0) {
    double sum = 0.0;
    for (int64_t j = 0; j < n; ++j) sum += gbuf[j];
    double mean = sum / (double)n;
    double ss = 0.0;
    for (int64_t j = 0; j < n; ++j) ss += (gbuf[j] - mean) * (gbuf[j] - mean);
    st->g_mean = mean;
    st->g_var = ss / (double)n;
    st->g_min = gmin;
    st->g_max = gmax;
  }
}

static void *sim_worker(void *arg) {
  sim_job *job = (sim_job *)arg;
  double *gbuf = (double *)malloc(sizeof(double) * (size_t)(job->sc->horizon > 0 ? job->sc->horizon : 1));
  if (!gbuf) return (void *)1;
  for (int64_t i = job->begin; i < job->end; ++i) simulate_one(job, i, gbuf);
  free(gbuf);
  return NULL;
}

int vcto_simulate(const vcto_pop_desc *d, int64_t first_patient, int64_t n, const double *rows,
                  const double *u_b, const double *x0, const vcto_scenario *sc,
                  const vcto_opts *o, vcto_stats *out, double *trace_g, double *trace_y,
                  double *trace_u, double *trace_x, double *trace_z, double *day_doses,
                  int nthreads) {
  if (n < 0 || o->substeps < 1 || o->ts_min <= 0.0 || sc->horizon < 0) return -1;
  if (o->integrator == 1 && d->sigma_q1 != 0.0) return -1;
  if (o->integrator == 1 && sc->glucagon) return -1;  /* RK4 covers the insulin model only */
  if (sc->glucagon && !(d->tau_gg_min > 0.0)) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = n > 0 ? (int)n : 1;
  sim_job *jobs = (sim_job *)calloc((size_t)nthreads, sizeof(sim_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) return -3;
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    sim_job j = {d, sc, o, first_patient, rows, u_b, x0, out, trace_g, trace_y, trace_u, trace_x,
                 trace_z, day_doses, n * t / nthreads, n * (t + 1) / nthreads};
    jobs[t] = j;
    pthread_create(&th[t], NULL, sim_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) {
    void *r = NULL;
    pthread_join(th[t], &r);
    if (r) rc = -3;
  }
  free(jobs);
  free(th);
  return rc;
}

typedef struct {
  const vcto_pop_desc *d;
  int64_t first, begin, end;
  double *rows, *ub, *x0;
  int32_t *status, *attempts;
} pop_job;

static void *pop_worker(void *arg) {
  pop_job *j = (pop_job *)arg;
  for (int64_t i = j->begin; i < j->end; ++i)
    create_one(j->d, (uint32_t)(j->first + i), j->rows + i * VCTO_NROW, j->ub + i,
               j->x0 + i * VCTO_NX, j->status + i, j->attempts + i);
  return NULL;
}

int vcto_create_population(const vcto_pop_desc *d, int64_t first_patient, int64_t n,
                           double *rows, double *u_b, double *x0, int32_t *status,
                           int32_t *attempts, int nthreads) {
  if (n < 0 || d->max_attempts < 1) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = n > 0 ? (int)n : 1;
  pop_job *jobs = (pop_job *)calloc((size_t)nthreads, sizeof(pop_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) return -3;
  for (int t = 0; t < nthreads; ++t) {
    pop_job j = {d, first_patient, n * t / nthreads, n * (t + 1) / nthreads,
                 rows, u_b, x0, status, attempts};
    jobs[t] = j;
    pthread_create(&th[t], NULL, pop_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return 0;
}
