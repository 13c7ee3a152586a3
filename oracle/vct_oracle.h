/*
 * vct_oracle.h -- plain FP64 CPU oracle of the closed-loop Monte Carlo path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, constant table or helper with the CUDA library: every
 * formula below is written out again from the paper (arXiv 2202.13927) and
 * the literature it cites, in the plainest order.
 *
 * Sections followed:
 *   Sec. III-A, Eq. (1a-d)  SDE patient form  dx = f dt + sigma dw, y_k = g(x_k) + v_k
 *   Sec. III-A, Eq. (2)     zero-order hold of u and d over [t_k, t_k+1)
 *   Sec. III-B, Eq. (3)     controller x^c_{k+1} = kappa(..), u_k = lambda(..)
 *   Sec. III-C              low-memory online accumulation of the indicators
 *   Sec. IV-A               five BG ranges (3 / 3.9 / 10 / 13.9 mmol/L)
 *   Sec. IV-B               Hovorka 2004 model + one-state CGM; parameter
 *                           acceptance (nonnegative, normals within 1 SD,
 *                           basal >= 0.4 U/h)
 *   Sec. IV (30 s step)     integration step
 *   Sec. IV-B, IV-C         two-state s.c. glucagon model and the AP's
 *                           glucagon mode (no insulin, glucagon microboli)
 * The model equations, the parameter table, the diffusion, the controller and
 * the random-number layout are project readings (the paper does not print
 * them); each reading is stated at the point where it is used.
 */
#ifndef VCT_ORACLE_H
#define VCT_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define VCTO_NPAR 16   /* model parameters, slot 16 of a parameter row is body weight */
#define VCTO_NROW 17
#define VCTO_NX 11
#define VCTO_MAXMEALS 8

/* parameter slots */
enum { VO_EGP0, VO_F01, VO_K12, VO_KA1, VO_KA2, VO_KA3, VO_SIT, VO_SID, VO_SIE,
       VO_KE, VO_VI, VO_VG, VO_TAUS, VO_TAUD, VO_AG, VO_TAUCGM, VO_BW };
/* state slots */
enum { XO_D1, XO_D2, XO_S1, XO_S2, XO_I, XO_X1, XO_X2, XO_X3, XO_Q1, XO_Q2, XO_GSC };

typedef struct {
  double bw_mean, bw_sd;            /* kg */
  double p_mean[VCTO_NPAR];
  double p_sd[VCTO_NPAR];           /* 0 = the parameter is fixed */
  double g_sp;                      /* setpoint, mmol/L */
  double min_basal_u_per_h;         /* acceptance threshold on the basal rate */
  double sigma_q1;                  /* diffusion on Q1, mmol min^-1/2 */
  double cgm_sd;                    /* CGM noise sd, mmol/L */
  uint64_t seed;
  int32_t max_attempts;             /* parameter-set attempts before giving up */
  int32_t pad;
  double tau_gg_min;                /* s.c. glucagon absorption time constant, min */
  double s_gg;                      /* glucagon sensitivity of EGP, kg/ug */
} vcto_pop_desc;

/* One protocol day (Sec. II-B): meals at minute[j] of g_per_kg[j] g/kg (Table II). */
typedef struct {
  int32_t n_meals;
  int32_t pad;
  float minute[VCTO_MAXMEALS];
  float g_per_kg[VCTO_MAXMEALS];
} vcto_day_plan;

typedef struct {
  double kp_mult, ki_mult, kd_mult; /* multipliers on the nominal gains */
  double kp_per_ub;                 /* nominal Kp = kp_per_ub * ub_hat per mmol/L */
  double ti_min, td_min;            /* integral and derivative times */
  double i_max;                     /* anti-windup clamp of the integral, mmol min/L */
  double basal_scale;               /* controller's belief of the basal = scale * u_b */
  double meal_mean_g, meal_sd_g;
  double meal_minute[VCTO_MAXMEALS];
  int32_t n_meals;
  int32_t bolus;                    /* 1 = announced meal bolus */
  int64_t horizon;                  /* control periods */
  uint32_t stream_id;               /* scenario word of the noise counters */
  uint32_t pad;
  const vcto_day_plan *day_plans;   /* protocol (NULL: the fixed daily meals above) */
  int32_t n_day_plans;              /* day d follows day_plans[d % n_day_plans] */
  float meal_cv;                    /* relative sd of protocol meal sizes */
  int32_t glucagon;                 /* 1 = glucagon mode below gg_threshold */
  int32_t pad2;
  double gg_threshold;              /* CGM value that switches to glucagon mode, mmol/L */
  double gg_gain;                   /* microbolus per mmol/L below the threshold, ug */
  double gg_max_ug;                 /* largest microbolus per period, ug */
} vcto_scenario;

typedef struct {
  double ts_min;                    /* control period */
  int32_t substeps;                 /* m integration steps per period */
  int32_t integrator;               /* 0 = Euler-Maruyama, 1 = RK4 (sigma must be 0) */
  int32_t noise_refine;             /* R >= 1: each step's normal is the scaled sum of R
                                       normals of an R-times finer grid (order tests) */
  int32_t pad;
  double edge_band[2][4];           /* two windows (mmol/L) around each range edge; a binned
                                       sample within edge_band[w][e] of edge e is counted in
                                       near_edge[w][e] (a sample there may fall on either side
                                       of the edge under rounding) */
} vcto_opts;

typedef struct {
  uint32_t tir[5];                  /* periods per BG range */
  uint32_t hypo_episodes;           /* entries into G < 70 mg/dL */
  uint32_t q1_clamps;               /* Q1 clamped at zero */
  uint32_t status;                  /* bit0: a state became non-finite */
  double g_mean, g_var;             /* mmol/L, (mmol/L)^2, over the binned samples */
  double g_min, g_max;
  double basal_u, bolus_u;          /* insulin delivered, U */
  uint32_t n_samples;
  uint32_t pad;
  double glucagon_ug;               /* glucagon delivered, ug */
  uint32_t near_edge[2][4];         /* binned samples with |G - edge e| <= edge_band[w][e] */
} vcto_stats;

void vcto_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void vcto_normals4(const uint32_t ctr[4], const uint32_t key[2], double z[4]);
/* Box-Muller of one word pair: u = (w + 1/2) 2^-32, z = sqrt(-2 ln u0) (cos, sin)(2 pi u1) */
void vcto_box_muller(uint32_t w0, uint32_t w1, double z[2]);

/* 0 = root found, 1 = no steady state at the setpoint */
int vcto_basal(const double *row, double g_sp, double *u_b, double *x0);

/* rows [n][17], u_b [n], x0 [n][11], status [n] (0 ok, 1 rejected), attempts [n] */
int vcto_create_population(const vcto_pop_desc *d, int64_t first_patient, int64_t n,
                           double *rows, double *u_b, double *x0, int32_t *status,
                           int32_t *attempts, int nthreads);

/* traces (may be NULL) are [n][horizon] (x: [n][horizon][11], z: the glucagon
 * compartments [n][horizon][2]), sampled at t_k; day_doses (may be NULL) is
 * [n][horizon / periods_per_day][3]: basal U, bolus U and glucagon ug delivered
 * in each whole day the patient ended with a finite state, NaN otherwise */
int vcto_simulate(const vcto_pop_desc *d, int64_t first_patient, int64_t n,
                  const double *rows, const double *u_b, const double *x0,
                  const vcto_scenario *sc, const vcto_opts *o, vcto_stats *out,
                  double *trace_g, double *trace_y, double *trace_u, double *trace_x,
                  double *trace_z, double *day_doses, int nthreads);

/* drift f(x, u, d) of the patient model, for tests */
void vcto_drift(const double *row, const double *x, double u, double d, double *f);

#ifdef __cplusplus
}
#endif
#endif
