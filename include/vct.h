/*
 * vct.h -- C-ABI of the GB300 closed-loop virtual-clinical-trial library.
 *
 * The library simulates a population of virtual type-1-diabetes patients in
 * closed loop (arXiv 2202.13927, "High-performance Uncertainty Quantification
 * in Large-scale Virtual Clinical Trials of Closed-loop Diabetes Treatment"):
 * each patient is the stochastic model of Sec. III-A, Eq. (1a-d), integrated
 * by Euler-Maruyama with the inputs held over each control period
 * (Sec. III-A, Eq. 2), driven by a controller evaluated at every sampling
 * time (Sec. III-B, Eq. 3), with the performance indicators accumulated
 * online instead of storing trajectories (Sec. III-C) in the five glucose
 * ranges of Sec. IV-A.  The patient model is the Hovorka 2004 model with a
 * one-state CGM and a two-state s.c. glucagon model (Sec. IV-B); its
 * parameters are drawn per patient with the acceptance rule of Sec. IV-B.
 *
 * Conventions
 *   - Every function returns a vct_status; nothing aborts or throws across
 *     the boundary.  On error, vct_last_error() returns a message for the
 *     calling thread.
 *   - "device" pointers are CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()); "host" pointers are ordinary CPU memory.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Functions marked "asynchronous" only enqueue work on it;
 *     errors raised by that work surface at the next vct_sync() on the stream
 *     or at the next synchronising call.
 *   - Patients are identified by a global id (first_patient + i); every random
 *     number is a function of (seed, global id, counter) alone, so results do
 *     not depend on launch shape, tuning, sharding or batching.
 *   - Units: minutes, mmol, mmol/L (glucose), mU/min (insulin infusion),
 *     mU/L (plasma insulin), kg, g of carbohydrate, U (insulin totals).
 */
#ifndef VCT_H
#define VCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
typedef int vct_status;
#define VCT_OK 0
#define VCT_ERR_ARG (-1)       /* invalid argument or descriptor */
#define VCT_ERR_CUDA (-2)      /* a CUDA call failed (message has the CUDA error) */
#define VCT_ERR_OOM (-3)       /* device or host allocation failed */
#define VCT_ERR_REJECT (-4)    /* some patients found no accepted parameter set */
#define VCT_ERR_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define VCT_ERR_NONFINITE (-6) /* reserved: non-finite patients are flagged, not fatal */
#define VCT_ERR_STATE (-7)     /* object used in the wrong state */

/* ------------------------------------------------------------ dimensions */
#define VCT_NPARAM 16     /* model parameters per patient (slot 16 of a row = body weight) */
#define VCT_NROW 17
#define VCT_NSTATE 11     /* D1 D2 S1 S2 I x1 x2 x3 Q1 Q2 Gsc */
#define VCT_MAX_MEALS 8   /* meals per day in one scenario */
#define VCT_NBINS 5       /* BG ranges of Sec. IV-A */

/* parameter slots of a row (Hovorka 2004 names) */
enum {
  VCT_P_EGP0 = 0, /* endogenous glucose production at zero insulin, mmol/kg/min */
  VCT_P_F01,      /* insulin-independent glucose flux, mmol/kg/min */
  VCT_P_K12,      /* transfer rate Q2 -> Q1, 1/min */
  VCT_P_KA1,      /* deactivation rates of insulin action, 1/min */
  VCT_P_KA2,
  VCT_P_KA3,
  VCT_P_SIT,      /* insulin sensitivity of transport, 1/min per mU/L */
  VCT_P_SID,      /* of disposal, 1/min per mU/L */
  VCT_P_SIE,      /* of endogenous production, per mU/L */
  VCT_P_KE,       /* insulin elimination, 1/min */
  VCT_P_VI,       /* insulin distribution volume, L/kg */
  VCT_P_VG,       /* glucose distribution volume, L/kg */
  VCT_P_TAUS,     /* s.c. insulin absorption time, min */
  VCT_P_TAUD,     /* carbohydrate absorption time, min */
  VCT_P_AG,       /* carbohydrate bioavailability, - */
  VCT_P_TAUCGM,   /* CGM lag, min */
  VCT_P_BW        /* body weight, kg */
};

/* precision of the integrated state */
#define VCT_FP64 0   /* plain form: FP64 state and arithmetic, one patient per thread */
#define VCT_FP32 1   /* fast form: FP32 state, FP64 initial state and long-horizon sums */

/* trace options */
#define VCT_TRACE_NONE 0
#define VCT_TRACE_F16 1
#define VCT_TRACE_F32 2
#define VCT_TRACE_F64 3
#define VCT_TRACE_CGM 0  /* trace y_k, the CGM measurement the controller sees */
#define VCT_TRACE_BG 1   /* trace G(t_k), the plasma glucose that is binned */

/* patient status bits */
#define VCT_PATIENT_NONFINITE 1u  /* a state became non-finite; later periods not binned */
#define VCT_PATIENT_REJECTED 2u   /* no parameter set accepted within max_attempts */

/* ------------------------------------------------------------ descriptors */

/* Population: the distribution table and noise levels (Sec. II-A, IV-B).
 * Parameter j is N(p_mean[j], p_sd[j]) truncated to within one SD and to
 * nonnegative values; p_sd[j] = 0 fixes it.  Body weight likewise.  A set is
 * accepted when the basal steady state at g_sp exists and needs at least
 * min_basal_u_per_h.  sigma_q1 is the diffusion on Q1 (Eq. 1b, additive,
 * mmol min^-1/2); cgm_sd the sd of v_k (Eq. 1d), mmol/L.
 * Glucagon (Sec. IV-B: two s.c. compartments, parameters shared by all
 * patients): Z1' = u_gg - Z1/tau_gg, Z2' = (Z1 - Z2)/tau_gg (ug), and
 * EGP = EGP0 BW (1 - x3 + s_gg Z2 / BW).  Zero at the basal state; only used by
 * scenarios with glucagon != 0 (which need tau_gg_min > 0). */
typedef struct vct_population_desc {
  int64_t n_patients;
  int64_t first_patient;       /* global id of patient 0; first + n <= 2^32 */
  uint64_t seed;
  double bw_mean, bw_sd;       /* kg */
  double p_mean[VCT_NPARAM];
  double p_sd[VCT_NPARAM];
  double g_sp;                 /* glucose setpoint, mmol/L */
  double min_basal_u_per_h;    /* 0.4 in the paper */
  double sigma_q1;
  double cgm_sd;
  int32_t max_attempts;        /* parameter-set attempts, 1..1024 */
  int32_t reserved;
  double tau_gg_min;           /* s.c. glucagon absorption time constant, min */
  double s_gg;                 /* glucagon sensitivity of EGP, kg/ug */
} vct_population_desc;

/* Scenario: one arm of a trial -- controller hyperparameters (p_kappa, p_mu
 * of Eq. 3) and protocol (Sec. II-B).  PID on the CGM signal around g_sp with
 * gains scaled to the controller's basal ub_hat = basal_scale * u_b:
 * Kp = kp_mult kp_per_ub ub_hat, Ki = ki_mult kp_per_ub ub_hat / ti_min,
 * Kd = kd_mult kp_per_ub ub_hat td_min; integral clamped to +-i_max.
 * Meals at meal_minute[] (minute of the day, a multiple of ts_min) with
 * carbohydrates max(0, N(meal_mean_g, meal_sd_g^2)); with bolus != 0 each
 * meal is announced and a bolus of carbs * TDD / 500 U (TDD = 48 ub_hat in
 * U/h) is given over the meal's period.  basal_scale = 0.5 is trial B of the
 * paper.  stream_id is the scenario word of every noise counter: equal ids
 * give common random numbers across scenarios. */
/* One day of a protocol (Sec. II-B): meals at minute[j] (ascending, distinct,
 * multiples of ts_min) of g_per_kg[j] g of carbohydrate per kg body weight
 * (Table II sizes: 1.29 / 0.86 / 0.57 / 0.29 g/kg). */
typedef struct vct_day_plan {
  int32_t n_meals;             /* 0..VCT_MAX_MEALS */
  int32_t reserved;
  float minute[VCT_MAX_MEALS];
  float g_per_kg[VCT_MAX_MEALS];
} vct_day_plan;

typedef struct vct_scenario {
  double kp_mult, ki_mult, kd_mult;
  double kp_per_ub;
  double ti_min, td_min;
  double i_max;                /* mmol min / L */
  double basal_scale;
  double meal_mean_g, meal_sd_g;
  double meal_minute[VCT_MAX_MEALS];
  int32_t n_meals;
  int32_t bolus;
  int64_t horizon_periods;     /* control periods H (52 weeks = 104,832) */
  uint32_t stream_id;
  uint32_t reserved;
  /* Protocol instead of the fixed daily meals (NULL / 0: fixed meals above).
   * Day d follows day_plans[d % n_day_plans]; meal j of day d has
   * max(0, g_per_kg BW (1 + meal_cv z)) g, z the normal of meal counter
   * (d * VCT_MAX_MEALS + j, patient, stream_id, 2).  Host array, copied. */
  const vct_day_plan *day_plans;
  int32_t n_day_plans;
  float meal_cv;
  /* Glucagon mode of the AP (Sec. IV-C: no insulin, only glucagon microboli).
   * With glucagon != 0, a period whose CGM value y_k is below gg_threshold
   * (mmol/L) withholds the PID insulin and the meal bolus (the PID state
   * still advances) and gives min(gg_gain (gg_threshold - y_k), gg_max_ug) ug
   * of glucagon over the period. */
  int32_t glucagon;
  int32_t reserved2;
  double gg_threshold, gg_gain, gg_max_ug;
} vct_scenario;

/* Options of one simulation call. */
typedef struct vct_sim_opts {
  int32_t precision;           /* VCT_FP64 or VCT_FP32 */
  int32_t substeps;            /* m Euler-Maruyama steps per control period (10: h = 30 s) */
  double ts_min;               /* control period Ts in minutes (5); 1440/ts must be an integer */
  void *trace;                 /* device buffer or NULL: [sum_s H_s][trace_patients] per
                                  scenario block, time-major; caller-owned */
  int64_t trace_patients;      /* the first trace_patients patients of every scenario */
  int32_t trace_dtype;         /* VCT_TRACE_NONE / F16 / F32 / F64 */
  int32_t trace_kind;          /* VCT_TRACE_CGM or VCT_TRACE_BG */
  int32_t block_size;          /* threads per block, multiple of 32 up to 256; 0 = library
                                  choice of block size, patients per thread and reg_cap */
  int32_t patients_per_thread; /* 1 or 2 (2: FP32 only); 0 = 1 */
  int32_t steps_per_chunk;     /* > 0: split the run into launches of this many periods (the
                                  state passes between them in device scratch); 0 = one
                                  launch; -1 = let vct_autotune pick launches of about 1 s */
  int32_t persistent;          /* 1 = persistent grid with a longest-first work queue */
  int32_t reg_cap;             /* registers per thread: 0 = compiler's choice, or 128, 112,
                                  96, 80 (FP32, substeps = 10, one patient per thread; 144
                                  and 128 with glucagon) or 168, 128 (two patients per
                                  thread) */
  int32_t reserved;
  int64_t period_begin;        /* resume point (0 = start from the basal state) */
  int64_t period_end;          /* stop point (<= 0 or >= horizon: run to the horizon) */
  void *state_in;              /* device, vct_state_bytes(): needed when period_begin > 0 */
  void *state_out;             /* device, vct_state_bytes(): written when the run stops early */
  uint32_t *bg_hist;           /* device [n_scen][VCT_BG_BINS] or NULL: the simulation ADDS the
                                  count of binned samples G(t_k) per 0.1 mmol/L bin (bin
                                  floor(10 G), the last bin >= 30 mmol/L) -- the population's
                                  BG distribution behind the mean CDF of Fig. 3; caller zeroes */
  uint32_t *dose_hist;         /* device [n_scen][3][VCT_DOSE_BINS] or NULL: the simulation ADDS,
                                  for every whole day a patient ends with a finite state, one
                                  count to the bin of the day's basal insulin (U), bolus insulin
                                  (U) and glucagon (ug): bin floor(dose / VCT_DOSE_*_BIN), the
                                  last bin open -- the distributions of Fig. 5; the dose is
                                  summed in the run's precision; caller zeroes */
  void *workspace;             /* device scratch of at least vct_simulate_workspace_bytes()
                                  bytes, 256-byte aligned, owned by the caller: the call then
                                  allocates nothing.  NULL: the call takes stream-ordered
                                  scratch from the device's memory pool (cudaMallocAsync) and
                                  returns it on the stream (cudaFreeAsync) */
  size_t workspace_bytes;      /* size of workspace */
} vct_sim_opts;

#define VCT_BG_BINS 301
#define VCT_DOSE_BINS 400
#define VCT_DOSE_BASAL_BIN 0.25     /* U per day */
#define VCT_DOSE_BOLUS_BIN 0.25     /* U per day */
#define VCT_DOSE_GLUCAGON_BIN 5.0   /* ug per day */

/* Per-patient indicators (Sec. III-C, IV-A), one per (scenario, patient). */
typedef struct vct_patient_stats {
  uint32_t tir[VCT_NBINS];     /* periods with G in <54, 54-70, 70-180, 180-250, >=250 mg/dL */
  uint32_t hypo_episodes;      /* entries into G < 70 mg/dL */
  uint32_t q1_clamps;          /* Euler-Maruyama steps that clamped Q1 at zero */
  uint32_t status;             /* VCT_PATIENT_* bits */
  uint32_t n_samples;          /* binned periods */
  uint32_t reserved;
  double g_mean, g_var;        /* mean and variance of G(t_k), mmol/L */
  double g_min, g_max;
  double basal_u, bolus_u;     /* insulin delivered, U */
  double glucagon_ug;          /* glucagon delivered, ug (Fig. 5) */
} vct_patient_stats;

/* Population summary of one scenario (Sec. IV-D: mean TIR, box plot,
 * worst-case patient). */
typedef struct vct_population_stats {
  int64_t n_patients;          /* patients counted (not rejected, not non-finite) */
  int64_t n_flagged;           /* non-finite or rejected patients */
  uint64_t tir_total[VCT_NBINS];
  double tir_mean[VCT_NBINS];       /* mean over patients of the per-patient fraction */
  double tir_quantile[VCT_NBINS][5];/* min, 25 %, median, 75 %, max of the per-patient
                                       fraction (inverse-CDF quantiles) */
  int64_t worst_patient;       /* global id with the lowest g_min (ties: lowest id) */
  double worst_g_min;
  double g_mean_mean;          /* mean over patients of g_mean */
  double g_mean_var;           /* variance over patients of g_mean */
  double basal_u_mean, bolus_u_mean;
  int64_t horizon_periods;
  /* span of Fig. 3 at the four range edges: over the counted patients, the
   * fewest and the most periods spent below 54, 70, 180, 250 mg/dL */
  uint32_t below_min[4], below_max[4];
  double glucagon_ug_mean;     /* mean over patients of glucagon_ug */
} vct_population_stats;

typedef struct vct_population vct_population;   /* opaque, library-owned */

/* ------------------------------------------------------------------ calls */

/* Message of the last failed call on the calling thread (thread-local; an
 * empty string if none failed).  The pointer stays valid until that thread's
 * next failing call. */
const char *vct_last_error(void);
/* Library version and the GPU architecture it was compiled for (static string). */
const char *vct_version(void);

/* Draw a population (Sec. IV-B): per patient, parameters by per-parameter
 * rejection inside the one-SD box, then the FP64 basal steady state
 * (bisection on the plasma-insulin equation) and acceptance on
 * min_basal_u_per_h, repeated up to max_attempts sets.  Allocates the
 * population on the current device (freed by vct_destroy_population);
 * synchronises the stream.  Returns VCT_OK even if some patients were
 * rejected; their count is in vct_population_info().n_rejected and they are
 * flagged VCT_PATIENT_REJECTED in every simulation. */
vct_status vct_create_population(const vct_population_desc *desc, void *cuda_stream,
                                 vct_population **out);

/* Build a population from host arrays instead of drawing it: rows [n][17],
 * u_b [n] (mU/min), x0 [n][11].  For fault injection and imported cohorts. */
vct_status vct_population_from_host(const vct_population_desc *desc, const double *rows,
                                    const double *u_b, const double *x0, void *cuda_stream,
                                    vct_population **out);

/* Free a population and its device buffers (NULL is accepted).  The caller
 * makes sure no simulation or plan that uses it is still running. */
vct_status vct_destroy_population(vct_population *pop);

/* Draw a new cohort of the same size and distribution with another seed into
 * an existing population (Sec. IV-B), asynchronously on the stream: the
 * device buffers and every plan built on the population stay valid.  The
 * rejected count is refreshed by the next vct_population_info_get. */
vct_status vct_population_redraw(vct_population *pop, uint64_t seed, void *cuda_stream);

typedef struct vct_population_info {
  int64_t n_patients;
  int64_t first_patient;
  int64_t n_rejected;
  const double *dev_rows;     /* device, [17][n_pad] parameter-major */
  const double *dev_u_b;      /* device, [n] */
  const double *dev_x0;       /* device, [11][n_pad] state-major */
  const uint32_t *dev_status; /* device, [n] */
  const int32_t *dev_attempts;/* device, [n] */
  int64_t n_pad;
} vct_population_info;
/* Sizes, rejected count and the device arrays of a population (the pointers
 * stay owned by the population).  When the rejected count is not yet known
 * (after a redraw) it copies the status array to the host, synchronously. */
vct_status vct_population_info_get(const vct_population *pop, vct_population_info *info);

/* Copy the population to host arrays (any pointer may be NULL):
 * rows [n][17], u_b [n], x0 [n][11], status [n], attempts [n].  Synchronous. */
vct_status vct_population_export(const vct_population *pop, double *rows, double *u_b,
                                 double *x0, uint32_t *status, int32_t *attempts);

/* Closed-loop Monte Carlo simulation of every patient under every scenario
 * (Sec. III, Eq. 1-3): at each period t_k bin G(t_k), take the CGM sample,
 * run the PID and the meal bolus, then m Euler-Maruyama steps with u_k, d_k
 * held.  scenarios: host array [n_scen].  out: device [n_scen][n_patients]
 * (written for the scenarios that reach their horizon in this run; may be
 * NULL when opts->period_end stops every scenario before its horizon).
 * Asynchronous. */
vct_status vct_simulate(const vct_population *pop, const vct_scenario *scenarios,
                        int32_t n_scen, const vct_sim_opts *opts, vct_patient_stats *out,
                        void *cuda_stream);

/* Bytes of device scratch that one vct_simulate call with these arguments
 * needs: the scenario table, the work counter and the protocol days, and with
 * steps_per_chunk > 0 two resumable states (the state passes between the
 * launches through them).  Passing that much as opts->workspace makes the call
 * allocate nothing.  Validates the arguments like vct_simulate.  Needs no GPU. */
vct_status vct_simulate_workspace_bytes(const vct_population *pop, const vct_scenario *scenarios,
                                        int32_t n_scen, const vct_sim_opts *opts, size_t *bytes);

/* Checkpoint and resume (the low-memory runtime of Sec. III-C keeps a
 * patient's whole state, not its trajectory, so a run can stop at any period
 * boundary and continue later).  vct_checkpoint runs every (scenario, patient)
 * from opts->period_begin (the basal state when it is 0, else opts->state_in)
 * up to period period_end and writes the resumable state there into state_out
 * (device, vct_state_bytes(n_scen, n_patients), caller-owned); a scenario whose
 * horizon is at most period_end finishes instead and writes its records into
 * out (device [n_scen][n_patients]; may be NULL when no scenario ends by
 * period_end).  vct_resume continues from state_in at period period_begin
 * (the period_end of the checkpoint that wrote it) to opts->period_end (0 =
 * every scenario's horizon; a later stop writes opts->state_out) and writes
 * the records into out.  The population, scenarios, precision and substeps
 * must be those of the run that wrote the state; the result is bitwise the
 * one of a run without the stop, because every draw is keyed by (seed,
 * patient, period).  The other fields of opts (period_end of vct_checkpoint,
 * period_begin and state_in of vct_resume) are overridden.  Asynchronous. */
vct_status vct_checkpoint(const vct_population *pop, const vct_scenario *scenarios,
                          int32_t n_scen, const vct_sim_opts *opts, int64_t period_end,
                          void *state_out, vct_patient_stats *out, void *cuda_stream);
vct_status vct_resume(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                      const vct_sim_opts *opts, int64_t period_begin, const void *state_in,
                      vct_patient_stats *out, void *cuda_stream);

/* Pick the launch shape of a simulation by timing: block size, patients per
 * thread and register cap are tried on a short run (the scenarios' first day)
 * and the fastest is written to *best (a copy of *base with those fields set;
 * steps_per_chunk = -1 in *base becomes launches of about one second).
 * Results do not depend on the choice (every draw is keyed by patient and
 * period), only the speed does.  out: device [n_scen][n_patients], used as
 * scratch.  Synchronises the stream.  best_ms: time of the winning short run. */
vct_status vct_autotune(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                        const vct_sim_opts *base, vct_patient_stats *out, void *cuda_stream,
                        vct_sim_opts *best, float *best_ms);

/* A simulation prepared once and launched many times: the scenario table and
 * work queue live in device memory owned by the plan, the launch sequence
 * (queue reset + one persistent kernel per chunk) is captured in a CUDA graph
 * and each vct_plan_launch replays it on the given stream (asynchronous).
 * The seed is a kernel argument: a launch that finds the population redrawn
 * since the last one rewrites the seed in every captured kernel node on the
 * host before the replay, so a redraw and the next launch belong on the same
 * stream (or in that order across streams).  With opts->block_size == 0 the
 * plan autotunes first.  The population and out (device [n_scen][n_patients])
 * must outlive the plan. */
typedef struct vct_plan vct_plan;
vct_status vct_plan_create(const vct_population *pop, const vct_scenario *scenarios,
                           int32_t n_scen, const vct_sim_opts *opts, vct_patient_stats *out,
                           void *cuda_stream, vct_plan **plan);
vct_status vct_plan_launch(vct_plan *plan, void *cuda_stream);
vct_status vct_plan_opts(const vct_plan *plan, vct_sim_opts *opts); /* the shape in use */
vct_status vct_plan_destroy(vct_plan *plan);

/* Bytes of the resumable state of n_scen x n_patients patients.  The layout is
 * the kernel's own (its state variables, some held scaled by per-patient
 * coefficients): a blob resumes the run, population and precision that wrote it
 * and is not meant to be read as model states. */
size_t vct_state_bytes(int32_t n_scen, int64_t n_patients);

/* Population reductions (Sec. IV-D) of dev_stats [n_scen][n_patients] into
 * host_out [n_scen]: exact integer histograms of the per-patient range counts
 * give the quantiles, the worst-case patient is the argmin of g_min.
 * horizons: host [n_scen] horizon of each scenario.  first_patient: global id
 * of patient 0.  Synchronises the stream. */
vct_status vct_stats(const vct_patient_stats *dev_stats, int32_t n_scen, int64_t n_patients,
                     const int64_t *horizons, int64_t first_patient,
                     vct_population_stats *host_out, void *cuda_stream);

/* vct_stats with the device scratch given by the caller (dev_workspace,
 * 256-byte aligned, at least vct_stats_workspace_bytes() bytes): the call
 * allocates no device memory; the workspace must not be in use by other work
 * until the call returns.  Same arguments and results as vct_stats.
 * Synchronises the stream. */
vct_status vct_stats_with_workspace(const vct_patient_stats *dev_stats, int32_t n_scen,
                                    int64_t n_patients, const int64_t *horizons,
                                    int64_t first_patient, void *dev_workspace,
                                    size_t workspace_bytes, vct_population_stats *host_out,
                                    void *cuda_stream);
/* Bytes of workspace vct_stats_with_workspace needs for these arguments (the
 * same count as vct_stats_noalloc_bytes); 0 after an argument error.  Needs no
 * GPU. */
size_t vct_stats_workspace_bytes(int32_t n_scen, int64_t n_patients, const int64_t *horizons);

/* Mean BG curve of Fig. 3 (Sec. IV-D) from the BG histograms a simulation
 * filled (opts->bg_hist, device [n_scen][VCT_BG_BINS]): dev_cdf (device
 * [n_scen][VCT_BG_BINS], FP64) receives, for every scenario and bin j, the
 * fraction of its binned samples G(t_k) in bins 0..j, i.e. below the bin's
 * upper edge (j + 1) / 10 mmol/L (1 for the last, open bin; 0 everywhere for a
 * scenario with no samples).  Counts are summed exactly in 64-bit integers
 * (a warp-shuffle scan per scenario) and divided once.  Asynchronous; no
 * allocation. */
vct_status vct_bg_cdf(const uint32_t *dev_bg_hist, int32_t n_scen, double *dev_cdf,
                      void *cuda_stream);

/* Quantiles of the daily doses of Fig. 5 (Sec. IV-D) from the daily-dose
 * histograms a simulation filled (opts->dose_hist, device
 * [n_scen][3][VCT_DOSE_BINS]: basal U, bolus U, glucagon ug per patient-day).
 * For quantile q of a histogram with N counts the rank is r = max(ceil(q N), 1)
 * (inverse-CDF definition); the result is the upper edge (b + 1) w of the
 * first bin b whose running count reaches r, w the bin width of that dose
 * (VCT_DOSE_*_BIN; the last bin is open, its "upper edge" is VCT_DOSE_BINS w),
 * and 0 for an empty histogram.  qs: host [n_q] in [0, 1], 1 <= n_q <=
 * VCT_MAX_QUANTILES (passed to the kernel by value).  dev_out: device
 * [n_scen][3][n_q], FP64.  Asynchronous; no allocation. */
#define VCT_MAX_QUANTILES 16
vct_status vct_dose_quantiles(const uint32_t *dev_dose_hist, int32_t n_scen, const double *qs,
                              int32_t n_q, double *dev_out, void *cuda_stream);

/* vct_stats without any allocation.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory while they run -- for
 * example a host whose device memory is already handed to its own pool
 * allocator, so that a fresh cudaMalloc fails or evicts, or a service that
 * must not call cudaMalloc/cudaFree after start-up because cudaFree waits for
 * the whole device.  Same arguments and results as vct_stats.
 *   - Scratch: one static device array of 8 MiB (VCT_STATS_NOALLOC_BYTES) in
 *     this library, held by every GPU that loads it until the process exits.
 *     A call needs vct_stats_noalloc_bytes() of it (below); larger requests
 *     -- a 52-week scenario takes about 2.1 MB of range histograms, so about
 *     three of them fit -- are rejected with VCT_ERR_ARG and a message; use
 *     vct_stats for those.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it; make
 *     that first call before any stream capture.  That first call (or any
 *     earlier call into this library on the device) also loads the
 *     library's device code, and the 8 MiB array with it, once; a caller
 *     that must not see even that at run time makes one warm-up call at
 *     start-up.  The cache belongs to the device's primary context (the one
 *     the CUDA runtime uses): after cudaDeviceReset, or under another
 *     context, the cached address is not valid.
 *   - All calls share the array.  Each call clears what must start at zero,
 *     but calls that overlap on the GPU (other streams, other threads) race
 *     on it: serialise them.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine, and
 *     allocates no host memory: the horizons are copied from the caller's
 *     array into the fixed array and the histogram offsets are formed there
 *     by a kernel.  Synchronises the stream. */
#define VCT_STATS_NOALLOC_BYTES ((size_t)8 << 20)
vct_status vct_stats_noalloc(const vct_patient_stats *dev_stats, int32_t n_scen,
                             int64_t n_patients, const int64_t *horizons, int64_t first_patient,
                             vct_population_stats *host_out, void *cuda_stream);
/* Bytes of the fixed array that vct_stats_noalloc needs for these arguments
 * (the call is accepted when this is at most VCT_STATS_NOALLOC_BYTES): five
 * regions, each rounded up to a multiple of 256 bytes -- 104 B of integer
 * accumulators per scenario; 32 B and 8 B of FP64 partial sums per reduction
 * block per scenario (ceil(n_patients / 1024) blocks, 1 to 1024); the results,
 * sizeof(vct_population_stats) per scenario; 4 * 5 * (H_s + 1) bytes of range
 * histograms summed over the scenarios -- then 16 B per scenario of offset
 * table.  0 for n_scen <= 0, a NULL horizons or a horizon outside
 * 0 .. 2^32 - 1.  Needs no GPU. */
size_t vct_stats_noalloc_bytes(int32_t n_scen, int64_t n_patients, const int64_t *horizons);

/* Wait for the stream and report the first error of asynchronous work. */
vct_status vct_sync(void *cuda_stream);

/* Diagnostics for tests: the device Philox4x32-10 and the device normals.
 * ctr: device uint32 [n][4], key: (lo, hi); out_words: device uint32 [n][4];
 * out_normals: device [n][4] in the given precision (VCT_FP64 -> double,
 * VCT_FP32 -> float, Box-Muller as the simulation uses it; VCT_FP64_LIBRARY
 * -> double, Box-Muller through the CUDA library's log, sqrt and sincospi,
 * the reference of the simulation's own FP64 transform).  Asynchronous. */
#define VCT_FP64_LIBRARY 2
vct_status vct_philox_fill(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *out_words,
                           void *out_normals, int32_t precision, void *cuda_stream);
/* Diagnostic of the FP64 Box-Muller transform alone (P10 of the reading of
 * Eq. 1b's noise): for every word pair dev_words [n][2] (uint32), the two
 * normals sqrt(-2 ln u0) (cos, sin)(2 pi u1), u = (w + 1/2) 2^-32, into dev_z
 * [n][2] (FP64): mode 0 = the simulation's own transform (table-driven
 * logarithm, Newton reciprocal square root, exact angle reduction), mode 1 =
 * the CUDA library's log, sqrt and sincospi.  Asynchronous. */
vct_status vct_box_muller_words(const uint32_t *dev_words, int64_t n, int32_t mode, double *dev_z,
                                void *cuda_stream);

/* ------------------------------------------------------------ surrogate
 * A learned surrogate of the closed loop -- not in the paper: an MLP maps a
 * patient's parameters and the controller's gain multipliers (hyperparameters
 * of Eq. 3) to the five range fractions of Sec. IV-A, so that many controller
 * tunings can be screened cheaply before the simulation (Sec. III) picks the
 * best.  Features (VCT_SURR_FEATURES = 18): the 14 Hovorka parameters
 * (EGP0 .. tau_D) and body weight, standardized by the population table
 * ((value - mean)/sd; sd 0 gives 0), then ln(kp_mult), ln(ki_mult),
 * ln(kd_mult) divided by ln 3; zero-padded to VCT_SURR_KF.  Network:
 * 18 -> 256 -> 256 -> 5 with ReLU and a softmax; loss the mean cross-entropy
 * against the simulated fractions; AdamW on FP32 master weights.  Tensor-core
 * GEMMs take BF16 operands and accumulate in FP32.
 * Packed parameter vector (FP32, vct_surrogate_n_params() floats):
 *   W1 [256][18], b1 [256], W2 [256][256], b2 [256], W3 [5][256], b3 [5]. */
#define VCT_SURR_FEATURES 18
#define VCT_SURR_KF 32
#define VCT_SURR_HIDDEN 256

typedef struct vct_surrogate_desc {
  int32_t batch;               /* training batch rows, multiple of 64 */
  int32_t reserved;
  uint64_t seed;               /* He-uniform initial weights */
  double lr, beta1, beta2, eps, weight_decay;   /* AdamW */
} vct_surrogate_desc;

typedef struct vct_surrogate vct_surrogate;   /* opaque, library-owned */

/* scale: the population table whose means and sds standardize the features. */
vct_status vct_surrogate_create(const vct_surrogate_desc *desc, const vct_population_desc *scale,
                                void *cuda_stream, vct_surrogate **out);
vct_status vct_surrogate_destroy(vct_surrogate *s);
size_t vct_surrogate_n_params(void);
/* Copy the packed FP32 weights and/or the last gradients to host (synchronous). */
vct_status vct_surrogate_get(const vct_surrogate *s, float *weights, float *grads);
vct_status vct_surrogate_set(vct_surrogate *s, const float *weights, void *cuda_stream);
/* Features of every (scenario, patient) pair: dev_x [n_scen][n][VCT_SURR_KF] FP32. */
vct_status vct_surrogate_features(const vct_surrogate *s, const vct_population *pop,
                                  const vct_scenario *scenarios, int32_t n_scen, float *dev_x,
                                  void *cuda_stream);
/* One forward + backward on explicit rows (dev_x [n][KF], dev_t [n][5] fractions,
 * n <= batch); with update != 0 also one AdamW step.  host_loss (may be NULL):
 * the mean cross-entropy of the rows (synchronises). */
vct_status vct_surrogate_step(vct_surrogate *s, const float *dev_x, const float *dev_t,
                              int64_t n_rows, int32_t update, double *host_loss,
                              void *cuda_stream);
/* Train on simulated runs: samples are the (scenario, patient) pairs of
 * dev_stats [n_scen][n] (targets tir / n_samples) with features from pop and the
 * scenarios' gains; each epoch is one shuffled pass in whole batches.
 * host_epoch_loss [epochs] (may be NULL).  Synchronises once, at the end.  The
 * call holds n_scen x n x 92 bytes of device memory (every sample's feature and
 * target row and its id) and two pinned host copies of the ids (16 bytes per
 * sample); VCT_ERR_OOM if they cannot be had. */
vct_status vct_surrogate_train(vct_surrogate *s, const vct_population *pop,
                               const vct_scenario *scenarios, int32_t n_scen,
                               const vct_patient_stats *dev_stats, int32_t epochs,
                               uint64_t shuffle_seed, double *host_epoch_loss, void *cuda_stream);
/* Learning rate of the AdamW steps that follow (finite, > 0), e.g. a step-down
 * schedule between vct_surrogate_train calls; the moments and the step count
 * (bias corrections) carry on.  Host-side, needs no synchronisation. */
vct_status vct_surrogate_set_lr(vct_surrogate *s, double lr);
/* VCT_ERR_TIMEOUT if a forward pass gave up a bounded wait on the tensor cores
 * (its outputs are then invalid), VCT_ERR_ARG if a device-side screen met an
 * invalid gain, else VCT_OK; an error is reported once and then cleared.
 * Synchronises the stream. */
vct_status vct_surrogate_status(const vct_surrogate *s, void *cuda_stream);
/* Test hook for the failure path (no counterpart in the paper): with on != 0
 * the following forward passes withhold their first tensor-core commit, so
 * every bounded wait in them runs out (about two seconds); the kernel flags
 * the error, waits for its own MMAs, frees TMEM and returns, and
 * vct_surrogate_status reports VCT_ERR_TIMEOUT.  Nothing faults or hangs. */
vct_status vct_surrogate_inject_stall(vct_surrogate *s, int32_t on);
/* Softmax outputs dev_p [n][5] for feature rows dev_x [n][KF].  Asynchronous. */
vct_status vct_surrogate_predict(const vct_surrogate *s, const float *dev_x, int64_t n_rows,
                                 float *dev_p, void *cuda_stream);
/* Screening: for each candidate c (host_gains [n_cand][3] multipliers kp, ki,
 * kd, each finite and > 0, else VCT_ERR_ARG), the predicted fraction of range
 * `bin` averaged over the panel's patients -> dev_scores [n_cand].
 * Asynchronous. */
vct_status vct_surrogate_screen(const vct_surrogate *s, const vct_population *panel,
                                const double *host_gains, int64_t n_cand, int32_t bin,
                                float *dev_scores, void *cuda_stream);
/* The same with the gains already in device memory (dev_gains [n_cand][3]):
 * nothing is computed on the host.  A gain that is not finite and > 0 makes
 * that candidate's score meaningless and the next vct_surrogate_status return
 * VCT_ERR_ARG.  Asynchronous. */
vct_status vct_surrogate_screen_device(const vct_surrogate *s, const vct_population *panel,
                                       const double *dev_gains, int64_t n_cand, int32_t bin,
                                       float *dev_scores, void *cuda_stream);

/* Throughput probe for roofline denominators: kind 0 = FP32 FMA, 1 = FP64 FMA,
 * 2 = INT32 multiply-add, 3 = MUFU lg2, 4 = high half of a 32 x 32 multiply
 * plus an add, 5 = packed FP32 FMA (fma.rn.f32x2: two FMAs per instruction,
 * counted as two lane operations), 6 = unsigned int to float conversion plus
 * an integer add, 7 = 32 x 32 -> 64-bit multiply (mul.wide.u32) plus an add
 * of its halves, `iters` iterations of eight
 * independent chains per thread over 8 x SM-count blocks of 256 threads.
 * ms_out: time of the second of two runs; ops_out: operations (lane ops) it
 * executed.  Synchronises the stream. */
vct_status vct_probe(int32_t kind, int32_t iters, float *ms_out, double *ops_out,
                     void *cuda_stream);

/* sizeof() of a public struct by name ("vct_scenario", ...), 0 if unknown;
 * lets bindings check their struct mirrors.  Needs no GPU. */
size_t vct_struct_size(const char *name);

#ifdef __cplusplus
}
#endif
#endif /* VCT_H */
