// vct_internal.cuh -- types shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "vct.h"
#include "vct_rng.cuh"

// The opaque population handle of the C-ABI.
struct vct_population {
  vct_population_desc desc;
  int device;
  void *mem;
  double *rows, *ub, *x0;
  uint32_t *status;
  int32_t *attempts;
  unsigned long long *next;  // the population kernel's work counter
  int64_t n, n_pad, first, n_rejected;
};

namespace vct {

// Population in device memory, structure of arrays (patient index fastest).
struct PopDev {
  const double *rows;      // [17][n_pad]
  const double *ub;        // [n]
  const double *x0;        // [11][n_pad]
  const uint32_t *status;  // [n]
  uint64_t key;            // the population's seed: the Philox key of its noise
  uint32_t rk[kPhiloxRoundKeys];  // its ten round keys (set_key)
  int64_t n, n_pad, first;
  double g_sp, sigma_q1, cgm_sd;
  double tau_gg, s_gg;     // s.c. glucagon model (shared by all patients)
};

inline void set_key(PopDev &d, uint64_t key) {
  d.key = key;
  philox_round_keys(key, d.rk);
}

// One scenario as the kernels read it.
struct ScenDev {
  double kp_mult, ki_mult, kd_mult, kp_per_ub, ti, td, i_max, basal_scale, meal_mean, meal_sd;
  int64_t horizon;
  int64_t trace_offset;  // element offset of this scenario's trace block
  uint32_t stream_id;
  int32_t n_meals;
  int32_t bolus;
  int32_t n_meal_slots;  // distinct meal periods in the day
  int32_t meal_kd[VCT_MAX_MEALS];    // within-day period index of each meal slot, ascending
  int32_t meal_slot[VCT_MAX_MEALS];  // slot of meal j (j = scenario order, the noise counter)
  const vct_day_plan *plan;          // device, protocol days, or nullptr (fixed daily meals)
  int32_t plan_days;
  float meal_cv;
  int32_t glucagon;                  // glucagon mode below gg_thr
  double gg_thr, gg_gain, gg_max;
};

// Resumable per-patient state, structure of arrays over n_scen * n_patients.
// 11 states, integral, y_prev, 3 partials, S1, S2, basal, bolus, min, max, then the
// glucagon compartments Z1, Z2, the day's glucagon partial and the glucagon total
// and the day's bolus (daily doses of Fig. 5)
constexpr int kStateDoubles = 27;
constexpr int kStateWords = 8;     // 4 edge counters, hypo, clamps, samples, flags

struct SimArgs {
  PopDev pop;
  const ScenDev *scen;     // [n_scen]
  const int32_t *order;    // [n_scen] scenarios, longest horizon first
  int32_t n_scen;
  int32_t blocks_per_scen; // work items per scenario
  int64_t n_items;
  int *queue;              // persistent work counter (zeroed before launch)
  int persistent;
  int m;                   // substeps per period
  double ts;               // control period, min
  int64_t period_begin, period_end;
  vct_patient_stats *out;
  void *trace;
  int64_t trace_patients;
  int trace_dtype, trace_kind;
  double *state_in_d;  uint32_t *state_in_w;   // nullptr: start from the basal state
  double *state_out_d; uint32_t *state_out_w;  // nullptr: no write-back
  int finalize;        // 1: the run reaches the horizon, write out[]
  int64_t state_stride;  // n_scen * n_patients
  uint32_t *bg_hist;   // [n_scen][VCT_BG_BINS] or nullptr
  int glucagon;        // 1: some scenario has glucagon mode (the kernel variant with Z1, Z2)
  uint32_t *dose_hist; // [n_scen][3][VCT_DOSE_BINS] or nullptr
  int lean;            // 1: no trace, BG histogram, protocol or glucagon (the lean FP32 variants
                       // apply); 2: a trace and none of the rest; 0: otherwise
};

// launchers (vct_sim.cu, vct_pop.cu, vct_stats.cu)
// (next: the work counter, one device word; zeroed on the stream before the launch)
cudaError_t launch_population(const vct_population_desc &d, double *rows, double *ub, double *x0,
                              uint32_t *status, int32_t *attempts, int64_t n_pad,
                              unsigned long long *next, cudaStream_t st);
// reg: 0 = natural register allocation, else a compiled cap (112, 96, 80)
// (the glucagon variant is chosen by a.glucagon)
cudaError_t launch_simulation(const SimArgs &a, int precision, int block, int ppt, int reg,
                              int grid, cudaStream_t st);
int sim_max_blocks_per_sm(int precision, int block, int ppt, int reg, int m, bool glu, int lean);
bool sim_variant_exists(int precision, int m, int ppt, int reg, bool glu, int lean);
cudaError_t launch_stats(const vct_patient_stats *in, int32_t n_scen, int64_t n_patients,
                         const int64_t *dev_hist_off, int64_t hist_words, void *scratch,
                         size_t scratch_bytes, cudaStream_t st);
size_t stats_scratch_bytes(int32_t n_scen, int64_t n_patients, int64_t hist_words);
vct_population_stats *stats_results(void *scratch, int32_t n_scen, int64_t n_patients,
                                    int64_t hist_words);
cudaError_t launch_box_muller_words(const uint32_t *words, int64_t n, int mode, double *z,
                                    cudaStream_t st);
cudaError_t launch_philox_fill(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *words,
                               void *normals, int precision, cudaStream_t st);

// Record the message vct_last_error() returns on this thread; returns code.
vct_status record_error(vct_status code, const char *msg);

// An NVTX range around a library call (visible to Nsight tools, free otherwise).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace vct
