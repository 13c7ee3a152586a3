// vct_run.cu -- host side of the simulation calls (Sec. III): argument checks,
// the device scenario table, launch shapes, chunked launches with the state
// carried in device scratch, the autotuner and graph-captured plans.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vct_internal.cuh"

struct vct_plan {
  const vct_population *pop;
  vct_sim_opts opts;
  int32_t n_scen;
  vct_patient_stats *out;
  void *dev_tab;   // scenario table + order + queue
  void *state_a, *state_b;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  uint64_t key;                       // the seed the simulation nodes carry
  std::vector<cudaGraphNode_t> nodes; // the simulation kernel nodes
};

namespace {

vct_status fail(vct_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return vct::record_error(code, buf);
}

#define VCT_TRY_CUDA(call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? VCT_ERR_OOM : VCT_ERR_CUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                   \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool finite_all(const double *v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

vct_status check_opts(const vct_sim_opts *o, const vct_population *pop) {
  if (!o) return fail(VCT_ERR_ARG, "options are NULL");
  if (o->precision != VCT_FP64 && o->precision != VCT_FP32)
    return fail(VCT_ERR_ARG, "precision must be VCT_FP64 or VCT_FP32");
  if (o->substeps < 1 || o->substeps > 4096) return fail(VCT_ERR_ARG, "substeps must be in 1..4096");
  if (!(o->ts_min > 0.0) || !std::isfinite(o->ts_min)) return fail(VCT_ERR_ARG, "ts_min must be > 0");
  const double ppd = 1440.0 / o->ts_min;
  if (std::fabs(ppd - std::llround(ppd)) > 1e-9 * ppd)
    return fail(VCT_ERR_ARG, "1440 / ts_min must be an integer");
  if (o->trace_dtype < VCT_TRACE_NONE || o->trace_dtype > VCT_TRACE_F64)
    return fail(VCT_ERR_ARG, "bad trace_dtype");
  if (o->trace_kind != VCT_TRACE_CGM && o->trace_kind != VCT_TRACE_BG)
    return fail(VCT_ERR_ARG, "bad trace_kind");
  if (o->trace && o->trace_dtype != VCT_TRACE_NONE &&
      (o->trace_patients < 0 || o->trace_patients > pop->n))
    return fail(VCT_ERR_ARG, "trace_patients must be in 0..n_patients");
  if (o->trace_dtype != VCT_TRACE_NONE && o->trace_patients > 0 && !o->trace)
    return fail(VCT_ERR_ARG, "trace_dtype set but trace is NULL");
  if (o->block_size != 0 && (o->block_size < 32 || o->block_size > 256 || o->block_size % 32))
    return fail(VCT_ERR_ARG, "block_size must be 0 or a multiple of 32 in 32..256");
  if (o->patients_per_thread < 0 || o->patients_per_thread > 2)
    return fail(VCT_ERR_ARG, "patients_per_thread must be 0, 1 or 2");
  if (o->patients_per_thread > 1 && o->precision == VCT_FP64)
    return fail(VCT_ERR_ARG, "patients_per_thread > 1 needs VCT_FP32");
  if (o->reg_cap != 0) {
    const bool one = o->patients_per_thread <= 1 &&
                     (o->reg_cap == 144 || o->reg_cap == 128 || o->reg_cap == 112 || o->reg_cap == 96 ||
                      o->reg_cap == 80);
    const bool two = o->patients_per_thread == 2 &&
                     (o->reg_cap == 192 || o->reg_cap == 168 || o->reg_cap == 128);
    if (o->precision != VCT_FP32 || o->substeps != 10 || !(one || two))
      return fail(VCT_ERR_ARG, "reg_cap needs VCT_FP32, substeps = 10 and 144 (glucagon only)/128/112/96/80 "
                               "with one patient per thread or 192 (lean runs only)/168/128 with two");
  }
  if (o->period_begin < 0) return fail(VCT_ERR_ARG, "period_begin < 0");
  if (o->period_begin > 0 && !o->state_in) return fail(VCT_ERR_ARG, "period_begin > 0 needs state_in");
  if (o->period_end > 0 && o->period_end <= o->period_begin)
    return fail(VCT_ERR_ARG, "period_end must exceed period_begin");
  if (o->steps_per_chunk < -1) return fail(VCT_ERR_ARG, "steps_per_chunk must be >= -1");
  return VCT_OK;
}

vct_status check_scenario(const vct_scenario *s, double ts, int idx) {
  const double v[] = {s->kp_mult, s->ki_mult, s->kd_mult, s->kp_per_ub, s->ti_min, s->td_min,
                      s->i_max, s->basal_scale, s->meal_mean_g, s->meal_sd_g};
  if (!finite_all(v, 10)) return fail(VCT_ERR_ARG, "scenario %d: non-finite field", idx);
  if (!(s->ti_min > 0.0)) return fail(VCT_ERR_ARG, "scenario %d: ti_min must be > 0", idx);
  if (s->i_max < 0.0 || s->meal_sd_g < 0.0 || s->basal_scale < 0.0)
    return fail(VCT_ERR_ARG, "scenario %d: i_max, meal_sd_g and basal_scale must be >= 0", idx);
  if (s->n_meals < 0 || s->n_meals > VCT_MAX_MEALS)
    return fail(VCT_ERR_ARG, "scenario %d: n_meals must be in 0..%d", idx, VCT_MAX_MEALS);
  if (s->horizon_periods < 0 || s->horizon_periods >= ((int64_t)1 << 32))
    return fail(VCT_ERR_ARG, "scenario %d: horizon_periods must be in 0..2^32-1", idx);
  for (int j = 0; j < s->n_meals; ++j) {
    const double m = s->meal_minute[j];
    if (!(m >= 0.0 && m < 1440.0)) return fail(VCT_ERR_ARG, "scenario %d: meal minute out of range", idx);
    const double q = m / ts;
    if (std::fabs(q - std::llround(q)) > 1e-9 * std::max(1.0, q))
      return fail(VCT_ERR_ARG, "scenario %d: meal minute %g is not a multiple of ts", idx, m);
  }
  if (s->day_plans || s->n_day_plans) {
    if (!s->day_plans || s->n_day_plans < 1 || s->n_day_plans > (1 << 20))
      return fail(VCT_ERR_ARG, "scenario %d: day_plans and 1..2^20 n_day_plans go together", idx);
    if (!(s->meal_cv >= 0.0f) || !std::isfinite(s->meal_cv))
      return fail(VCT_ERR_ARG, "scenario %d: meal_cv must be >= 0", idx);
    for (int d = 0; d < s->n_day_plans; ++d) {
      const vct_day_plan &p = s->day_plans[d];
      if (p.n_meals < 0 || p.n_meals > VCT_MAX_MEALS)
        return fail(VCT_ERR_ARG, "scenario %d day %d: n_meals must be in 0..%d", idx, d, VCT_MAX_MEALS);
      for (int j = 0; j < p.n_meals; ++j) {
        const double m = p.minute[j];
        const double q = m / ts;
        if (!(m >= 0.0 && m < 1440.0) || std::fabs(q - std::llround(q)) > 1e-6 * std::max(1.0, q) ||
            (j > 0 && !(m > p.minute[j - 1])))
          return fail(VCT_ERR_ARG, "scenario %d day %d: meal minutes must ascend, be distinct, in "
                                   "[0, 1440) and multiples of ts", idx, d);
        if (!(p.g_per_kg[j] >= 0.0f) || !std::isfinite(p.g_per_kg[j]))
          return fail(VCT_ERR_ARG, "scenario %d day %d: g_per_kg must be >= 0", idx, d);
      }
    }
  }
  if (s->glucagon) {
    const double g[] = {s->gg_threshold, s->gg_gain, s->gg_max_ug};
    if (!finite_all(g, 3) || s->gg_gain < 0.0 || s->gg_max_ug < 0.0)
      return fail(VCT_ERR_ARG, "scenario %d: gg_threshold must be finite, gg_gain and gg_max_ug >= 0",
                  idx);
  }
  return VCT_OK;
}

vct::PopDev pop_dev(const vct_population *p) {
  vct::PopDev d;
  d.rows = p->rows;
  d.ub = p->ub;
  d.x0 = p->x0;
  d.status = p->status;
  vct::set_key(d, p->desc.seed);
  d.n = p->n;
  d.n_pad = p->n_pad;
  d.first = p->first;
  d.g_sp = p->desc.g_sp;
  d.sigma_q1 = p->desc.sigma_q1;
  d.cgm_sd = p->desc.cgm_sd;
  d.tau_gg = p->desc.tau_gg_min;
  d.s_gg = p->desc.s_gg;
  return d;
}

// Scenario table: meal slots (distinct within-day periods) and trace offsets;
// order = scenarios by horizon, longest first (the work queue's order).
struct Tables {
  std::vector<vct::ScenDev> tab;
  std::vector<int32_t> order;
  std::vector<vct_day_plan> plans;     // all scenarios' protocol days
  std::vector<int64_t> plan_off;       // first plan of scenario s, -1 without a protocol
  int64_t max_h = 0;
  bool glucagon = false;               // some scenario has glucagon mode
  // device addresses of the protocol days, once the tables have a home
  void set_plan_base(vct_day_plan *dev) {
    for (size_t s = 0; s < tab.size(); ++s) tab[s].plan = plan_off[s] >= 0 ? dev + plan_off[s] : nullptr;
  }
};

vct_status build_tables(const vct_scenario *scenarios, int32_t n_scen, const vct_sim_opts &o,
                        bool tracing, Tables &T) {
  T.tab.assign((size_t)n_scen, vct::ScenDev());
  T.plans.clear();
  T.plan_off.clear();
  int64_t trace_off = 0;
  T.max_h = 0;
  T.glucagon = false;
  for (int s = 0; s < n_scen; ++s) {
    const vct_scenario &sc = scenarios[s];
    vct_status rc = check_scenario(&sc, o.ts_min, s);
    if (rc) return rc;
    vct::ScenDev &d = T.tab[s];
    std::memset(&d, 0, sizeof(d));
    d.kp_mult = sc.kp_mult;
    d.ki_mult = sc.ki_mult;
    d.kd_mult = sc.kd_mult;
    d.kp_per_ub = sc.kp_per_ub;
    d.ti = sc.ti_min;
    d.td = sc.td_min;
    d.i_max = sc.i_max;
    d.basal_scale = sc.basal_scale;
    d.meal_mean = sc.meal_mean_g;
    d.meal_sd = sc.meal_sd_g;
    d.horizon = sc.horizon_periods;
    d.stream_id = sc.stream_id;
    d.n_meals = sc.n_meals;
    d.bolus = sc.bolus;
    d.glucagon = sc.glucagon ? 1 : 0;
    d.gg_thr = sc.gg_threshold;
    d.gg_gain = sc.gg_gain;
    d.gg_max = sc.gg_max_ug;
    T.glucagon = T.glucagon || sc.glucagon;
    std::vector<int> kds;
    for (int j = 0; j < sc.n_meals; ++j) kds.push_back((int)std::llround(sc.meal_minute[j] / o.ts_min));
    std::vector<int> uniq = kds;
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    d.n_meal_slots = (int)uniq.size();
    for (size_t t = 0; t < uniq.size(); ++t) d.meal_kd[t] = uniq[t];
    for (int j = 0; j < sc.n_meals; ++j)
      d.meal_slot[j] = (int)(std::lower_bound(uniq.begin(), uniq.end(), kds[j]) - uniq.begin());
    d.trace_offset = trace_off;
    if (tracing) trace_off += sc.horizon_periods * o.trace_patients;
    T.max_h = std::max<int64_t>(T.max_h, sc.horizon_periods);
    if (sc.day_plans) {
      T.plan_off.push_back((int64_t)T.plans.size());
      T.plans.insert(T.plans.end(), sc.day_plans, sc.day_plans + sc.n_day_plans);
      d.plan_days = sc.n_day_plans;
      d.meal_cv = sc.meal_cv;
    } else {
      T.plan_off.push_back(-1);
    }
  }
  T.order.resize((size_t)n_scen);
  for (int s = 0; s < n_scen; ++s) T.order[s] = s;
  std::stable_sort(T.order.begin(), T.order.end(),
                   [&](int a, int b) { return T.tab[a].horizon > T.tab[b].horizon; });
  return VCT_OK;
}

struct Shape {
  int block, ppt, reg, grid;
  bool glu;   // the glucagon variant
  int lean;   // 1: no trace, BG histogram, protocol or glucagon; 2: a trace and none of the rest
  int64_t bps, n_items;
};

vct_status make_shape(const vct_population *pop, int32_t n_scen, const vct_sim_opts &o, bool glu,
                      int lean, Shape &S) {
  S.glu = glu;
  S.lean = lean;
  if (o.block_size == 0) {
    // library choice of the whole shape (measured on GB300 at one million patients
    // over 52 weeks: the FP32 m = 10 kernel runs fastest with 128-thread blocks and
    // a 128-register cap, 16 warps per SM)
    const bool capped = o.precision == VCT_FP32 && o.substeps == 10;
    S.ppt = 1;
    S.block = 128;
    S.reg = capped ? 128 : 0;
  } else {
    S.ppt = o.precision == VCT_FP64 ? 1 : (o.patients_per_thread ? o.patients_per_thread : 1);
    S.block = o.block_size;
    S.reg = o.reg_cap;
  }
  if (!vct::sim_variant_exists(o.precision, o.substeps, S.ppt, S.reg, glu, lean))
    return fail(VCT_ERR_ARG, "no compiled kernel for precision %d, substeps %d, ppt %d, reg_cap %d%s",
                o.precision, o.substeps, S.ppt, S.reg, glu ? " with glucagon" : "");
  const int64_t per_item = (int64_t)S.block * S.ppt;
  S.bps = (pop->n + per_item - 1) / per_item;
  S.n_items = S.bps * n_scen;
  if (S.n_items > ((int64_t)1 << 31) - 1) return fail(VCT_ERR_ARG, "too many work items");
  S.grid = (int)S.n_items;
  if (o.persistent) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = vct::sim_max_blocks_per_sm(o.precision, S.block, S.ppt, S.reg, o.substeps, glu, lean);
    if (per_sm < 1) return fail(VCT_ERR_ARG, "block size %d does not fit on an SM", S.block);
    S.grid = (int)std::min<int64_t>(S.n_items, (int64_t)sms * per_sm);
  }
  return VCT_OK;
}

// Device layout of the per-call tables:
// [ScenDev x S][int32 order x S][int queue][protocol days]
struct DevTables {
  size_t tab_bytes, ord_bytes, plan_off, plan_bytes, total;
  DevTables(int32_t S, size_t n_plans) {
    tab_bytes = align256(sizeof(vct::ScenDev) * S);
    ord_bytes = align256(sizeof(int32_t) * S);
    plan_off = tab_bytes + ord_bytes + 256;
    plan_bytes = align256(sizeof(vct_day_plan) * n_plans);
    total = plan_off + plan_bytes;
  }
};

// Upload the tables into dev (laid out by DevTables), plans first so that the
// scenario table can point at them.
cudaError_t upload_tables(Tables &T, char *dev, const DevTables &L, cudaStream_t st, bool sync_copy) {
  T.set_plan_base((vct_day_plan *)(dev + L.plan_off));
  const size_t S = T.tab.size();
  cudaError_t e = cudaSuccess;
  if (sync_copy) {
    if (!T.plans.empty())
      e = cudaMemcpy(dev + L.plan_off, T.plans.data(), sizeof(vct_day_plan) * T.plans.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dev, T.tab.data(), sizeof(vct::ScenDev) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(dev + L.tab_bytes, T.order.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice);
  } else {
    if (!T.plans.empty())
      e = cudaMemcpyAsync(dev + L.plan_off, T.plans.data(), sizeof(vct_day_plan) * T.plans.size(),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev, T.tab.data(), sizeof(vct::ScenDev) * S, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dev + L.tab_bytes, T.order.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, st);
  }
  return e;
}

vct::SimArgs base_args(const vct_population *pop, const vct_sim_opts &o, const Shape &S,
                       int32_t n_scen, void *dev_tab, vct_patient_stats *out, bool tracing) {
  DevTables L(n_scen, 0);
  vct::SimArgs a;
  std::memset(&a, 0, sizeof(a));
  a.pop = pop_dev(pop);
  a.scen = (const vct::ScenDev *)dev_tab;
  a.order = (const int32_t *)((char *)dev_tab + L.tab_bytes);
  a.queue = (int *)((char *)dev_tab + L.tab_bytes + L.ord_bytes);
  a.n_scen = n_scen;
  a.blocks_per_scen = (int32_t)S.bps;
  a.n_items = S.n_items;
  a.persistent = o.persistent ? 1 : 0;
  a.m = o.substeps;
  a.ts = o.ts_min;
  a.out = out;
  a.trace = tracing ? o.trace : nullptr;
  a.trace_patients = tracing ? o.trace_patients : 0;
  a.trace_dtype = o.trace_dtype;
  a.trace_kind = o.trace_kind;
  a.state_stride = (int64_t)n_scen * pop->n;
  a.finalize = 1;
  a.bg_hist = o.bg_hist;
  a.dose_hist = o.dose_hist;
  a.glucagon = S.glu ? 1 : 0;
  a.lean = S.lean;  // which lean variant applies (see Shape)
  return a;
}

void set_state(vct::SimArgs &a, void *in, void *out) {
  const int64_t S = a.state_stride;
  a.state_in_d = (double *)in;
  a.state_in_w = in ? (uint32_t *)((char *)in + sizeof(double) * vct::kStateDoubles * S) : nullptr;
  a.state_out_d = (double *)out;
  a.state_out_w = out ? (uint32_t *)((char *)out + sizeof(double) * vct::kStateDoubles * S) : nullptr;
}

// Enqueue the run over [begin, end) in launches of at most `chunk` periods.
// Between launches the state goes through scratch_a / scratch_b.
cudaError_t enqueue_run(vct::SimArgs a, const vct_sim_opts &o, const Shape &S, int64_t max_h,
                        void *scratch_a, void *scratch_b, cudaStream_t st) {
  const int64_t begin = o.period_begin;
  const int64_t end = o.period_end > 0 ? o.period_end : max_h;
  const int64_t chunk = o.steps_per_chunk > 0 ? o.steps_per_chunk : 0;
  void *in = o.state_in;
  int64_t c0 = begin;
  int idx = 0;
  for (;;) {
    const bool last = chunk == 0 || c0 + chunk >= end;
    const int64_t c1 = last ? o.period_end : c0 + chunk;  // 0: each scenario to its horizon
    void *out = last ? o.state_out : (idx % 2 == 0 ? scratch_a : scratch_b);
    a.period_begin = c0;
    a.period_end = c1;
    set_state(a, (c0 > 0 || in) ? in : nullptr, out);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
    if (e == cudaSuccess) e = vct::launch_simulation(a, o.precision, S.block, S.ppt, S.reg, S.grid, st);
    if (e != cudaSuccess || last) return e;
    in = out;
    c0 = c1;
    ++idx;
  }
}

bool chunked(const vct_sim_opts &o, int64_t max_h) {
  const int64_t end = o.period_end > 0 ? o.period_end : max_h;
  return o.steps_per_chunk > 0 && o.period_begin + o.steps_per_chunk < end;
}

vct_status prepare(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                   const vct_sim_opts *opts, bool *tracing, Tables &T, Shape &S) {
  if (!pop) return fail(VCT_ERR_ARG, "population is NULL");
  if (n_scen < 0) return fail(VCT_ERR_ARG, "n_scen < 0");
  if (n_scen > 0 && !scenarios) return fail(VCT_ERR_ARG, "scenarios is NULL");
  vct_status rc = check_opts(opts, pop);
  if (rc) return rc;
  *tracing = opts->trace && opts->trace_dtype != VCT_TRACE_NONE && opts->trace_patients > 0;
  if (n_scen == 0 || pop->n == 0) return VCT_OK;
  if ((rc = build_tables(scenarios, n_scen, *opts, *tracing, T))) return rc;
  if (T.glucagon && !(pop->desc.tau_gg_min > 0.0))
    return fail(VCT_ERR_ARG, "glucagon mode needs tau_gg_min > 0 in the population");
  const int lean = (opts->bg_hist == nullptr && T.plans.empty() && !T.glucagon) ? (*tracing ? 2 : 1) : 0;
  return make_shape(pop, n_scen, *opts, T.glucagon, lean, S);
}

}  // namespace

extern "C" {

vct_status vct_simulate(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                        const vct_sim_opts *opts, vct_patient_stats *out, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_simulate");
  Tables T;
  Shape S;
  bool tracing = false;
  vct_status rc = prepare(pop, scenarios, n_scen, opts, &tracing, T, S);
  if (rc) return rc;
  if (n_scen == 0 || pop->n == 0) return VCT_OK;
  if (!out) {
    // records are written only by scenarios that reach their horizon in this run
    bool finishes = opts->period_end <= 0;
    for (int32_t s = 0; s < n_scen && !finishes; ++s) finishes = scenarios[s].horizon_periods <= opts->period_end;
    if (finishes) return fail(VCT_ERR_ARG, "out is NULL but a scenario reaches its horizon in this run");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevTables L(n_scen, T.plans.size());
  const bool ch = chunked(*opts, T.max_h);
  const size_t state_bytes = ch ? align256(vct_state_bytes(n_scen, pop->n)) : 0;
  const size_t need = L.total + 2 * state_bytes;
  void *scratch = nullptr;
  const bool own = opts->workspace == nullptr;
  if (own) {
    VCT_TRY_CUDA(cudaMallocAsync(&scratch, need, st));
  } else {
    if (opts->workspace_bytes < need)
      return fail(VCT_ERR_ARG, "workspace of %zu bytes, the call needs %zu (vct_simulate_workspace_bytes)",
                  opts->workspace_bytes, need);
    if ((uintptr_t)opts->workspace % 256 != 0) return fail(VCT_ERR_ARG, "workspace must be 256-byte aligned");
    scratch = opts->workspace;
  }
  char *sb = (char *)scratch;
  cudaError_t e = upload_tables(T, sb, L, st, false);
  if (e == cudaSuccess) {
    vct::SimArgs a = base_args(pop, *opts, S, n_scen, sb, out, tracing);
    e = enqueue_run(a, *opts, S, T.max_h, ch ? sb + L.total : nullptr,
                    ch ? sb + L.total + state_bytes : nullptr, st);
  }
  cudaError_t ef = own ? cudaFreeAsync(scratch, st) : cudaSuccess;
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "simulation launch: %s", cudaGetErrorString(e));
  if (ef != cudaSuccess) return fail(VCT_ERR_CUDA, "cudaFreeAsync: %s", cudaGetErrorString(ef));
  return VCT_OK;
}

vct_status vct_simulate_workspace_bytes(const vct_population *pop, const vct_scenario *scenarios,
                                        int32_t n_scen, const vct_sim_opts *opts, size_t *bytes) {
  if (!bytes) return fail(VCT_ERR_ARG, "bytes is NULL");
  *bytes = 0;
  if (!pop) return fail(VCT_ERR_ARG, "population is NULL");
  if (n_scen < 0) return fail(VCT_ERR_ARG, "n_scen < 0");
  if (n_scen > 0 && !scenarios) return fail(VCT_ERR_ARG, "scenarios is NULL");
  vct_status rc = check_opts(opts, pop);
  if (rc) return rc;
  if (n_scen == 0 || pop->n == 0) return VCT_OK;
  const bool tracing = opts->trace && opts->trace_dtype != VCT_TRACE_NONE && opts->trace_patients > 0;
  Tables T;
  if ((rc = build_tables(scenarios, n_scen, *opts, tracing, T))) return rc;
  DevTables L(n_scen, T.plans.size());
  const size_t state_bytes = chunked(*opts, T.max_h) ? align256(vct_state_bytes(n_scen, pop->n)) : 0;
  *bytes = L.total + 2 * state_bytes;
  return VCT_OK;
}

vct_status vct_checkpoint(const vct_population *pop, const vct_scenario *scenarios,
                          int32_t n_scen, const vct_sim_opts *opts, int64_t period_end,
                          void *state_out, vct_patient_stats *out, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_checkpoint");
  if (!opts) return fail(VCT_ERR_ARG, "options are NULL");
  if (!state_out) return fail(VCT_ERR_ARG, "state_out is NULL");
  if (period_end <= opts->period_begin) return fail(VCT_ERR_ARG, "period_end must exceed period_begin");
  vct_sim_opts o = *opts;
  o.period_end = period_end;
  o.state_out = state_out;
  return vct_simulate(pop, scenarios, n_scen, &o, out, cuda_stream);
}

vct_status vct_resume(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                      const vct_sim_opts *opts, int64_t period_begin, const void *state_in,
                      vct_patient_stats *out, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_resume");
  if (!opts) return fail(VCT_ERR_ARG, "options are NULL");
  if (period_begin <= 0 || !state_in) return fail(VCT_ERR_ARG, "resume needs period_begin > 0 and state_in");
  vct_sim_opts o = *opts;
  o.period_begin = period_begin;
  o.state_in = const_cast<void *>(state_in);
  return vct_simulate(pop, scenarios, n_scen, &o, out, cuda_stream);
}

vct_status vct_autotune(const vct_population *pop, const vct_scenario *scenarios, int32_t n_scen,
                        const vct_sim_opts *base, vct_patient_stats *out, void *cuda_stream,
                        vct_sim_opts *best, float *best_ms) {
  vct::NvtxRange nvtx_range_("vct_autotune");
  if (!best) return fail(VCT_ERR_ARG, "best is NULL");
  Tables T;
  Shape S;
  bool tracing = false;
  vct_status rc = prepare(pop, scenarios, n_scen, base, &tracing, T, S);
  if (rc) return rc;
  *best = *base;
  if (best_ms) *best_ms = 0.0f;
  if (n_scen == 0 || pop->n == 0) return VCT_OK;
  if (!out) return fail(VCT_ERR_ARG, "out is NULL");
  // timing runs: the first day of every scenario, no trace, no state
  std::vector<vct_scenario> shortened(scenarios, scenarios + n_scen);
  const int64_t day = (int64_t)std::llround(1440.0 / base->ts_min);
  for (auto &s : shortened) s.horizon_periods = std::min<int64_t>(s.horizon_periods, day);
  vct_sim_opts t = *base;
  t.trace = nullptr;
  t.trace_dtype = VCT_TRACE_NONE;
  t.trace_patients = 0;
  t.period_begin = 0;
  t.period_end = 0;
  t.state_in = t.state_out = nullptr;
  t.steps_per_chunk = 0;
  struct Cand { int block, ppt, reg; };
  std::vector<Cand> cands;
  const int blocks[] = {64, 128, 256};
  for (int b : blocks) {
    if (base->precision == VCT_FP64) {
      cands.push_back({b, 1, 0});
      continue;
    }
    cands.push_back({b, 1, 0});
    cands.push_back({b, 2, 0});
    if (base->substeps == 10) {
      for (int r : {144, 128, 112, 96, 80}) cands.push_back({b, 1, r});
      for (int r : {192, 168, 128}) cands.push_back({b, 2, r});
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  VCT_TRY_CUDA(cudaEventCreate(&e0));
  VCT_TRY_CUDA(cudaEventCreate(&e1));
  float best_t = -1.0f;
  Cand win = cands[0];
  for (const Cand &c : cands) {
    vct_sim_opts o = t;
    o.block_size = c.block;
    o.patients_per_thread = c.ppt;
    o.reg_cap = c.reg;
    Tables T2;
    Shape S2;
    bool tr2 = false;
    if (prepare(pop, shortened.data(), n_scen, &o, &tr2, T2, S2) != VCT_OK) continue;
    if (vct_simulate(pop, shortened.data(), n_scen, &o, out, cuda_stream) != VCT_OK) continue;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2; ++r) vct_simulate(pop, shortened.data(), n_scen, &o, out, cuda_stream);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(VCT_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms *= 0.5f;
    if (best_t < 0.0f || ms < best_t) {
      best_t = ms;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_t < 0.0f) return fail(VCT_ERR_CUDA, "autotune: no candidate ran");
  best->block_size = win.block;
  best->patients_per_thread = win.ppt;
  best->reg_cap = win.reg;
  if (best_ms) *best_ms = best_t;
  if (base->steps_per_chunk < 0) {
    // launches of about one second at the measured per-period rate, whole days
    int64_t periods_per_run = 0;
    for (auto &s : shortened) periods_per_run = std::max<int64_t>(periods_per_run, s.horizon_periods);
    const double ms_per_period = periods_per_run ? best_t / (double)periods_per_run : 0.0;
    int64_t chunk = ms_per_period > 0.0 ? (int64_t)(1000.0 / ms_per_period) : 0;
    chunk = std::max<int64_t>(day, chunk / day * day);
    best->steps_per_chunk = (int32_t)std::min<int64_t>(chunk, ((int64_t)1 << 30));
  }
  return VCT_OK;
}

vct_status vct_plan_create(const vct_population *pop, const vct_scenario *scenarios,
                           int32_t n_scen, const vct_sim_opts *opts, vct_patient_stats *out,
                           void *cuda_stream, vct_plan **plan) {
  vct::NvtxRange nvtx_range_("vct_plan_create");
  if (!plan) return fail(VCT_ERR_ARG, "plan is NULL");
  *plan = nullptr;
  if (n_scen < 1) return fail(VCT_ERR_ARG, "a plan needs at least one scenario");
  if (!out) return fail(VCT_ERR_ARG, "out is NULL");
  if (!opts) return fail(VCT_ERR_ARG, "options are NULL");
  vct_sim_opts o = *opts;
  if (o.block_size == 0 || o.steps_per_chunk < 0) {
    vct_sim_opts tuned;
    vct_status rc = vct_autotune(pop, scenarios, n_scen, &o, out, cuda_stream, &tuned, nullptr);
    if (rc) return rc;
    o = tuned;
  }
  Tables T;
  Shape S;
  bool tracing = false;
  vct_status rc = prepare(pop, scenarios, n_scen, &o, &tracing, T, S);
  if (rc) return rc;
  if (pop->n == 0) return fail(VCT_ERR_ARG, "empty population");
  auto *p = new (std::nothrow) vct_plan();
  if (!p) return fail(VCT_ERR_OOM, "host allocation failed");
  p->pop = pop;
  p->opts = o;
  p->n_scen = n_scen;
  p->out = out;
  DevTables L(n_scen, T.plans.size());
  const bool ch = chunked(o, T.max_h);
  const size_t state_bytes = ch ? align256(vct_state_bytes(n_scen, pop->n)) : 0;
  cudaError_t e = cudaMalloc(&p->dev_tab, L.total + 2 * state_bytes);
  if (e != cudaSuccess) {
    delete p;
    return fail(VCT_ERR_OOM, "plan tables: %s", cudaGetErrorString(e));
  }
  char *sb = (char *)p->dev_tab;
  if (ch) {
    p->state_a = sb + L.total;
    p->state_b = sb + L.total + state_bytes;
  }
  e = upload_tables(T, sb, L, nullptr, true);
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    vct::SimArgs a = base_args(pop, o, S, n_scen, sb, out, tracing);
    cudaError_t el = enqueue_run(a, o, S, T.max_h, p->state_a, p->state_b, cap);
    cudaError_t ec = cudaStreamEndCapture(cap, &p->graph);
    e = el != cudaSuccess ? el : ec;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  // the kernel nodes carry the seed by value; a launch after a redraw rewrites it
  p->key = pop->desc.seed;
  size_t n_nodes = 0;
  if (e == cudaSuccess) e = cudaGraphGetNodes(p->graph, nullptr, &n_nodes);
  if (e == cudaSuccess && n_nodes > 0) {
    std::vector<cudaGraphNode_t> all(n_nodes);
    e = cudaGraphGetNodes(p->graph, all.data(), &n_nodes);
    for (size_t j = 0; e == cudaSuccess && j < n_nodes; ++j) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(all[j], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) p->nodes.push_back(all[j]);
    }
  }
  if (e != cudaSuccess) {
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->dev_tab);
    delete p;
    return fail(VCT_ERR_CUDA, "plan capture: %s", cudaGetErrorString(e));
  }
  *plan = p;
  return VCT_OK;
}

vct_status vct_plan_launch(vct_plan *plan, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_plan_launch");
  if (!plan) return fail(VCT_ERR_ARG, "plan is NULL");
  const uint64_t key = plan->pop->desc.seed;
  if (key != plan->key) {
    // the population was redrawn: every simulation node gets the new seed
    for (cudaGraphNode_t node : plan->nodes) {
      cudaKernelNodeParams kp;
      VCT_TRY_CUDA(cudaGraphKernelNodeGetParams(node, &kp));
      vct::SimArgs a = *(const vct::SimArgs *)kp.kernelParams[0];
      vct::set_key(a.pop, key);
      void *args[1] = {&a};
      kp.kernelParams = args;
      kp.extra = nullptr;
      VCT_TRY_CUDA(cudaGraphKernelNodeSetParams(node, &kp));
      VCT_TRY_CUDA(cudaGraphExecKernelNodeSetParams(plan->exec, node, &kp));
    }
    plan->key = key;
  }
  VCT_TRY_CUDA(cudaGraphLaunch(plan->exec, (cudaStream_t)cuda_stream));
  return VCT_OK;
}

vct_status vct_plan_opts(const vct_plan *plan, vct_sim_opts *opts) {
  if (!plan || !opts) return fail(VCT_ERR_ARG, "NULL argument");
  *opts = plan->opts;
  return VCT_OK;
}

vct_status vct_plan_destroy(vct_plan *plan) {
  if (!plan) return VCT_OK;
  cudaError_t e = cudaSuccess;
  if (plan->exec) e = cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->dev_tab) cudaFree(plan->dev_tab);
  delete plan;
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "plan destroy: %s", cudaGetErrorString(e));
  return VCT_OK;
}

}  // extern "C"
