// vct_host.cu -- host side of the C-ABI declared in include/vct.h: errors,
// population handles, population reductions, diagnostics.  The simulation
// calls are in vct_run.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vct_internal.cuh"



namespace {

thread_local std::string g_err;

vct_status fail(vct_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define VCT_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? VCT_ERR_OOM : VCT_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                      \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool finite_all(const double *v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

vct_status check_desc(const vct_population_desc *d) {
  if (!d) return fail(VCT_ERR_ARG, "population descriptor is NULL");
  if (d->n_patients < 0) return fail(VCT_ERR_ARG, "n_patients < 0");
  if (d->first_patient < 0 || d->first_patient + d->n_patients > (int64_t)1 << 32)
    return fail(VCT_ERR_ARG, "patient ids must fit in 32 bits (first_patient + n_patients <= 2^32)");
  if (d->max_attempts < 1 || d->max_attempts > 1024)
    return fail(VCT_ERR_ARG, "max_attempts must be in 1..1024");
  if (!finite_all(d->p_mean, VCT_NPARAM) || !finite_all(d->p_sd, VCT_NPARAM) ||
      !std::isfinite(d->bw_mean) || !std::isfinite(d->bw_sd))
    return fail(VCT_ERR_ARG, "non-finite entry in the parameter table");
  for (int j = 0; j < VCT_NPARAM; ++j)
    if (d->p_sd[j] < 0.0) return fail(VCT_ERR_ARG, "p_sd[%d] < 0", j);
  if (d->bw_sd < 0.0 || d->bw_mean <= 0.0) return fail(VCT_ERR_ARG, "body weight mean must be > 0, sd >= 0");
  const int positive[] = {VCT_P_VI, VCT_P_VG, VCT_P_TAUS, VCT_P_TAUD, VCT_P_TAUCGM, VCT_P_KE};
  for (int j : positive)
    if (!(d->p_mean[j] > 0.0)) return fail(VCT_ERR_ARG, "p_mean[%d] must be > 0", j);
  if (!(d->g_sp > 0.0) || !std::isfinite(d->g_sp)) return fail(VCT_ERR_ARG, "g_sp must be > 0");
  if (!(d->sigma_q1 >= 0.0) || !std::isfinite(d->sigma_q1)) return fail(VCT_ERR_ARG, "sigma_q1 must be >= 0");
  if (!(d->cgm_sd >= 0.0) || !std::isfinite(d->cgm_sd)) return fail(VCT_ERR_ARG, "cgm_sd must be >= 0");
  if (!std::isfinite(d->min_basal_u_per_h)) return fail(VCT_ERR_ARG, "min_basal_u_per_h not finite");
  if (!(d->tau_gg_min >= 0.0) || !std::isfinite(d->tau_gg_min) || !(d->s_gg >= 0.0) ||
      !std::isfinite(d->s_gg))
    return fail(VCT_ERR_ARG, "tau_gg_min and s_gg must be finite and >= 0");
  return VCT_OK;
}

vct_status alloc_population(const vct_population_desc *d, vct_population **out) {
  auto *p = new (std::nothrow) vct_population();
  if (!p) return fail(VCT_ERR_OOM, "host allocation failed");
  p->desc = *d;
  p->n = d->n_patients;
  p->n_pad = std::max<int64_t>(32, (d->n_patients + 31) / 32 * 32);
  p->first = d->first_patient;
  cudaGetDevice(&p->device);
  size_t off = 0;
  const size_t o_rows = off;
  off = align256(off + sizeof(double) * VCT_NROW * p->n_pad);
  const size_t o_ub = off;
  off = align256(off + sizeof(double) * p->n_pad);
  const size_t o_x0 = off;
  off = align256(off + sizeof(double) * VCT_NSTATE * p->n_pad);
  const size_t o_st = off;
  off = align256(off + sizeof(uint32_t) * p->n_pad);
  const size_t o_at = off;
  off = align256(off + sizeof(int32_t) * p->n_pad);
  const size_t o_next = off;
  off = align256(off + sizeof(unsigned long long));
  cudaError_t e = cudaMalloc(&p->mem, off);
  if (e != cudaSuccess) {
    delete p;
    return fail(VCT_ERR_OOM, "cudaMalloc(%zu) for the population: %s", off, cudaGetErrorString(e));
  }
  char *b = (char *)p->mem;
  p->rows = (double *)(b + o_rows);
  p->ub = (double *)(b + o_ub);
  p->x0 = (double *)(b + o_x0);
  p->status = (uint32_t *)(b + o_st);
  p->attempts = (int32_t *)(b + o_at);
  p->next = (unsigned long long *)(b + o_next);
  *out = p;
  return VCT_OK;
}

}  // namespace

vct_status vct::record_error(vct_status code, const char *msg) {
  g_err = msg;
  return code;
}

extern "C" {

const char *vct_last_error(void) { return g_err.c_str(); }

const char *vct_version(void) { return "vct-gb300 0.1 (sm_103a)"; }

vct_status vct_create_population(const vct_population_desc *desc, void *cuda_stream,
                                 vct_population **out) {
  vct::NvtxRange nvtx_range_("vct_create_population");
  if (!out) return fail(VCT_ERR_ARG, "out is NULL");
  *out = nullptr;
  vct_status rc = check_desc(desc);
  if (rc) return rc;
  vct_population *p = nullptr;
  if ((rc = alloc_population(desc, &p))) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = vct::launch_population(*desc, p->rows, p->ub, p->x0, p->status, p->attempts,
                                         p->n_pad, p->next, st);
  std::vector<uint32_t> status((size_t)p->n);
  if (e == cudaSuccess && p->n)
    e = cudaMemcpyAsync(status.data(), p->status, sizeof(uint32_t) * p->n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(p->mem);
    delete p;
    return fail(VCT_ERR_CUDA, "population kernel: %s", cudaGetErrorString(e));
  }
  p->n_rejected = std::count_if(status.begin(), status.end(), [](uint32_t s) { return s != 0; });
  *out = p;
  return VCT_OK;
}

vct_status vct_population_redraw(vct_population *pop, uint64_t seed, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_population_redraw");
  if (!pop) return fail(VCT_ERR_ARG, "population is NULL");
  pop->desc.seed = seed;
  cudaError_t e = vct::launch_population(pop->desc, pop->rows, pop->ub, pop->x0, pop->status,
                                         pop->attempts, pop->n_pad, pop->next,
                                         (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "population kernel: %s", cudaGetErrorString(e));
  pop->n_rejected = -1;  // counted again by vct_population_info_get
  return VCT_OK;
}

vct_status vct_population_from_host(const vct_population_desc *desc, const double *rows,
                                    const double *u_b, const double *x0, void *cuda_stream,
                                    vct_population **out) {
  if (!out || !rows || !u_b || !x0) return fail(VCT_ERR_ARG, "NULL argument");
  *out = nullptr;
  vct_status rc = check_desc(desc);
  if (rc) return rc;
  vct_population *p = nullptr;
  if ((rc = alloc_population(desc, &p))) return rc;
  const int64_t n = p->n, np = p->n_pad;
  std::vector<double> r((size_t)VCT_NROW * np, 0.0), x((size_t)VCT_NSTATE * np, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    for (int j = 0; j < VCT_NROW; ++j) r[(size_t)j * np + i] = rows[i * VCT_NROW + j];
    for (int j = 0; j < VCT_NSTATE; ++j) x[(size_t)j * np + i] = x0[i * VCT_NSTATE + j];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(p->rows, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->x0, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n)
    e = cudaMemcpyAsync(p->ub, u_b, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(uint32_t) * np, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->attempts, 0, sizeof(int32_t) * np, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(p->mem);
    delete p;
    return fail(VCT_ERR_CUDA, "population upload: %s", cudaGetErrorString(e));
  }
  p->n_rejected = 0;
  *out = p;
  return VCT_OK;
}

vct_status vct_destroy_population(vct_population *pop) {
  if (!pop) return VCT_OK;
  cudaError_t e = cudaFree(pop->mem);
  delete pop;
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
  return VCT_OK;
}

vct_status vct_population_info_get(const vct_population *pop, vct_population_info *info) {
  if (!pop || !info) return fail(VCT_ERR_ARG, "NULL argument");
  info->n_patients = pop->n;
  info->first_patient = pop->first;
  if (pop->n_rejected < 0) {
    std::vector<uint32_t> status((size_t)pop->n);
    if (pop->n) {
      cudaError_t e = cudaMemcpy(status.data(), pop->status, sizeof(uint32_t) * pop->n,
                                 cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "status copy: %s", cudaGetErrorString(e));
    }
    const_cast<vct_population *>(pop)->n_rejected =
        std::count_if(status.begin(), status.end(), [](uint32_t s) { return s != 0; });
  }
  info->n_rejected = pop->n_rejected;
  info->dev_rows = pop->rows;
  info->dev_u_b = pop->ub;
  info->dev_x0 = pop->x0;
  info->dev_status = pop->status;
  info->dev_attempts = pop->attempts;
  info->n_pad = pop->n_pad;
  return VCT_OK;
}

vct_status vct_population_export(const vct_population *pop, double *rows, double *u_b, double *x0,
                                 uint32_t *status, int32_t *attempts) {
  if (!pop) return fail(VCT_ERR_ARG, "population is NULL");
  const int64_t n = pop->n, np = pop->n_pad;
  if (rows) {
    std::vector<double> r((size_t)VCT_NROW * np);
    VCT_CUDA(cudaMemcpy(r.data(), pop->rows, sizeof(double) * r.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < VCT_NROW; ++j) rows[i * VCT_NROW + j] = r[(size_t)j * np + i];
  }
  if (x0) {
    std::vector<double> x((size_t)VCT_NSTATE * np);
    VCT_CUDA(cudaMemcpy(x.data(), pop->x0, sizeof(double) * x.size(), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < VCT_NSTATE; ++j) x0[i * VCT_NSTATE + j] = x[(size_t)j * np + i];
  }
  if (u_b && n) VCT_CUDA(cudaMemcpy(u_b, pop->ub, sizeof(double) * n, cudaMemcpyDeviceToHost));
  if (status && n) VCT_CUDA(cudaMemcpy(status, pop->status, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost));
  if (attempts && n)
    VCT_CUDA(cudaMemcpy(attempts, pop->attempts, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  return VCT_OK;
}

size_t vct_state_bytes(int32_t n_scen, int64_t n_patients) {
  if (n_scen <= 0 || n_patients <= 0) return 0;
  return (size_t)n_scen * (size_t)n_patients *
         (sizeof(double) * vct::kStateDoubles + sizeof(uint32_t) * vct::kStateWords);
}

vct_status vct_stats(const vct_patient_stats *dev_stats, int32_t n_scen, int64_t n_patients,
                     const int64_t *horizons, int64_t first_patient,
                     vct_population_stats *host_out, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_stats");
  if (n_scen < 0 || n_patients < 0) return fail(VCT_ERR_ARG, "negative size");
  if (n_scen == 0) return VCT_OK;
  if (!horizons || !host_out) return fail(VCT_ERR_ARG, "NULL argument");
  if (n_patients > 0 && !dev_stats) return fail(VCT_ERR_ARG, "dev_stats is NULL");
  std::vector<int64_t> meta((size_t)2 * n_scen);
  int64_t words = 0;
  for (int s = 0; s < n_scen; ++s) {
    if (horizons[s] < 0 || horizons[s] >= ((int64_t)1 << 32))
      return fail(VCT_ERR_ARG, "horizon of scenario %d out of range", s);
    meta[s] = words;
    meta[n_scen + s] = horizons[s];
    words += (int64_t)VCT_NBINS * (horizons[s] + 1);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t need = vct::stats_scratch_bytes(n_scen, std::max<int64_t>(n_patients, 1), words);
  const size_t meta_bytes = align256(sizeof(int64_t) * meta.size());
  void *scratch = nullptr;
  VCT_CUDA(cudaMallocAsync(&scratch, need + meta_bytes, st));
  int64_t *dmeta = (int64_t *)((char *)scratch + need);
  cudaError_t e = cudaMemcpyAsync(dmeta, meta.data(), sizeof(int64_t) * meta.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = vct::launch_stats(dev_stats, n_scen, n_patients, dmeta, words, scratch, need, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, vct::stats_results(scratch, n_scen, std::max<int64_t>(n_patients, 1), words),
                        sizeof(vct_population_stats) * n_scen, cudaMemcpyDeviceToHost, st);
  cudaError_t ef = cudaFreeAsync(scratch, st);
  if (e == cudaSuccess) e = ef;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "vct_stats: %s", cudaGetErrorString(e));
  for (int s = 0; s < n_scen; ++s)
    if (host_out[s].worst_patient >= 0) host_out[s].worst_patient += first_patient;
  return VCT_OK;
}

size_t vct_stats_workspace_bytes(int32_t n_scen, int64_t n_patients, const int64_t *horizons) {
  return vct_stats_noalloc_bytes(n_scen, n_patients, horizons);
}

vct_status vct_stats_with_workspace(const vct_patient_stats *dev_stats, int32_t n_scen,
                                    int64_t n_patients, const int64_t *horizons,
                                    int64_t first_patient, void *dev_workspace,
                                    size_t workspace_bytes, vct_population_stats *host_out,
                                    void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_stats_with_workspace");
  if (n_scen < 0 || n_patients < 0) return fail(VCT_ERR_ARG, "negative size");
  if (n_scen == 0) return VCT_OK;
  if (!horizons || !host_out) return fail(VCT_ERR_ARG, "NULL argument");
  if (n_patients > 0 && !dev_stats) return fail(VCT_ERR_ARG, "dev_stats is NULL");
  if (!dev_workspace) return fail(VCT_ERR_ARG, "dev_workspace is NULL");
  if ((uintptr_t)dev_workspace % 256 != 0) return fail(VCT_ERR_ARG, "dev_workspace must be 256-byte aligned");
  std::vector<int64_t> meta((size_t)2 * n_scen);
  int64_t words = 0;
  for (int s = 0; s < n_scen; ++s) {
    if (horizons[s] < 0 || horizons[s] >= ((int64_t)1 << 32))
      return fail(VCT_ERR_ARG, "horizon of scenario %d out of range", s);
    meta[s] = words;
    meta[n_scen + s] = horizons[s];
    words += (int64_t)VCT_NBINS * (horizons[s] + 1);
  }
  const int64_t np = std::max<int64_t>(n_patients, 1);
  const size_t need = vct::stats_scratch_bytes(n_scen, np, words);
  const size_t meta_bytes = sizeof(int64_t) * meta.size();
  if (workspace_bytes < need + meta_bytes)
    return fail(VCT_ERR_ARG, "workspace of %zu bytes, the call needs %zu (vct_stats_workspace_bytes)",
                workspace_bytes, need + meta_bytes);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t *dmeta = (int64_t *)((char *)dev_workspace + need);
  cudaError_t e = cudaMemcpyAsync(dmeta, meta.data(), meta_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = vct::launch_stats(dev_stats, n_scen, n_patients, dmeta, words, dev_workspace, need, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, vct::stats_results(dev_workspace, n_scen, np, words),
                        sizeof(vct_population_stats) * n_scen, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "vct_stats_with_workspace: %s", cudaGetErrorString(e));
  for (int s = 0; s < n_scen; ++s)
    if (host_out[s].worst_patient >= 0) host_out[s].worst_patient += first_patient;
  return VCT_OK;
}

vct_status vct_sync(void *cuda_stream) {
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(VCT_ERR_CUDA, "asynchronous error: %s", cudaGetErrorString(e));
  return VCT_OK;
}

vct_status vct_philox_fill(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *out_words,
                           void *out_normals, int32_t precision, void *cuda_stream) {
  if (n < 0) return fail(VCT_ERR_ARG, "n < 0");
  if (n > 0 && !ctr) return fail(VCT_ERR_ARG, "ctr is NULL");
  if (precision != VCT_FP64 && precision != VCT_FP32 && precision != VCT_FP64_LIBRARY)
    return fail(VCT_ERR_ARG, "bad precision");
  VCT_CUDA(vct::launch_philox_fill(ctr, n, seed, out_words, out_normals, precision,
                                   (cudaStream_t)cuda_stream));
  return VCT_OK;
}

vct_status vct_box_muller_words(const uint32_t *dev_words, int64_t n, int32_t mode, double *dev_z,
                                void *cuda_stream) {
  if (n < 0) return fail(VCT_ERR_ARG, "n < 0");
  if (mode != 0 && mode != 1) return fail(VCT_ERR_ARG, "mode must be 0 or 1");
  if (n > 0 && (!dev_words || !dev_z)) return fail(VCT_ERR_ARG, "NULL argument");
  VCT_CUDA(vct::launch_box_muller_words(dev_words, n, mode, dev_z, (cudaStream_t)cuda_stream));
  return VCT_OK;
}

size_t vct_struct_size(const char *name) {
  if (!name) return 0;
  if (!std::strcmp(name, "vct_population_desc")) return sizeof(vct_population_desc);
  if (!std::strcmp(name, "vct_scenario")) return sizeof(vct_scenario);
  if (!std::strcmp(name, "vct_sim_opts")) return sizeof(vct_sim_opts);
  if (!std::strcmp(name, "vct_patient_stats")) return sizeof(vct_patient_stats);
  if (!std::strcmp(name, "vct_population_stats")) return sizeof(vct_population_stats);
  if (!std::strcmp(name, "vct_population_info")) return sizeof(vct_population_info);
  if (!std::strcmp(name, "vct_surrogate_desc")) return sizeof(vct_surrogate_desc);
  if (!std::strcmp(name, "vct_day_plan")) return sizeof(vct_day_plan);
  return 0;
}

}  // extern "C"
