// vct_stats.cu -- population reductions of the per-patient indicators
// (Sec. IV-D: mean TIR, box plot of the TIRs, worst-case patient; Sec. III-C:
// indicators merged after the simulations).
//
// Integer work is exact and order-free: per-patient range counts go into
// per-(scenario, range) histograms over 0..H with integer atomics, and the
// quantiles of the box plot are read off their prefix sums (inverse-CDF
// definition: the smallest count whose cumulative share reaches p).  The
// worst-case patient is the argmin of g_min with ties to the lowest id.  FP64
// sums are reduced in a fixed tree order (per-block shared-memory trees, then
// block partials summed in block order), so repeated calls agree bit for bit.
#include "vct_internal.cuh"

namespace vct {
namespace {

constexpr int kThreads = 256;
constexpr int kP1 = 4;           // FP64 partial sums per block in pass 1

struct ScenAcc {          // integer accumulators of one scenario
  unsigned long long counted, flagged;
  unsigned long long tir_total[VCT_NBINS];
  unsigned long long worst_key, worst_id;
  unsigned below_min[4], below_max[4];  // periods below each range edge
};

struct StatsLayout {
  ScenAcc *acc;           // [S]
  double *part1;          // [S][nblk][kP1]: sum g_mean, basal, bolus, glucagon
  double *part2;          // [S][nblk]: sum (g_mean - mean)^2
  unsigned *hist;         // [sum_s 5 (H_s + 1)]
  vct_population_stats *res;  // [S]
  int nblk;
};

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ bool counted(const vct_patient_stats &p) { return p.status == 0; }

template <int N>
__device__ void block_sum(double (&v)[N], double (*sh)[kThreads]) {
#pragma unroll
  for (int j = 0; j < N; ++j) sh[j][threadIdx.x] = v[j];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int j = 0; j < N; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < N; ++j) v[j] = sh[j][0];
}

__global__ void __launch_bounds__(kThreads) pass1(const vct_patient_stats *in, int64_t n,
                                                  const int64_t *hist_off,
                                                  const int64_t *horizon, StatsLayout L) {
  __shared__ double sh[kP1][kThreads];
  const int s = blockIdx.y;
  const int64_t chunk = (n + L.nblk - 1) / L.nblk;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
  const int64_t H = horizon[s];
  unsigned *hist = L.hist + hist_off[s];
  ScenAcc &acc = L.acc[s];
  double v[kP1] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long c = 0, f = 0, t[VCT_NBINS] = {0, 0, 0, 0, 0};
  unsigned long long wk = ~0ull;
  unsigned bmin[4] = {~0u, ~0u, ~0u, ~0u}, bmax[4] = {0u, 0u, 0u, 0u};
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const vct_patient_stats p = in[(int64_t)s * n + i];
    if (!counted(p)) {
      ++f;
      continue;
    }
    ++c;
    v[0] += p.g_mean;
    v[1] += p.basal_u;
    v[2] += p.bolus_u;
    v[3] += p.glucagon_ug;
#pragma unroll
    for (int b = 0; b < VCT_NBINS; ++b) {
      t[b] += p.tir[b];
      const int64_t cnt = min((int64_t)p.tir[b], H);
      atomicAdd(hist + b * (H + 1) + cnt, 1u);
    }
    wk = min(wk, ordered_bits(p.g_min));
    unsigned cum = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      cum += p.tir[e];
      bmin[e] = min(bmin[e], cum);
      bmax[e] = max(bmax[e], cum);
    }
  }
  if (c) atomicAdd(&acc.counted, c);
  if (f) atomicAdd(&acc.flagged, f);
#pragma unroll
  for (int b = 0; b < VCT_NBINS; ++b)
    if (t[b]) atomicAdd(&acc.tir_total[b], t[b]);
  if (wk != ~0ull) atomicMin(&acc.worst_key, wk);
  if (c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      atomicMin(&acc.below_min[e], bmin[e]);
      atomicMax(&acc.below_max[e], bmax[e]);
    }
  block_sum<kP1>(v, sh);
  if (threadIdx.x == 0)
    for (int j = 0; j < kP1; ++j) L.part1[((int64_t)s * L.nblk + blockIdx.x) * kP1 + j] = v[j];
}

__global__ void __launch_bounds__(kThreads) pass2(const vct_patient_stats *in, int64_t n,
                                                  int64_t first, StatsLayout L) {
  __shared__ double sh[1][kThreads];
  const int s = blockIdx.y;
  ScenAcc &acc = L.acc[s];
  const unsigned long long cnt = acc.counted;
  double sum = 0.0;
  for (int b = 0; b < L.nblk; ++b) sum += L.part1[((int64_t)s * L.nblk + b) * kP1];
  const double mean = cnt ? sum / (double)cnt : 0.0;
  const unsigned long long wk = acc.worst_key;
  const int64_t chunk = (n + L.nblk - 1) / L.nblk;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
  double v[1] = {0.0};
  unsigned long long wid = ~0ull;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const vct_patient_stats p = in[(int64_t)s * n + i];
    if (!counted(p)) continue;
    const double d = p.g_mean - mean;
    v[0] = fma(d, d, v[0]);
    if (ordered_bits(p.g_min) == wk) wid = min(wid, (unsigned long long)(first + i));
  }
  if (wid != ~0ull) atomicMin(&acc.worst_id, wid);
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) L.part2[(int64_t)s * L.nblk + blockIdx.x] = v[0];
}

// Smallest count c in [0, H] with #{patients with count <= c} >= rank.
__device__ int64_t hist_rank(const unsigned *h, int64_t H, unsigned long long rank,
                             unsigned long long *sh_sums, int64_t *sh_res) {
  const int64_t len = H + 1;
  const int64_t per = (len + kThreads - 1) / kThreads;
  const int64_t lo = min(len, (int64_t)threadIdx.x * per), hi = min(len, lo + per);
  unsigned long long mine = 0;
  for (int64_t c = lo; c < hi; ++c) mine += h[c];
  sh_sums[threadIdx.x] = mine;
  if (threadIdx.x == 0) *sh_res = H;
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive prefix over the thread chunks
    unsigned long long run = 0;
    for (int t = 0; t < kThreads; ++t) {
      unsigned long long x = sh_sums[t];
      sh_sums[t] = run;
      run += x;
    }
  }
  __syncthreads();
  unsigned long long run = sh_sums[threadIdx.x];
  if (run < rank && run + mine >= rank) {
    for (int64_t c = lo; c < hi; ++c) {
      run += h[c];
      if (run >= rank) {
        *sh_res = c;
        break;
      }
    }
  }
  __syncthreads();
  int64_t r = *sh_res;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) finalize(const int64_t *hist_off,
                                                     const int64_t *horizon, StatsLayout L) {
  __shared__ unsigned long long sh_sums[kThreads];
  __shared__ int64_t sh_res;
  const int s = blockIdx.x;
  const ScenAcc &acc = L.acc[s];
  const int64_t H = horizon[s];
  const unsigned long long n = acc.counted;
  vct_population_stats &r = L.res[s];
  for (int b = 0; b < VCT_NBINS; ++b) {
    const unsigned *h = L.hist + hist_off[s] + b * (H + 1);
    for (int q = 0; q <= 4; ++q) {
      unsigned long long rank = (n * (unsigned long long)q + 3ull) / 4ull;  // ceil(n q / 4)
      if (rank < 1) rank = 1;
      int64_t c = n ? hist_rank(h, H, rank, sh_sums, &sh_res) : 0;
      if (threadIdx.x == 0) r.tir_quantile[b][q] = H > 0 ? (double)c / (double)H : 0.0;
    }
  }
  if (threadIdx.x == 0) {
    double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;
    for (int b = 0; b < L.nblk; ++b) {
      const double *p = L.part1 + ((int64_t)s * L.nblk + b) * kP1;
      s1 += p[0];
      s2 += p[1];
      s3 += p[2];
      s5 += p[3];
      s4 += L.part2[(int64_t)s * L.nblk + b];
    }
    r.n_patients = (int64_t)n;
    r.n_flagged = (int64_t)acc.flagged;
    for (int b = 0; b < VCT_NBINS; ++b) {
      r.tir_total[b] = acc.tir_total[b];
      r.tir_mean[b] = (n && H) ? (double)acc.tir_total[b] / ((double)n * (double)H) : 0.0;
    }
    unsigned long long wk = acc.worst_key;
    unsigned long long bits = (wk >> 63) ? (wk & 0x7fffffffffffffffull) : ~wk;
    r.worst_patient = n ? (int64_t)acc.worst_id : -1;
    r.worst_g_min = n ? __longlong_as_double((long long)bits) : 0.0;
    r.g_mean_mean = n ? s1 / (double)n : 0.0;
    r.g_mean_var = n ? s4 / (double)n : 0.0;
    r.basal_u_mean = n ? s2 / (double)n : 0.0;
    r.bolus_u_mean = n ? s3 / (double)n : 0.0;
    r.glucagon_ug_mean = n ? s5 / (double)n : 0.0;
    r.horizon_periods = H;
    for (int e = 0; e < 4; ++e) {
      r.below_min[e] = n ? acc.below_min[e] : 0u;
      r.below_max[e] = n ? acc.below_max[e] : 0u;
    }
  }
}

__global__ void init_acc(ScenAcc *acc, int S) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  ScenAcc z = {};
  z.worst_key = ~0ull;
  z.worst_id = ~0ull;
  for (int e = 0; e < 4; ++e) z.below_min[e] = ~0u;
  acc[s] = z;
}

int stats_blocks(int64_t n) {
  int64_t nb = (n + 4 * kThreads - 1) / (4 * kThreads);
  return (int)(nb < 1 ? 1 : (nb > 1024 ? 1024 : nb));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

StatsLayout carve(void *scratch, int32_t S, int64_t n, int64_t hist_words, size_t *total) {
  StatsLayout L;
  L.nblk = stats_blocks(n);
  char *p = (char *)scratch;
  size_t off = 0;
  L.acc = (ScenAcc *)(p + off);
  off = align256(off + sizeof(ScenAcc) * S);
  L.part1 = (double *)(p + off);
  off = align256(off + sizeof(double) * kP1 * S * (size_t)L.nblk);
  L.part2 = (double *)(p + off);
  off = align256(off + sizeof(double) * S * (size_t)L.nblk);
  L.res = (vct_population_stats *)(p + off);
  off = align256(off + sizeof(vct_population_stats) * S);
  L.hist = (unsigned *)(p + off);
  off = align256(off + sizeof(unsigned) * (size_t)hist_words);
  *total = off;
  return L;
}

}  // namespace

size_t stats_scratch_bytes(int32_t n_scen, int64_t n_patients, int64_t hist_words) {
  size_t total = 0;
  carve(nullptr, n_scen, n_patients, hist_words, &total);
  return total;
}

// scratch must hold stats_scratch_bytes(); the first 8 * n_scen int64 words
// after the results are the histogram offsets and horizons, staged by the caller
// in dev_hist_off[0..S) and dev_hist_off[S..2S).  Results land in the
// vct_population_stats array returned through the scratch layout.
cudaError_t launch_stats(const vct_patient_stats *in, int32_t n_scen, int64_t n_patients,
                         const int64_t *dev_hist_off, int64_t hist_words, void *scratch,
                         size_t scratch_bytes, cudaStream_t st) {
  size_t need = 0;
  StatsLayout L = carve(scratch, n_scen, n_patients, hist_words, &need);
  if (need > scratch_bytes) return cudaErrorInvalidValue;
  const int64_t *horizon = dev_hist_off + n_scen;
  init_acc<<<(n_scen + 127) / 128, 128, 0, st>>>(L.acc, n_scen);
  cudaError_t e = cudaMemsetAsync(L.hist, 0, sizeof(unsigned) * (size_t)hist_words, st);
  if (e != cudaSuccess) return e;
  dim3 g(L.nblk, n_scen);
  pass1<<<g, kThreads, 0, st>>>(in, n_patients, dev_hist_off, horizon, L);
  // first patient id is folded into the worst id by the host (ids are local here)
  pass2<<<g, kThreads, 0, st>>>(in, n_patients, 0, L);
  finalize<<<n_scen, kThreads, 0, st>>>(dev_hist_off, horizon, L);
  return cudaGetLastError();
}

// Device address of the results inside a scratch block laid out by launch_stats.
vct_population_stats *stats_results(void *scratch, int32_t n_scen, int64_t n_patients,
                                    int64_t hist_words) {
  size_t total = 0;
  return carve(scratch, n_scen, n_patients, hist_words, &total).res;
}

}  // namespace vct

// ---------------------------------------------------------------------------
// vct_stats_noalloc: the population reductions of vct_stats without any
// allocation.  Its scratch (histograms, partial sums, results, the offset
// table) lives in one fixed array in device memory, defined below; every GPU
// that loads this library keeps that array until the process exits.
// ---------------------------------------------------------------------------
#include <cstdio>
#include <mutex>
#include <vector>

namespace {

constexpr size_t kNoAllocScratchBytes = VCT_STATS_NOALLOC_BYTES;  // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Host code may not use g_noalloc_scratch as a pointer: on the host that name
// is a stand-in, not the device address.  The address is asked of the runtime
// once per device, with that device current, and cached.
vct_status noalloc_scratch(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "vct_stats_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return vct::record_error(VCT_ERR_CUDA, msg);
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char msg[256];
      snprintf(msg, sizeof(msg), "vct_stats_noalloc: cudaGetSymbolAddress: %s",
               cudaGetErrorString(e));
      return vct::record_error(VCT_ERR_CUDA, msg);
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return VCT_OK;
}

}  // namespace

extern "C" vct_status vct_stats_noalloc(const vct_patient_stats *dev_stats, int32_t n_scen,
                                        int64_t n_patients, const int64_t *horizons,
                                        int64_t first_patient, vct_population_stats *host_out,
                                        void *cuda_stream) {
  if (n_scen < 0 || n_patients < 0)
    return vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: negative size");
  if (n_scen == 0) return VCT_OK;
  if (!horizons || !host_out) return vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: NULL argument");
  if (n_patients > 0 && !dev_stats)
    return vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: dev_stats is NULL");
  std::vector<int64_t> meta((size_t)2 * n_scen);
  int64_t words = 0;
  for (int s = 0; s < n_scen; ++s) {
    if (horizons[s] < 0 || horizons[s] >= ((int64_t)1 << 32))
      return vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: horizon out of range");
    meta[s] = words;
    meta[n_scen + s] = horizons[s];
    words += (int64_t)VCT_NBINS * (horizons[s] + 1);
  }
  const int64_t np = n_patients > 0 ? n_patients : 1;
  const size_t need = vct::stats_scratch_bytes(n_scen, np, words);
  const size_t meta_bytes = sizeof(int64_t) * meta.size();
  if (need + meta_bytes > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "vct_stats_noalloc: needs %zu bytes of scratch, the static array holds %zu "
             "(use vct_stats)", need + meta_bytes, kNoAllocScratchBytes);
    return vct::record_error(VCT_ERR_ARG, msg);
  }
  void *scratch = nullptr;
  vct_status rc = noalloc_scratch(&scratch);
  if (rc != VCT_OK) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t *dmeta = (int64_t *)((char *)scratch + need);
  cudaError_t e = cudaMemcpyAsync(dmeta, meta.data(), meta_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = vct::launch_stats(dev_stats, n_scen, n_patients, dmeta, words, scratch, need, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_out, vct::stats_results(scratch, n_scen, np, words),
                        sizeof(vct_population_stats) * n_scen, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "vct_stats_noalloc: %s", cudaGetErrorString(e));
    return vct::record_error(VCT_ERR_CUDA, msg);
  }
  for (int s = 0; s < n_scen; ++s)
    if (host_out[s].worst_patient >= 0) host_out[s].worst_patient += first_patient;
  return VCT_OK;
}
