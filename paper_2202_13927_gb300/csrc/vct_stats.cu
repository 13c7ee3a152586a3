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

// Block sum in a fixed order: a butterfly of warp shuffles within each warp,
// the warps' partials through shared memory, then the same butterfly over them
// in warp 0 (every call adds the same numbers in the same order).
template <int N>
__device__ void block_sum(double (&v)[N], double (*sh)[kThreads / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < N; ++j) sh[j][warp] = v[j];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double x = lane < kThreads / 32 ? sh[j][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[j] = x;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) pass1(const vct_patient_stats *in, int64_t n,
                                                  const int64_t *hist_off,
                                                  const int64_t *horizon, StatsLayout L) {
  __shared__ double sh[kP1][kThreads / 32];
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
  __shared__ double sh[1][kThreads / 32];
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
  if (threadIdx.x == 0) *sh_res = H;
  // exclusive prefix over the thread chunks: a warp-shuffle scan per warp, the
  // warp totals scanned by warp 0
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) sh_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < kThreads / 32 ? sh_sums[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh_sums[32 + lane] = w;  // inclusive over the warps
  }
  __syncthreads();
  unsigned long long run = inc - mine + (warp > 0 ? sh_sums[32 + warp - 1] : 0ull);
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
  __shared__ unsigned long long sh_sums[64];
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

namespace {

// ---------------------------------------------------------------------------
// Population views of Figs. 3 and 5 from the histograms the simulation fills:
// a running count per scenario (and dose), taken with a block-wide scan built
// from warp shuffles, exact in 64-bit integers.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;  // one thread per bin: >= VCT_BG_BINS and VCT_DOSE_BINS
static_assert(kScanThreads >= VCT_BG_BINS && kScanThreads >= VCT_DOSE_BINS, "one thread per bin");

// Inclusive prefix sum of one value per thread: every warp scans its 32
// values with shuffles, warp 0 scans the warp totals the same way, and each
// thread adds the totals of the warps before its own.
__device__ unsigned long long block_inclusive_scan(unsigned long long v, unsigned long long *sh_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < (int)(blockDim.x >> 5) ? sh_warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh_warp[lane] = w;
  }
  __syncthreads();
  return warp > 0 ? v + sh_warp[warp - 1] : v;
}

// Fig. 3's mean curve: cdf[s][j] = (samples in bins 0..j) / (samples), block s.
__global__ void __launch_bounds__(kScanThreads) bg_cdf_kernel(const uint32_t *hist, double *cdf) {
  __shared__ unsigned long long sh_warp[32];
  __shared__ unsigned long long sh_total;
  const int s = blockIdx.x, j = threadIdx.x;
  const unsigned long long v = j < VCT_BG_BINS ? hist[(int64_t)s * VCT_BG_BINS + j] : 0ull;
  const unsigned long long c = block_inclusive_scan(v, sh_warp);
  if (j == VCT_BG_BINS - 1) sh_total = c;
  __syncthreads();
  const unsigned long long total = sh_total;
  if (j < VCT_BG_BINS) cdf[(int64_t)s * VCT_BG_BINS + j] = total ? (double)c / (double)total : 0.0;
}

struct QuantileArgs {
  double q[VCT_MAX_QUANTILES];
  int32_t n_q;
};

// Fig. 5's quantiles: block (s, dose); the bin b with running count
// c_b >= r > c_{b-1}, r = max(ceil(q N), 1), gives the upper edge (b + 1) w.
__global__ void __launch_bounds__(kScanThreads) dose_quantile_kernel(const uint32_t *hist,
                                                                     const __grid_constant__ QuantileArgs qa,
                                                                     double *out) {
  __shared__ unsigned long long sh_warp[32];
  __shared__ unsigned long long sh_total;
  const int sd = blockIdx.x, j = threadIdx.x;  // sd = s * 3 + dose
  const int dose = sd % 3;
  const double width = dose == 0 ? VCT_DOSE_BASAL_BIN : (dose == 1 ? VCT_DOSE_BOLUS_BIN : VCT_DOSE_GLUCAGON_BIN);
  const unsigned long long v = j < VCT_DOSE_BINS ? hist[(int64_t)sd * VCT_DOSE_BINS + j] : 0ull;
  const unsigned long long c = block_inclusive_scan(v, sh_warp);
  if (j == VCT_DOSE_BINS - 1) sh_total = c;
  __syncthreads();
  const unsigned long long total = sh_total;
  double *o = out + (int64_t)sd * qa.n_q;
  for (int i = 0; i < qa.n_q; ++i) {
    if (total == 0) {
      if (j == 0) o[i] = 0.0;
      continue;
    }
    const double r = fmax(ceil(qa.q[i] * (double)total), 1.0);
    if (j < VCT_DOSE_BINS && (double)c >= r && (double)(c - v) < r) o[i] = (double)(j + 1) * width;
  }
}

}  // namespace

}  // namespace vct

extern "C" vct_status vct_bg_cdf(const uint32_t *dev_bg_hist, int32_t n_scen, double *dev_cdf,
                                 void *cuda_stream) {
  if (n_scen < 0) return vct::record_error(VCT_ERR_ARG, "vct_bg_cdf: n_scen < 0");
  if (n_scen == 0) return VCT_OK;
  if (!dev_bg_hist || !dev_cdf) return vct::record_error(VCT_ERR_ARG, "vct_bg_cdf: NULL argument");
  vct::bg_cdf_kernel<<<n_scen, vct::kScanThreads, 0, (cudaStream_t)cuda_stream>>>(dev_bg_hist, dev_cdf);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vct::record_error(VCT_ERR_CUDA, cudaGetErrorString(e));
  return VCT_OK;
}

extern "C" vct_status vct_dose_quantiles(const uint32_t *dev_dose_hist, int32_t n_scen,
                                         const double *qs, int32_t n_q, double *dev_out,
                                         void *cuda_stream) {
  if (n_scen < 0) return vct::record_error(VCT_ERR_ARG, "vct_dose_quantiles: n_scen < 0");
  if (n_q < 1 || n_q > VCT_MAX_QUANTILES)
    return vct::record_error(VCT_ERR_ARG, "vct_dose_quantiles: n_q must be in 1..VCT_MAX_QUANTILES");
  if (!qs) return vct::record_error(VCT_ERR_ARG, "vct_dose_quantiles: qs is NULL");
  vct::QuantileArgs qa = {};
  qa.n_q = n_q;
  for (int i = 0; i < n_q; ++i) {
    if (!(qs[i] >= 0.0 && qs[i] <= 1.0))
      return vct::record_error(VCT_ERR_ARG, "vct_dose_quantiles: quantiles must lie in [0, 1]");
    qa.q[i] = qs[i];
  }
  if (n_scen == 0) return VCT_OK;
  if (!dev_dose_hist || !dev_out) return vct::record_error(VCT_ERR_ARG, "vct_dose_quantiles: NULL argument");
  vct::dose_quantile_kernel<<<n_scen * 3, vct::kScanThreads, 0, (cudaStream_t)cuda_stream>>>(
      dev_dose_hist, qa, dev_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vct::record_error(VCT_ERR_CUDA, cudaGetErrorString(e));
  return VCT_OK;
}

// ---------------------------------------------------------------------------
// vct_stats_noalloc: the population reductions of vct_stats without any
// allocation.  Its scratch (histograms, partial sums, results, the offset
// table) lives in one fixed array in device memory, defined below; every GPU
// that loads this library keeps that array until the process exits.
// ---------------------------------------------------------------------------
#include <cstdio>
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = VCT_STATS_NOALLOC_BYTES;  // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Host code may not use g_noalloc_scratch as a pointer: on the host that name
// is a stand-in, not the device address.  The address is asked of the runtime
// once per device, with that device current, and cached (valid for the
// device's primary context until the process exits or the device is reset).
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

// Histogram offsets from the horizons, on the device: meta[S + s] holds the
// horizon of scenario s (copied there from the caller's array), meta[s]
// receives the first histogram word of scenario s (5 (H + 1) words each).
// One thread: the table has one entry per scenario.
__global__ void noalloc_offsets(int64_t *meta, int32_t S) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int64_t words = 0;
  for (int32_t s = 0; s < S; ++s) {
    meta[s] = words;
    words += (int64_t)VCT_NBINS * (meta[S + s] + 1);
  }
}

// Bytes of the fixed array a call needs: the layout of vct_stats plus the
// offset table (two int64 per scenario).  0 after an argument error.
size_t noalloc_bytes(int32_t n_scen, int64_t n_patients, const int64_t *horizons, int64_t *words_out,
                     vct_status *rc) {
  *rc = VCT_OK;
  int64_t words = 0;
  for (int32_t s = 0; s < n_scen; ++s) {
    if (horizons[s] < 0 || horizons[s] >= ((int64_t)1 << 32)) {
      *rc = vct::record_error(VCT_ERR_ARG, "vct_stats_noalloc: horizon out of range");
      return 0;
    }
    words += (int64_t)VCT_NBINS * (horizons[s] + 1);
  }
  if (words_out) *words_out = words;
  const int64_t np = n_patients > 0 ? n_patients : 1;
  return vct::stats_scratch_bytes(n_scen, np, words) + sizeof(int64_t) * 2 * (size_t)n_scen;
}

}  // namespace

extern "C" size_t vct_stats_noalloc_bytes(int32_t n_scen, int64_t n_patients,
                                          const int64_t *horizons) {
  if (n_scen <= 0 || n_patients < 0 || !horizons) return 0;
  vct_status rc = VCT_OK;
  const size_t b = noalloc_bytes(n_scen, n_patients, horizons, nullptr, &rc);
  return rc == VCT_OK ? b : 0;
}

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
  int64_t words = 0;
  vct_status rc = VCT_OK;
  const size_t total = noalloc_bytes(n_scen, n_patients, horizons, &words, &rc);
  if (rc != VCT_OK) return rc;
  if (total > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "vct_stats_noalloc: needs %zu bytes of scratch, the static array holds %zu "
             "(use vct_stats)", total, kNoAllocScratchBytes);
    return vct::record_error(VCT_ERR_ARG, msg);
  }
  void *scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch)) != VCT_OK) return rc;
  const int64_t np = n_patients > 0 ? n_patients : 1;
  const size_t need = vct::stats_scratch_bytes(n_scen, np, words);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the offset table sits after the layout of vct_stats: horizons copied from
  // the caller's array, offsets computed from them on the device
  int64_t *dmeta = (int64_t *)((char *)scratch + need);
  cudaError_t e = cudaMemcpyAsync(dmeta + n_scen, horizons, sizeof(int64_t) * (size_t)n_scen,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    noalloc_offsets<<<1, 1, 0, st>>>(dmeta, n_scen);
    e = cudaGetLastError();
  }
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
