// vct_pop.cu -- population draw and FP64 basal steady state (Sec. IV-B).
//
// Parameter j is drawn as mean + sd z with z the next normal of its own
// Philox sequence that satisfies |z| <= 1 (within one standard deviation) and
// gives a nonnegative value; the set is kept when the basal steady state at
// the setpoint exists and needs at least the minimum basal rate, else the next
// set attempt is drawn.  FP64 throughout.
//
// Work layout: a grid of resident CTAs; every lane takes its next patient
// from a device counter when the current one is decided, and each trip of the
// lane's loop evaluates one Box-Muller pair.  Set-level rejection (about two
// attempts per patient on average, up to six for the slowest lane of a warp)
// and the per-parameter acceptance thus keep the lanes of a warp on the same
// instruction instead of waiting for the slowest of 32 patients.  Every
// result is a function of the global patient id alone, so the order in which
// lanes take patients does not change it.
#include <algorithm>

#include "vct_internal.cuh"
#include "vct_rng.cuh"

namespace vct {
namespace {

constexpr int kPopBlock = 32;  // one warp: a small cohort still spreads over many SMs

struct PopKernelArgs {
  vct_population_desc d;
  double *rows, *ub, *x0;
  uint32_t *status;
  int32_t *attempts;
  int64_t n_pad;
  unsigned long long *next;
};

// Residual of the steady-state condition on plasma insulin I at G = G_sp:
// dQ1/dt with every other state at its equilibrium for that I (Hovorka 2004):
//   EGP0 BW (1 - S_IE I) - F01c - F_R - Q1 S_IT I S_ID I / (k12 + S_ID I).
__device__ double basal_residual(const double *p, double g_sp, double i) {
  double bw = p[VCT_P_BW];
  double q1 = g_sp * p[VCT_P_VG] * bw;
  double f01c = p[VCT_P_F01] * bw * fmin(1.0, g_sp / 4.5);
  double f_r = fmax(0.0, 0.003 * (g_sp - 9.0) * p[VCT_P_VG] * bw);
  double x1 = p[VCT_P_SIT] * i, x2 = p[VCT_P_SID] * i, x3 = p[VCT_P_SIE] * i;
  return p[VCT_P_EGP0] * bw * (1.0 - x3) - f01c - f_r - q1 * x1 * x2 / (p[VCT_P_K12] + x2);
}

// The residual is strictly decreasing on I >= 0, positive at 0 (checked) and
// not positive at 1/S_IE.  Multiplied by k12 + S_ID I > 0 it is the quadratic
//   c0 + b1 I - a2 I^2,  a2 = B S_ID + C,  b1 = A S_ID - B k12,  c0 = A k12 > 0,
// with A = EGP0 BW - F01c - F_R, B = EGP0 BW S_IE, C = Q1 S_IT S_ID, whose
// one nonnegative root is taken in the form without cancellation:
//   I = (b1 + sqrt(D)) / (2 a2) for b1 >= 0,  I = 2 c0 / (sqrt(D) - b1) else,
// D = b1^2 + 4 a2 c0 (a sum of nonnegative terms).  Then every state follows.
__device__ bool basal_state(const double *p, double g_sp, double &ub, double x[VCT_NSTATE]) {
  for (int j = 0; j < VCT_NROW; ++j)
    if (!isfinite(p[j])) return false;
  if (!(p[VCT_P_SIE] > 0.0)) return false;
  const double hi = 1.0 / p[VCT_P_SIE];
  if (!(basal_residual(p, g_sp, 0.0) > 0.0)) return false;
  const double bw = p[VCT_P_BW];
  const double q1 = g_sp * p[VCT_P_VG] * bw;
  double i_ss;
  {
    const double f01c = p[VCT_P_F01] * bw * fmin(1.0, g_sp / 4.5);
    const double f_r = fmax(0.0, 0.003 * (g_sp - 9.0) * p[VCT_P_VG] * bw);
    const double A = p[VCT_P_EGP0] * bw - f01c - f_r, B = p[VCT_P_EGP0] * bw * p[VCT_P_SIE];
    const double C = q1 * p[VCT_P_SIT] * p[VCT_P_SID], k12 = p[VCT_P_K12], sid = p[VCT_P_SID];
    const double a2 = B * sid + C, b1 = A * sid - B * k12, c0 = A * k12;
    const double sd = sqrt(b1 * b1 + 4.0 * a2 * c0);
    i_ss = b1 >= 0.0 ? (b1 + sd) / (2.0 * a2) : (2.0 * c0) / (sd - b1);
    // no root below 1/S_IE only when the residual never turns (a2 = 0, b1 >= 0):
    // the steady state is then the interval's end
    if (!(i_ss <= hi)) i_ss = hi;
  }
  ub = i_ss * p[VCT_P_VI] * bw * p[VCT_P_KE];
  double x1 = p[VCT_P_SIT] * i_ss, x2 = p[VCT_P_SID] * i_ss;
  x[0] = 0.0;                 // D1
  x[1] = 0.0;                 // D2
  x[2] = ub * p[VCT_P_TAUS];  // S1
  x[3] = ub * p[VCT_P_TAUS];  // S2
  x[4] = i_ss;                // I
  x[5] = x1;
  x[6] = x2;
  x[7] = p[VCT_P_SIE] * i_ss;
  x[8] = q1;
  x[9] = x1 * q1 / (p[VCT_P_K12] + x2);
  x[10] = g_sp;               // CGM at rest reads the plasma value
  return true;
}

__device__ __forceinline__ double row_mean(const vct_population_desc &d, int j) {
  return j < VCT_NPARAM ? d.p_mean[j] : d.bw_mean;
}
__device__ __forceinline__ double row_sd(const vct_population_desc &d, int j) {
  return j < VCT_NPARAM ? d.p_sd[j] : d.bw_sd;
}

// The draw of parameter j of set s: Philox call t of counter (s, pid, 256 j + t,
// PARAM) gives the normals 4t .. 4t + 3 (two Box-Muller pairs), tried in order;
// the first acceptable one is kept; 16 calls without one fail the set.
__global__ void __launch_bounds__(kPopBlock) population_kernel(PopKernelArgs a) {
  __shared__ double sp[VCT_NROW][kPopBlock];  // the lane's current parameter set
  const int t = threadIdx.x;
  const vct_population_desc &d = a.d;
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  const unsigned long long n = (unsigned long long)d.n_patients;
  const uint32_t max_sets = (uint32_t)d.max_attempts;

  // the next parameter to draw at or after `from` (fixed ones are set directly)
  auto skip_fixed = [&](int from) {
    int j = from;
    while (j < VCT_NROW && row_sd(d, j) == 0.0) {
      sp[j][t] = row_mean(d, j);
      ++j;
    }
    return j;
  };

  unsigned long long i = atomicAdd(a.next, 1ull);
  uint32_t pid = 0, set = 0, call = 0;
  int j = VCT_NROW;
  bool second = false;  // the call's second Box-Muller pair is next
  Words4 w{0u, 0u, 0u, 0u};
  if (i < n) {
    pid = (uint32_t)(d.first_patient + (int64_t)i);
    for (int q = 0; q < VCT_NROW; ++q) sp[q][t] = 0.0;
    j = skip_fixed(0);
  }
  while (i < n) {
    bool decided = j >= VCT_NROW;  // the set is complete (every parameter fixed)
    bool drawn = decided;
    if (!decided) {
      const double mean = row_mean(d, j), sd = row_sd(d, j);
      if (!second) w = philox4x32_10(Words4{set, pid, (uint32_t)j * 256u + call, kTagParam}, k0, k1);
      double z0, z1;
      box_muller_f64(second ? w.c : w.a, second ? w.d : w.b, z0, z1);
      const double v0 = mean + sd * z0, v1 = mean + sd * z1;
      const bool ok0 = fabs(z0) <= 1.0 && v0 >= 0.0, ok1 = fabs(z1) <= 1.0 && v1 >= 0.0;
      if (ok0 || ok1) {
        sp[j][t] = ok0 ? v0 : v1;
        j = skip_fixed(j + 1);
        call = 0;
        second = false;
        decided = drawn = j >= VCT_NROW;
      } else if (!second) {
        second = true;
      } else {
        second = false;
        if (++call == 16u) decided = true;  // no acceptable draw: the set fails
      }
    }
    if (!decided) continue;
    double p[VCT_NROW], x[VCT_NSTATE], u = 0.0;
#pragma unroll
    for (int q = 0; q < VCT_NROW; ++q) p[q] = sp[q][t];
    const bool kept = drawn && basal_state(p, d.g_sp, u, x) && !(u * 60.0 / 1000.0 < d.min_basal_u_per_h);
    if (!kept && set + 1u < max_sets) {  // the next set attempt
      ++set;
      j = skip_fixed(0);
      call = 0;
      second = false;
      continue;
    }
    // decided: write the patient (a rejected one keeps the last values drawn)
    if (!kept) {
      u = 0.0;
#pragma unroll
      for (int q = 0; q < VCT_NSTATE; ++q) x[q] = 0.0;
    }
#pragma unroll
    for (int q = 0; q < VCT_NROW; ++q) a.rows[q * a.n_pad + (int64_t)i] = p[q];
#pragma unroll
    for (int q = 0; q < VCT_NSTATE; ++q) a.x0[q * a.n_pad + (int64_t)i] = x[q];
    a.ub[i] = u;
    a.status[i] = kept ? 0u : VCT_PATIENT_REJECTED;
    a.attempts[i] = kept ? (int32_t)(set + 1u) : d.max_attempts;
    i = atomicAdd(a.next, 1ull);
    if (i < n) {
      pid = (uint32_t)(d.first_patient + (int64_t)i);
      set = 0;
      call = 0;
      second = false;
#pragma unroll
      for (int q = 0; q < VCT_NROW; ++q) sp[q][t] = 0.0;
      j = skip_fixed(0);
    }
  }
}

__global__ void philox_fill_kernel(const uint32_t *ctr, int64_t n, uint32_t k0, uint32_t k1,
                                   uint32_t *words, void *normals, int precision) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Words4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  Words4 w = philox4x32_10(c, k0, k1);
  // the factorised first round of the simulation loop must agree with the plain one
  PhiloxLane lane = make_lane(c.b, c.c, k0, k1);
  Words4 w2 = lane.call(__umulhi(kPhiloxM0, c.a), kPhiloxM0 * c.a, c.d);
  if (w2.a != w.a || w2.b != w.b || w2.c != w.c || w2.d != w.d) w.a = w.b = w.c = w.d = 0u;
  // and so must the form with precomputed round keys
  uint32_t rk[kPhiloxRoundKeys];
  philox_round_keys((uint64_t)k0 | ((uint64_t)k1 << 32), rk);
  Words4 w3 = PhiloxLaneRk{lane.w0, lane.w1, rk}.call(__umulhi(kPhiloxM0, c.a), kPhiloxM0 * c.a, c.d);
  if (w3.a != w.a || w3.b != w.b || w3.c != w.c || w3.d != w.d) w.a = w.b = w.c = w.d = 0u;
  if (words) {
    words[4 * i] = w.a;
    words[4 * i + 1] = w.b;
    words[4 * i + 2] = w.c;
    words[4 * i + 3] = w.d;
  }
  if (normals) {
    if (precision == VCT_FP64) {          // the simulation's own FP64 transform
      double *z = (double *)normals + 4 * i;
      box_muller_f64t(w.a, w.b, z[0], z[1]);
      box_muller_f64t(w.c, w.d, z[2], z[3]);
    } else if (precision == VCT_FP64_LIBRARY) {   // the CUDA library's log, sqrt, sincospi
      double *z = (double *)normals + 4 * i;
      box_muller_f64(w.a, w.b, z[0], z[1]);
      box_muller_f64(w.c, w.d, z[2], z[3]);
    } else {
      float *z = (float *)normals + 4 * i;
      box_muller_f32(w.a, w.b, z[0], z[1]);
      box_muller_f32(w.c, w.d, z[2], z[3]);
    }
  }
}

}  // namespace

cudaError_t launch_population(const vct_population_desc &d, double *rows, double *ub, double *x0,
                              uint32_t *status, int32_t *attempts, int64_t n_pad,
                              unsigned long long *next, cudaStream_t st) {
  if (d.n_patients <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, population_kernel, kPopBlock, 0)) !=
      cudaSuccess)
    return e;
  const int64_t resident = (int64_t)std::max(sms, 1) * std::max(per_sm, 1);
  const int64_t blocks = std::min<int64_t>((d.n_patients + kPopBlock - 1) / kPopBlock, resident);
  PopKernelArgs a{d, rows, ub, x0, status, attempts, n_pad, next};
  population_kernel<<<(unsigned)blocks, kPopBlock, 0, st>>>(a);
  return cudaGetLastError();
}

namespace {
// Box-Muller on given word pairs (the transform alone, any words)
__global__ void box_muller_words_kernel(const uint32_t *words, int64_t n, int mode, double *z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t w0 = words[2 * i], w1 = words[2 * i + 1];
  if (mode == 0)
    box_muller_f64t(w0, w1, z[2 * i], z[2 * i + 1]);
  else
    box_muller_f64(w0, w1, z[2 * i], z[2 * i + 1]);
}
}  // namespace

cudaError_t launch_box_muller_words(const uint32_t *words, int64_t n, int mode, double *z,
                                    cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  box_muller_words_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(words, n, mode, z);
  return cudaGetLastError();
}

cudaError_t launch_philox_fill(const uint32_t *ctr, int64_t n, uint64_t seed, uint32_t *words,
                               void *normals, int precision, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  philox_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(ctr, n, (uint32_t)seed,
                                                       (uint32_t)(seed >> 32), words, normals,
                                                       precision);
  return cudaGetLastError();
}

}  // namespace vct
