// vct_pop.cu -- population draw and FP64 basal steady state (Sec. IV-B).
//
// One thread per patient.  Parameter j is drawn as mean + sd z with z the
// next normal of its own Philox sequence that satisfies |z| <= 1 (within one
// standard deviation) and gives a nonnegative value; the set is kept when the
// basal steady state at the setpoint exists and needs at least the minimum
// basal rate, else the next set attempt is drawn.  FP64 throughout.
#include "vct_internal.cuh"
#include "vct_rng.cuh"

namespace vct {
namespace {

struct PopKernelArgs {
  vct_population_desc d;
  double *rows, *ub, *x0;
  uint32_t *status;
  int32_t *attempts;
  int64_t n_pad;
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

// Bisection on [0, 1/S_IE] (the residual is strictly decreasing in I >= 0)
// until the midpoint no longer moves; then every state follows from I.  Each
// step needs only the residual's sign: with r(I) = A - B I - C I^2 / (k12 + S_ID I),
// A = EGP0 BW - F01c - F_R, B = EGP0 BW S_IE, C = Q1 S_IT S_ID, and k12 + S_ID I > 0,
// sign r = sign((A - B I)(k12 + S_ID I) - C I^2), free of the division.
__device__ bool basal_state(const double *p, double g_sp, double &ub, double x[VCT_NSTATE]) {
  for (int j = 0; j < VCT_NROW; ++j)
    if (!isfinite(p[j])) return false;
  if (!(p[VCT_P_SIE] > 0.0)) return false;
  double lo = 0.0, hi = 1.0 / p[VCT_P_SIE];
  if (!(basal_residual(p, g_sp, lo) > 0.0)) return false;
  {
    const double bw = p[VCT_P_BW];
    const double q1 = g_sp * p[VCT_P_VG] * bw;
    const double f01c = p[VCT_P_F01] * bw * fmin(1.0, g_sp / 4.5);
    const double f_r = fmax(0.0, 0.003 * (g_sp - 9.0) * p[VCT_P_VG] * bw);
    const double A = p[VCT_P_EGP0] * bw - f01c - f_r, B = p[VCT_P_EGP0] * bw * p[VCT_P_SIE];
    const double C = q1 * p[VCT_P_SIT] * p[VCT_P_SID], k12 = p[VCT_P_K12], sid = p[VCT_P_SID];
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if ((A - B * mid) * (k12 + sid * mid) - C * mid * mid > 0.0)
        lo = mid;
      else
        hi = mid;
    }
  }
  double i_ss = 0.5 * (lo + hi);
  double bw = p[VCT_P_BW];
  ub = i_ss * p[VCT_P_VI] * bw * p[VCT_P_KE];
  double q1 = g_sp * p[VCT_P_VG] * bw;
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

__device__ bool draw_set(const vct_population_desc &d, uint32_t pid, uint32_t set, double *p) {
  const uint32_t k0 = (uint32_t)d.seed, k1 = (uint32_t)(d.seed >> 32);
  for (int j = 0; j < VCT_NROW; ++j) {
    double mean = j < VCT_NPARAM ? d.p_mean[j] : d.bw_mean;
    double sd = j < VCT_NPARAM ? d.p_sd[j] : d.bw_sd;
    if (sd == 0.0) {
      p[j] = mean;
      continue;
    }
    bool ok = false;
    for (uint32_t call = 0; call < 16 && !ok; ++call) {
      Words4 w = philox4x32_10(Words4{set, pid, (uint32_t)j * 256u + call, kTagParam}, k0, k1);
      double z[4];
      // the second Box-Muller pair only when the first has no acceptable draw
      for (int q = 0; q < 4 && !ok; ++q) {
        if (q == 0) box_muller_f64(w.a, w.b, z[0], z[1]);
        if (q == 2) box_muller_f64(w.c, w.d, z[2], z[3]);
        double v = mean + sd * z[q];
        if (fabs(z[q]) <= 1.0 && v >= 0.0) {
          p[j] = v;
          ok = true;
        }
      }
    }
    if (!ok) return false;
  }
  return true;
}

__global__ void __launch_bounds__(128) population_kernel(PopKernelArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.d.n_patients) return;
  uint32_t pid = (uint32_t)(a.d.first_patient + i);
  double p[VCT_NROW], x[VCT_NSTATE], ub = 0.0;
  uint32_t st = VCT_PATIENT_REJECTED;
  int32_t used = a.d.max_attempts;
  for (int s = 0; s < a.d.max_attempts; ++s) {
    if (!draw_set(a.d, pid, (uint32_t)s, p)) continue;
    double u;
    if (!basal_state(p, a.d.g_sp, u, x)) continue;
    if (u * 60.0 / 1000.0 < a.d.min_basal_u_per_h) continue;
    ub = u;
    st = 0;
    used = s + 1;
    break;
  }
  if (st != 0)
    for (int j = 0; j < VCT_NSTATE; ++j) x[j] = 0.0;
  for (int j = 0; j < VCT_NROW; ++j) a.rows[j * a.n_pad + i] = p[j];
  for (int j = 0; j < VCT_NSTATE; ++j) a.x0[j * a.n_pad + i] = x[j];
  a.ub[i] = ub;
  a.status[i] = st;
  a.attempts[i] = used;
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
  if (words) {
    words[4 * i] = w.a;
    words[4 * i + 1] = w.b;
    words[4 * i + 2] = w.c;
    words[4 * i + 3] = w.d;
  }
  if (normals) {
    if (precision == VCT_FP64) {
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
                              uint32_t *status, int32_t *attempts, int64_t n_pad, cudaStream_t st) {
  PopKernelArgs a{d, rows, ub, x0, status, attempts, n_pad};
  int64_t blocks = d.n_patients > 0 ? (d.n_patients + 127) / 128 : 1;
  population_kernel<<<(unsigned)blocks, 128, 0, st>>>(a);
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
