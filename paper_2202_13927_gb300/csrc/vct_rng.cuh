// vct_rng.cuh -- device random numbers: Philox4x32-10 and Box-Muller.
//
// Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
// Shaw (SC'11): ten rounds, each multiplying counter words 0 and 2 by two
// 32-bit constants and mixing the high halves with words 1, 3 and the key;
// the key is bumped by two Weyl constants between rounds.  The paper
// integrates an SDE (Sec. III-A, Eq. 1b) without naming its generator; a
// counter-based one makes every draw a pure function of (seed, counter), so a
// patient's noise does not depend on which thread, launch or shard runs it.
//
// Counter layout (fourth word = stream tag | call << 8):
//   period k    (k, patient, stream, 0 | call << 8): normals 4*call .. 4*call+3 of
//               the period; normal 0 is the CGM noise v_k, normal 1 + s drives
//               Euler step s (so m = 10 steps need three calls)
//   meal size   (day * n_meals + meal, patient, stream, 2), normal 0
//   parameters  (set attempt, patient, slot * 256 + draw / 4, 3), normal draw % 4
#pragma once
#include <cstdint>

#include "vct_bm_tables.cuh"

namespace vct {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr uint32_t kTagSde = 0, kTagMeal = 2, kTagParam = 3;

struct Words4 {
  uint32_t a, b, c, d;
};

// Both halves of m x in one widening multiply.
__device__ __forceinline__ void mul_wide(uint32_t m, uint32_t x, uint32_t &hi, uint32_t &lo) {
  unsigned long long p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(x), "r"(m));
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

__device__ __forceinline__ Words4 philox_round(Words4 s, uint32_t k0, uint32_t k1) {
  // The M0 product as one widening multiply, the M1 product as separate high
  // and low halves: in the FP32 simulation this mix measured faster than
  // separate halves for both (0.4 % over 52 weeks, 2.6 % over 4) and than
  // widening both (it balances instruction issue against the pipe that runs
  // the integer multiplies).
  uint32_t hi0, lo0;
  mul_wide(kPhiloxM0, s.a, hi0, lo0);
  const uint32_t hi1 = __umulhi(kPhiloxM1, s.c), lo1 = kPhiloxM1 * s.c;
  return Words4{hi1 ^ s.b ^ k0, lo1, hi0 ^ s.d ^ k1, lo0};
}

// Rounds 2..10 applied to the state left by round 1 (keys of round 1 = k0, k1).
__device__ __forceinline__ Words4 philox_rounds_2_to_10(Words4 s, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 1; r < 10; ++r) s = philox_round(s, k0 + r * kPhiloxW0, k1 + r * kPhiloxW1);
  return s;
}

__device__ __forceinline__ Words4 philox4x32_10(Words4 ctr, uint32_t k0, uint32_t k1) {
  return philox_rounds_2_to_10(philox_round(ctr, k0, k1), k0, k1);
}

// The key of every round, precomputed once per seed: round r (0-based) uses
// (k0 + r W0, k1 + r W1).  Kept in a kernel parameter, the keys are read as
// constant operands instead of being formed in the loop.
constexpr int kPhiloxRoundKeys = 20;
__host__ __device__ inline void philox_round_keys(uint64_t seed, uint32_t rk[kPhiloxRoundKeys]) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0 + (uint32_t)r * kPhiloxW0;
    rk[2 * r + 1] = k1 + (uint32_t)r * kPhiloxW1;
  }
}

__device__ __forceinline__ Words4 philox_rounds_2_to_10(Words4 s, const uint32_t *rk) {
#pragma unroll
  for (int r = 1; r < 10; ++r) s = philox_round(s, rk[2 * r], rk[2 * r + 1]);
  return s;
}

// Round 1 factorised for the simulation loop.  Counter words 1 and 2
// (patient, stream) are fixed per thread, word 0 (the period) is shared by all
// calls of one period, word 3 differs per call only by an XOR:
//   round-1 out = (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0)).
struct PhiloxLane {
  uint32_t w0, w1;  // first two words after round 1 (per patient, per stream)
  uint32_t k0, k1;
  // all calls of counter word 0 = c0: hi/lo of M0 c0, computed once
  __device__ __forceinline__ Words4 call(uint32_t c0_hi, uint32_t c0_lo, uint32_t c3) const {
    return philox_rounds_2_to_10(Words4{w0, w1, c0_hi ^ c3 ^ k1, c0_lo}, k0, k1);
  }
};

// The same with the round keys precomputed (rk from philox_round_keys).
struct PhiloxLaneRk {
  uint32_t w0, w1;
  const uint32_t *rk;
  __device__ __forceinline__ Words4 call(uint32_t c0_hi, uint32_t c0_lo, uint32_t c3) const {
    return philox_rounds_2_to_10(Words4{w0, w1, c0_hi ^ c3 ^ rk[1], c0_lo}, rk);
  }
};

__device__ __forceinline__ PhiloxLane make_lane(uint32_t patient, uint32_t stream, uint32_t key0,
                                                uint32_t key1) {
  PhiloxLane l;
  l.w0 = __umulhi(kPhiloxM1, stream) ^ patient ^ key0;
  l.w1 = kPhiloxM1 * stream;
  l.k0 = key0;
  l.k1 = key1;
  return l;
}

// ---------------------------------------------------------------- Box-Muller
// FP64 through the CUDA library: u = (w + 1/2) 2^-32 (exact), r = sqrt(-2 ln u0),
// angle 2 pi u1 (the population draw, and the reference of the form below).
__device__ __forceinline__ void box_muller_f64(uint32_t w0, uint32_t w1, double &z0, double &z1) {
  const double scale = 2.3283064365386962890625e-10;  // 2^-32
  double u0 = ((double)w0 + 0.5) * scale;
  double u1 = ((double)w1 + 0.5) * scale;
  double r = sqrt(-2.0 * log(u0));
  double s, c;
  sincospi(2.0 * u1, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// FP64 with the project's own logarithm, reciprocal square root and angle
// reduction, from the same words to the same normals (within a few units in
// the last place of the library form above):
//   u0 = v 2^-33 with v = 2 w0 + 1 (odd, at most 33 bits).  Its significand
//   m, taken in [0.75, 1.5), and exponent k come from v by integer operations;
//   the 12 bits after the leading one pick one of 4096 reduction intervals j
//   whose reciprocal c_j has 20 significant bits, so r = m c_j - 1 is exact in
//   one fma and |r| < 1.01 2^-13 (table-driven logarithm after Tang, ACM TOMS
//   16(4) 1990, with the short-reciprocal reduction of Muller, "Elementary
//   Functions", ch. 6).  H = -ln(u0) / 8 = -k ln2 / 8 + ln(c_j) / 8 - ln(1+r) / 8
//   with the two table terms in two parts and the degree-4 Taylor polynomial
//   of ln(1 + r) (truncation below 2^-54 relative).
//   Radius sqrt(-2 ln u0) = 4 sqrt(2) H w, w = 1/sqrt(2 H) from the hardware
//   approximation refined by two Newton steps w <- w (3/2 - H w^2).
//   Angle 2 pi u1 = 2 pi (j1 + 1/2) / 4096 + 2 pi q 2^-33 with j1 the top 12 bits
//   of w1 and q = 2 (w1 mod 2^20) + 1 - 2^20 an exact odd integer, |q| < 2^20
//   (|angle| < 2 pi / 8192 rad): sin and 1 - cos of the small angle by their
//   Taylor polynomials in q (degree 3 and 4), then the addition formulas with
//   the table's sin and cos of the interval centre (scaled by 4 sqrt(2)).
// Only FP64 adds, multiplies and fmas run on the FP64 pipe (29 per pair); the
// index and exponent work is integer.  The tables (160 KB, read through L1)
// save three FP64 operations per pair over 256 log intervals and 1024 angles.
__device__ __forceinline__ double rsqrt_seed_f64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ void box_muller_f64t(uint32_t w0, uint32_t w1, double &z0, double &z1) {
  using namespace bm64;
  const unsigned long long v = 2ull * (unsigned long long)w0 + 1ull;
  const int n = 63 - __clzll((long long)v);                      // v in [2^n, 2^(n+1))
  const unsigned long long frac = (v << (52 - n)) & 0x000FFFFFFFFFFFFFull;
  const uint32_t j = (uint32_t)(frac >> 40);
  const bool upper = j >= 2048u;                                 // m >= 1.5: take m / 2
  const double m = __longlong_as_double(
      (long long)(frac | (upper ? 0x3FE0000000000000ull : 0x3FF0000000000000ull)));
  const int kn = 33 - n - (upper ? 1 : 0);                       // -k, 0 .. 33
  const double r = fma(m, __ldg(&kLogC[j]), -1.0);
  double p = fma(r, kLogP3, kLogP2);
  p = fma(r, p, kLogP1);
  p = fma(r, p, kLogP0);
  const double2 t = __ldg(&kLogT[j]);
  const double2 kk = __ldg(&kLogK[kn]);
  const double H = (kk.x + t.x) + ((kk.y + t.y) + r * p);
  double w = rsqrt_seed_f64(H + H);
  w = fma(w, fma(-H, w * w, 0.5), w);
  w = fma(w, fma(-H, w * w, 0.5), w);
  const double rad = H * w;                                      // radius / (4 sqrt 2)
  const int qi = (int)(2u * (w1 & 0x000FFFFFu) + 1u) - (1 << 20);
  const double x = __longlong_as_double(0x4338000000000000LL + (long long)qi) - 6755399441055744.0;
  const double xx = x * x;
  const double sn = x * fma(xx, kSinP1, kSinP0);
  const double cm = xx * fma(xx, kCosP1, kCosP0);
  const double2 sc = __ldg(&kAngle[w1 >> 20]);                   // 4 sqrt2 (sin, cos) of the centre
  z0 = rad * fma(-sc.x, sn, fma(-sc.y, cm, sc.y));               // 4 sqrt2 cos(a + theta)
  z1 = rad * fma(sc.y, sn, fma(-sc.x, cm, sc.x));                // 4 sqrt2 sin(a + theta)
}

// FP32: the same mapping evaluated with the fast hardware functions.
// u0 = rz(w0) 2^-32 + 2^-33 stays in (0, 1) and keeps relative accuracy near
// 0, where the logarithm is steep; the angle is taken as 2 pi (u1 - 1/2) in
// [-pi, pi] so that __sincosf stays in its accurate range, and the sign flip
// that the shift causes is undone on r.
__device__ __forceinline__ void box_muller_f32(uint32_t w0, uint32_t w1, float &z0, float &z1) {
  const float two_m32 = 2.3283064365386963e-10f;  // 2^-32
  const float two_m33 = 1.1641532182693481e-10f;  // 2^-33
  float u0 = fmaf(__uint2float_rz(w0), two_m32, two_m33);
  float r2 = -2.0f * __logf(u0);
  r2 = fmaxf(r2, 1e-30f);
  float r = r2 * rsqrtf(r2);
  const float two_pi_m32 = 1.4629180792671596e-09f;  // 2 pi 2^-32
  float ang = fmaf(__uint2float_rz(w1), two_pi_m32, 7.3145904e-10f - 3.14159265358979f);
  float s, c;
  __sincosf(ang, &s, &c);
  z0 = -r * c;  // cos(2 pi u1) = -cos(2 pi (u1 - 1/2))
  z1 = -r * s;
}

template <typename Real>
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, Real &z0, Real &z1);
template <>
__device__ __forceinline__ void box_muller<double>(uint32_t w0, uint32_t w1, double &z0,
                                                   double &z1) {
  box_muller_f64t(w0, w1, z0, z1);
}
template <>
__device__ __forceinline__ void box_muller<float>(uint32_t w0, uint32_t w1, float &z0,
                                                  float &z1) {
  box_muller_f32(w0, w1, z0, z1);
}

// A Box-Muller pair already scaled and shifted for the Euler step:
// n_i = scale z_i + offset (FP32: the product -r scale is formed once per pair).
__device__ __forceinline__ void box_muller_axpb(uint32_t w0, uint32_t w1, float scale,
                                                float offset, float &n0, float &n1) {
  const float two_m32 = 2.3283064365386963e-10f;
  const float two_m33 = 1.1641532182693481e-10f;
  float u0 = fmaf(__uint2float_rz(w0), two_m32, two_m33);
  float r2 = fmaxf(-2.0f * __logf(u0), 1e-30f);
  float rs = -(r2 * rsqrtf(r2)) * scale;
  const float two_pi_m32 = 1.4629180792671596e-09f;
  float ang = fmaf(__uint2float_rz(w1), two_pi_m32, 7.3145904e-10f - 3.14159265358979f);
  float s, c;
  __sincosf(ang, &s, &c);
  n0 = fmaf(rs, c, offset);
  n1 = fmaf(rs, s, offset);
}
__device__ __forceinline__ void box_muller_axpb(uint32_t w0, uint32_t w1, double scale,
                                                double offset, double &n0, double &n1) {
  double z0, z1;
  box_muller_f64t(w0, w1, z0, z1);
  n0 = fma(scale, z0, offset);
  n1 = fma(scale, z1, offset);
}

// Only the first normal of a pair (CGM and meal draws use one normal).
__device__ __forceinline__ double box_muller_first(uint32_t w0, uint32_t w1, double) {
  double z0, z1;
  box_muller_f64t(w0, w1, z0, z1);
  return z0;
}
__device__ __forceinline__ float box_muller_first(uint32_t w0, uint32_t w1, float) {
  const float two_m32 = 2.3283064365386963e-10f;
  const float two_m33 = 1.1641532182693481e-10f;
  float u0 = fmaf(__uint2float_rz(w0), two_m32, two_m33);
  float r2 = fmaxf(-2.0f * __logf(u0), 1e-30f);
  float r = r2 * rsqrtf(r2);
  const float two_pi_m32 = 1.4629180792671596e-09f;
  float ang = fmaf(__uint2float_rz(w1), two_pi_m32, 7.3145904e-10f - 3.14159265358979f);
  return -r * __cosf(ang);
}

}  // namespace vct
