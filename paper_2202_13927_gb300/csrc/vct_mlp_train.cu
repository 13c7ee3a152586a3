// vct_mlp_train.cu -- the surrogate network: features -> 256 -> 256 -> 5 range
// fractions (softmax), BF16 operands with FP32 accumulation on the tensor
// cores, trained on the simulator's own runs and used to screen controller
// tunings (the hyperparameters of the controller, Sec. III-B Eq. 3) before the
// closed-loop simulation (Sec. III) judges the best.  Not in the paper.
//
// Kernels
//   features_kernel    standardized features of (patient, scenario) pairs
//   forward (vct_mlp_fwd.cu) fused 3-layer forward on tcgen05, weights resident
//                      in shared memory (train: keeps H1, H2, logits; predict:
//                      softmax; screen: mean range fraction per candidate)
//   xent_kernel        softmax + cross-entropy + dlogits
//   gemm_kernel        strided BF16 GEMM with split-K partials (backward pass)
//   colsum / reduce    bias gradients and split-K sums in a fixed order
//   adamw_kernel       AdamW on FP32 master weights, BF16 copies for the GEMMs
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "vct_mlp.cuh"

namespace vct {
namespace {

constexpr int H = VCT_SURR_HIDDEN;   // hidden width
constexpr int KF = VCT_SURR_KF;      // padded feature width
constexpr int NF = VCT_SURR_FEATURES;
constexpr int NO = VCT_NBINS;        // outputs
constexpr int NOP = 8;               // outputs padded to one n8 tile
constexpr int NOK = 16;              // outputs padded to one k16 step (backward)
constexpr int PADK = 8;              // smem row padding (bf16) against bank conflicts

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

// A fragment of a 16x16 tile stored [row][k] with row stride ld (elements).
__device__ __forceinline__ void load_a(uint32_t a[4], const bf16 *base, int ld, int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(base + g * ld + 2 * t);
  a[1] = ld32(base + (g + 8) * ld + 2 * t);
  a[2] = ld32(base + g * ld + 2 * t + 8);
  a[3] = ld32(base + (g + 8) * ld + 2 * t + 8);
}
// B fragment of a 16(k) x 8(n) tile stored [n][k] with row stride ld.
__device__ __forceinline__ void load_b(uint32_t b[2], const bf16 *base, int ld, int lane) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = ld32(base + g * ld + 2 * t);
  b[1] = ld32(base + g * ld + 2 * t + 8);
}

// ------------------------------------------------------------------ features
struct FeatArgs {
  PopDev pop;
  const double *gains;    // [n_scen][3] multipliers (kp, ki, kd)
  int32_t n_scen;
  const int64_t *ids;     // sample ids (s * n + i) or nullptr = all in order
  int64_t n_rows;
  float mean[NF], inv_sd[NF];
  bf16 *xb;               // [rows][KF] or nullptr
  float *xf;              // [rows][KF] or nullptr
  const vct_patient_stats *stats;  // targets or nullptr
  float *t;               // [rows][NO]
};

// Feature j < 15: parameter slot (the 14 Hovorka parameters, then body weight),
// standardized by the population table; 15..17: log gain multipliers / ln 3.
__device__ __constant__ int kFeatSlot[15] = {VCT_P_EGP0, VCT_P_F01, VCT_P_K12, VCT_P_KA1, VCT_P_KA2,
                                             VCT_P_KA3,  VCT_P_SIT, VCT_P_SID, VCT_P_SIE, VCT_P_KE,
                                             VCT_P_VI,   VCT_P_VG,  VCT_P_TAUS, VCT_P_TAUD, VCT_P_BW};

__global__ void features_kernel(FeatArgs a) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_rows) return;
  const int64_t id = a.ids ? a.ids[r] : r;
  const int64_t n = a.pop.n;
  const int s = (int)(id / n);
  const int64_t i = id % n;
  float f[KF];
#pragma unroll
  for (int j = 0; j < 15; ++j)
    f[j] = (float)((a.pop.rows[kFeatSlot[j] * a.pop.n_pad + i] - a.mean[j]) * a.inv_sd[j]);
#pragma unroll
  for (int j = 0; j < 3; ++j) f[15 + j] = (float)(log(a.gains[3 * s + j]) * a.inv_sd[15 + j]);
#pragma unroll
  for (int j = NF; j < KF; ++j) f[j] = 0.0f;
  if (a.xb)
    for (int j = 0; j < KF; ++j) a.xb[r * KF + j] = __float2bfloat16_rn(f[j]);
  if (a.xf)
    for (int j = 0; j < KF; ++j) a.xf[r * KF + j] = f[j];
  if (a.t) {
    const vct_patient_stats &p = a.stats[id];
    const float inv = p.n_samples ? 1.0f / (float)p.n_samples : 0.0f;
    for (int b = 0; b < NO; ++b) a.t[r * NO + b] = (float)p.tir[b] * inv;
  }
}

// Standardized log gains of the screened candidates, lg = log(g) / sd, in
// FP64 then rounded to FP32; a gain that is not finite and > 0 sets bit 2 of
// the error word (and a NaN feature).
__global__ void cand_lg_kernel(const double *gains, int64_t n, double inv0, double inv1, double inv2,
                               float *lg, int *error) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const double g = gains[i];
  const int j = (int)(i % 3);
  const double inv = j == 0 ? inv0 : (j == 1 ? inv1 : inv2);
  if (!(g > 0.0) || !isfinite(g)) {
    atomicOr(error, 2);
    lg[i] = __int_as_float(0x7fc00000);
    return;
  }
  lg[i] = (float)(log(g) * inv);
}

// ------------------------------------------------------------------ loss
// p = softmax(logits), loss partial per row, dZ3 = (p sum(t) - t) / B as BF16 [rows][NOK]
__global__ void xent_kernel(const float *logits, const float *t, int64_t n_rows, float inv_b,
                            bf16 *dz3, float *row_loss) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  float m = logits[r * NOP];
  for (int b = 1; b < NO; ++b) m = fmaxf(m, logits[r * NOP + b]);
  float ex[NO], sum = 0.0f, ts = 0.0f;
  for (int b = 0; b < NO; ++b) {
    ex[b] = expf(logits[r * NOP + b] - m);
    sum += ex[b];
    ts += t[r * NO + b];
  }
  const float lse = m + logf(sum);
  float l = 0.0f;
  for (int b = 0; b < NO; ++b) {
    const float p = ex[b] / sum;
    l -= t[r * NO + b] * (logits[r * NOP + b] - lse);
    dz3[r * NOK + b] = __float2bfloat16_rn((p * ts - t[r * NO + b]) * inv_b);
  }
  for (int b = NO; b < NOK; ++b) dz3[r * NOK + b] = __float2bfloat16_rn(0.0f);
  row_loss[r] = l;
}

// ------------------------------------------------------------------ backward GEMM
// C[M][N] = sum_k A(m, k) B(k, n); A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn].
// Split-K: blockIdx.z covers k in [z kc, (z+1) kc) and writes partial[z][M][N]
// (mode 0), or a single pass writes BF16 outputs masked by mask(m, n) > 0 (mode 1).
struct GemmArgs {
  const bf16 *A, *B;
  int64_t sam, sak, sbk, sbn;
  int M, N;
  int64_t K, kc;
  float *partial;        // mode 0
  bf16 *out;             // mode 1: [M][N]
  const bf16 *mask;      // mode 1: [M][N] (ReLU outputs)
};

constexpr int GT = 64, GK = 32, GTHREADS = 128;

template <int MODE>
__global__ void __launch_bounds__(GTHREADS) gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) bf16 As[GT][GK + PADK];
  __shared__ __align__(16) bf16 Bs[GT][GK + PADK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps of 32 x 32
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int64_t kb = (int64_t)blockIdx.z * g.kc, ke = min(g.K, kb + g.kc);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
  const bf16 zero = __float2bfloat16_rn(0.0f);
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    for (int e = tid; e < GT * GK; e += GTHREADS) {
      const int r = e / GK, k = e % GK;
      const int64_t kk = k0 + k;
      const bool kin = kk < ke;
      As[r][k] = (kin && m0 + r < g.M) ? g.A[(int64_t)(m0 + r) * g.sam + kk * g.sak] : zero;
      Bs[r][k] = (kin && n0 + r < g.N) ? g.B[kk * g.sbk + (int64_t)(n0 + r) * g.sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) load_a(a[i], &As[wm * 32 + i * 16][kk], GK + PADK, lane);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t b[2];
        load_b(b, &Bs[wn * 32 + j * 8][kk], GK + PADK, lane);
#pragma unroll
        for (int i = 0; i < 2; ++i) mma16816(acc[i][j], a[i], b);
      }
    }
    __syncthreads();
  }
  const int gq = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 32 + i * 16 + gq + 8 * h;
        const int n = n0 + wn * 32 + j * 8 + 2 * t;
        if (m >= g.M) continue;
        for (int c = 0; c < 2; ++c) {
          if (n + c >= g.N) continue;
          const float v = acc[i][j][2 * h + c];
          if (MODE == 0) {
            g.partial[((int64_t)blockIdx.z * g.M + m) * g.N + n + c] = v;
          } else {
            const bool on = __bfloat162float(g.mask[(int64_t)m * g.N + n + c]) > 0.0f;
            g.out[(int64_t)m * g.N + n + c] = __float2bfloat16_rn(on ? v : 0.0f);
          }
        }
      }
}

// out[i] = sum_z partial[z][i] in z order
__global__ void reduce_partials(const float *partial, int splits, int64_t count, float *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float s = 0.0f;
  for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * count + i];
  out[i] = s;
}

// column sums of a BF16 [rows][ld] matrix over its first n columns (fixed order)
__global__ void colsum_kernel(const bf16 *x, int64_t rows, int ld, int n, float *out) {
  __shared__ float sh[8][33];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int rgrp = threadIdx.x >> 5;  // 8 row groups
  float s = 0.0f;
  if (c < n)
    for (int64_t r = rgrp; r < rows; r += 8) s += __bfloat162float(x[r * ld + c]);
  sh[rgrp][threadIdx.x & 31] = s;
  __syncthreads();
  if (rgrp == 0 && c < n) {
    float v = 0.0f;
    for (int k = 0; k < 8; ++k) v += sh[k][threadIdx.x & 31];
    out[c] = v;
  }
}

// ------------------------------------------------------------------ AdamW
struct AdamArgs {
  float *w, *m, *v;
  const float *g;
  bf16 *wb;             // BF16 copy (rows of ld_b, first cols_b of each row of cols) or null
  int64_t count;
  int cols, ld_b;       // master is [count / cols][cols]; copy is [rows][ld_b]
  float lr, b1, b2, eps, wd, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
  int decay;
};

__global__ void adamw_kernel(AdamArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const float g = a.g[i];
  const float m = a.b1 * a.m[i] + (1.0f - a.b1) * g;
  const float v = a.b2 * a.v[i] + (1.0f - a.b2) * g * g;
  a.m[i] = m;
  a.v[i] = v;
  float w = a.w[i];
  if (a.decay) w -= a.lr * a.wd * w;
  w -= a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
  a.w[i] = w;
  if (a.wb) a.wb[(i / a.cols) * a.ld_b + i % a.cols] = __float2bfloat16_rn(w);
}

__global__ void to_bf16_kernel(const float *w, int64_t count, int cols, int ld_b, bf16 *wb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) wb[(i / cols) * ld_b + i % cols] = __float2bfloat16_rn(w[i]);
}

}  // namespace
}  // namespace vct

// =================================================================== host side
struct vct_surrogate {
  vct_surrogate_desc desc;
  float mean[VCT_SURR_FEATURES], inv_sd[VCT_SURR_FEATURES];
  void *mem;
  // master FP32 parameters, moments, gradients: W1 [H][NF], b1, W2 [H][H], b2, W3 [NO][H], b3
  float *w, *m, *v, *g;
  int64_t n_params;
  // BF16 copies laid out for the kernels
  __nv_bfloat16 *W1b, *W2b, *W3b;
  float *b1, *b2, *b3;  // padded copies for the forward (b3: [8])
  int64_t step;
  // training buffers (batch rows)
  __nv_bfloat16 *xb, *h1, *h2, *dz3, *dz2, *dz1;
  float *tgt, *logits, *row_loss, *partial;
  int64_t batch;
  int *err;  // device: set by the forward kernel if a bounded wait gives up
  int stall_test;  // test hook (vct_surrogate_inject_stall)
};

namespace {

using vct::H;
using vct::KF;
using vct::NF;
using vct::NO;
using vct::NOK;
using vct::NOP;
typedef __nv_bfloat16 bf16;

vct_status sfail(vct_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return vct::record_error(code, buf);
}

#define S_CUDA(call)                                                                        \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return sfail(e_ == cudaErrorMemoryAllocation ? VCT_ERR_OOM : VCT_ERR_CUDA, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                 \
  } while (0)

// parameter offsets in the packed FP32 vector
constexpr int64_t kOffW1 = 0;
constexpr int64_t kOffB1 = kOffW1 + (int64_t)H * NF;
constexpr int64_t kOffW2 = kOffB1 + H;
constexpr int64_t kOffB2 = kOffW2 + (int64_t)H * H;
constexpr int64_t kOffW3 = kOffB2 + H;
constexpr int64_t kOffB3 = kOffW3 + (int64_t)NO * H;
constexpr int64_t kNParams = kOffB3 + NO;

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t blocks_for(int64_t n, int t) { return (n + t - 1) / t; }

cudaError_t refresh_bf16(vct_surrogate *s, cudaStream_t st) {
  // padded BF16 copies: W1 [H][KF] (cols >= NF zero), W2 [H][H], W3 [NOP][H] (rows >= NO zero)
  vct::to_bf16_kernel<<<blocks_for((int64_t)H * NF, 256), 256, 0, st>>>(s->w + kOffW1, (int64_t)H * NF, NF, KF, s->W1b);
  vct::to_bf16_kernel<<<blocks_for((int64_t)H * H, 256), 256, 0, st>>>(s->w + kOffW2, (int64_t)H * H, H, H, s->W2b);
  vct::to_bf16_kernel<<<blocks_for((int64_t)NO * H, 256), 256, 0, st>>>(s->w + kOffW3, (int64_t)NO * H, H, H, s->W3b);
  cudaError_t e = cudaMemcpyAsync(s->b1, s->w + kOffB1, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->b2, s->w + kOffB2, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->b3, s->w + kOffB3, sizeof(float) * NO, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

vct::FwdArgs fwd_args(const vct_surrogate *s) {
  vct::FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.W1 = s->W1b;
  a.W2 = s->W2b;
  a.W3 = s->W3b;
  a.b1 = s->b1;
  a.b2 = s->b2;
  a.b3 = s->b3;
  a.error = s->err;
  a.stall_test = s->stall_test;
  return a;
}

int64_t row_tiles(int64_t rows) { return (rows + 127) / 128; }

// C (split-K partials or masked BF16) = A B with strided operands
cudaError_t gemm(int mode, const bf16 *A, int64_t sam, int64_t sak, const bf16 *B, int64_t sbk,
                 int64_t sbn, int M, int N, int64_t K, float *partial, int splits, bf16 *out,
                 const bf16 *mask, cudaStream_t st) {
  vct::GemmArgs g;
  g.A = A;
  g.B = B;
  g.sam = sam;
  g.sak = sak;
  g.sbk = sbk;
  g.sbn = sbn;
  g.M = M;
  g.N = N;
  g.K = K;
  g.kc = (K + splits - 1) / splits;
  g.kc = (g.kc + vct::GK - 1) / vct::GK * vct::GK;
  g.partial = partial;
  g.out = out;
  g.mask = mask;
  dim3 grid((N + vct::GT - 1) / vct::GT, (M + vct::GT - 1) / vct::GT, splits);
  if (mode == 0)
    vct::gemm_kernel<0><<<grid, vct::GTHREADS, 0, st>>>(g);
  else
    vct::gemm_kernel<1><<<grid, vct::GTHREADS, 0, st>>>(g);
  return cudaGetLastError();
}

int splits_for(int64_t K) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, K / 256)); }

// weight gradient dW [M][N] = dZ^T [M][B] X [B][N] (+ the split-K sum) into gdst
cudaError_t weight_grad(vct_surrogate *s, const bf16 *dz, int ldz, int M, const bf16 *x, int ldx, int N,
                        int64_t B, float *gdst, cudaStream_t st) {
  const int sp = splits_for(B);
  cudaError_t e = gemm(0, dz, 1, ldz, x, ldx, 1, M, N, B, s->partial, sp, nullptr, nullptr, st);
  if (e != cudaSuccess) return e;
  vct::reduce_partials<<<blocks_for((int64_t)M * N, 256), 256, 0, st>>>(s->partial, sp, (int64_t)M * N, gdst);
  return cudaGetLastError();
}

vct_status ensure_batch(vct_surrogate *s, int64_t B) {
  if (B <= s->batch) return VCT_OK;
  return sfail(VCT_ERR_ARG, "batch %lld exceeds the surrogate's batch capacity %lld", (long long)B,
               (long long)s->batch);
}

// forward + loss + backward on the rows already in s->xb / s->tgt; then AdamW if update
vct_status train_rows(vct_surrogate *s, int64_t B, bool update, cudaStream_t st) {
  vct::FwdArgs a = fwd_args(s);
  a.x = s->xb;
  a.n_rows = B;
  a.h1 = s->h1;
  a.h2 = s->h2;
  a.logits = s->logits;
  S_CUDA(vct::launch_forward(a, vct::MODE_TRAIN, row_tiles(B), st));
  vct::xent_kernel<<<blocks_for(B, 256), 256, 0, st>>>(s->logits, s->tgt, B, 1.0f / (float)B, s->dz3, s->row_loss);
  S_CUDA(cudaGetLastError());
  float *g = s->g;
  // layer 3: dW3 = dZ3^T H2, db3 = colsum dZ3, dZ2 = (dZ3 W3) * [H2 > 0]
  S_CUDA(weight_grad(s, s->dz3, NOK, NO, s->h2, H, H, B, g + kOffW3, st));
  vct::colsum_kernel<<<1, 256, 0, st>>>(s->dz3, B, NOK, NO, g + kOffB3);
  S_CUDA(gemm(1, s->dz3, NOK, 1, s->W3b, H, 1, (int)B, H, NOK, nullptr, 1, s->dz2, s->h2, st));
  // layer 2
  S_CUDA(weight_grad(s, s->dz2, H, H, s->h1, H, H, B, g + kOffW2, st));
  vct::colsum_kernel<<<H / 32, 256, 0, st>>>(s->dz2, B, H, H, g + kOffB2);
  S_CUDA(gemm(1, s->dz2, H, 1, s->W2b, H, 1, (int)B, H, H, nullptr, 1, s->dz1, s->h1, st));
  // layer 1
  S_CUDA(weight_grad(s, s->dz1, H, H, s->xb, KF, NF, B, g + kOffW1, st));
  vct::colsum_kernel<<<H / 32, 256, 0, st>>>(s->dz1, B, H, H, g + kOffB1);
  S_CUDA(cudaGetLastError());
  if (update) {
    s->step += 1;
    const vct_surrogate_desc &d = s->desc;
    vct::AdamArgs A;
    std::memset(&A, 0, sizeof(A));
    A.lr = (float)d.lr;
    A.b1 = (float)d.beta1;
    A.b2 = (float)d.beta2;
    A.eps = (float)d.eps;
    A.wd = (float)d.weight_decay;
    A.c1 = (float)(1.0 / (1.0 - std::pow(d.beta1, (double)s->step)));
    A.c2 = (float)(1.0 / (1.0 - std::pow(d.beta2, (double)s->step)));
    struct Seg { int64_t off, count; int cols, ld; bf16 *wb; int decay; };
    const Seg segs[] = {{kOffW1, (int64_t)H * NF, NF, KF, s->W1b, 1}, {kOffB1, H, H, H, nullptr, 0},
                        {kOffW2, (int64_t)H * H, H, H, s->W2b, 1},  {kOffB2, H, H, H, nullptr, 0},
                        {kOffW3, (int64_t)NO * H, H, H, s->W3b, 1}, {kOffB3, NO, NO, NO, nullptr, 0}};
    for (const Seg &sg : segs) {
      A.w = s->w + sg.off;
      A.m = s->m + sg.off;
      A.v = s->v + sg.off;
      A.g = s->g + sg.off;
      A.count = sg.count;
      A.cols = sg.cols;
      A.ld_b = sg.ld;
      A.wb = sg.wb;
      A.decay = sg.decay;
      vct::adamw_kernel<<<blocks_for(sg.count, 256), 256, 0, st>>>(A);
    }
    S_CUDA(cudaGetLastError());
    S_CUDA(cudaMemcpyAsync(s->b1, s->w + kOffB1, sizeof(float) * H, cudaMemcpyDeviceToDevice, st));
    S_CUDA(cudaMemcpyAsync(s->b2, s->w + kOffB2, sizeof(float) * H, cudaMemcpyDeviceToDevice, st));
    S_CUDA(cudaMemcpyAsync(s->b3, s->w + kOffB3, sizeof(float) * NO, cudaMemcpyDeviceToDevice, st));
  }
  return VCT_OK;
}

vct_status check_err(const vct_surrogate *s, cudaStream_t st) {
  int e = 0;
  S_CUDA(cudaMemcpyAsync(&e, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  S_CUDA(cudaStreamSynchronize(st));
  if (e) S_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));  // reported once
  if (e & 2) return sfail(VCT_ERR_ARG, "surrogate screen: a candidate's gains were not finite and > 0");
  if (e) return sfail(VCT_ERR_TIMEOUT, "surrogate forward: a tensor-core wait gave up");
  return VCT_OK;
}

vct_status loss_of_rows(vct_surrogate *s, int64_t B, cudaStream_t st, double *out) {
  std::vector<float> l((size_t)B);
  S_CUDA(cudaMemcpyAsync(l.data(), s->row_loss, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
  S_CUDA(cudaStreamSynchronize(st));
  double sum = 0.0;
  for (float x : l) sum += x;
  *out = sum / (double)B;
  return VCT_OK;
}

vct::FeatArgs feat_args(const vct_surrogate *s, const vct_population *pop) {
  vct::FeatArgs f;
  std::memset(&f, 0, sizeof(f));
  f.pop.rows = pop->rows;
  f.pop.n = pop->n;
  f.pop.n_pad = pop->n_pad;
  for (int j = 0; j < NF; ++j) {
    f.mean[j] = s->mean[j];
    f.inv_sd[j] = s->inv_sd[j];
  }
  return f;
}

vct_status upload_gains(const vct_scenario *sc, int32_t n_scen, cudaStream_t st, double **dev) {
  std::vector<double> g((size_t)3 * n_scen);
  for (int s = 0; s < n_scen; ++s) {
    const double v[3] = {sc[s].kp_mult, sc[s].ki_mult, sc[s].kd_mult};
    for (int j = 0; j < 3; ++j) {
      if (!(v[j] > 0.0) || !std::isfinite(v[j]))
        return sfail(VCT_ERR_ARG, "scenario %d: gain multipliers must be > 0 for the surrogate", s);
      g[3 * s + j] = v[j];
    }
  }
  S_CUDA(cudaMallocAsync((void **)dev, sizeof(double) * g.size(), st));
  S_CUDA(cudaMemcpyAsync(*dev, g.data(), sizeof(double) * g.size(), cudaMemcpyHostToDevice, st));
  return VCT_OK;
}

}  // namespace

extern "C" {

vct_status vct_surrogate_create(const vct_surrogate_desc *desc, const vct_population_desc *scale,
                                void *cuda_stream, vct_surrogate **out) {
  if (!desc || !scale || !out) return sfail(VCT_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (desc->batch < 64 || desc->batch % 64 || desc->batch > (1 << 22))
    return sfail(VCT_ERR_ARG, "batch must be a multiple of 64 in 64..2^22");
  if (!(desc->lr > 0.0) || !(desc->beta1 >= 0.0 && desc->beta1 < 1.0) ||
      !(desc->beta2 >= 0.0 && desc->beta2 < 1.0) || !(desc->eps > 0.0) || !(desc->weight_decay >= 0.0))
    return sfail(VCT_ERR_ARG, "bad optimiser settings");
  auto *s = new (std::nothrow) vct_surrogate();
  if (!s) return sfail(VCT_ERR_OOM, "host allocation failed");
  s->desc = *desc;
  s->batch = desc->batch;
  s->n_params = kNParams;
  // feature scales from the population table (sd 0 -> feature 0)
  static const int slots[15] = {VCT_P_EGP0, VCT_P_F01, VCT_P_K12, VCT_P_KA1, VCT_P_KA2, VCT_P_KA3,
                                VCT_P_SIT,  VCT_P_SID, VCT_P_SIE, VCT_P_KE,  VCT_P_VI,  VCT_P_VG,
                                VCT_P_TAUS, VCT_P_TAUD, VCT_P_BW};
  for (int j = 0; j < 15; ++j) {
    const int sl = slots[j];
    const double mean = sl == VCT_P_BW ? scale->bw_mean : scale->p_mean[sl];
    const double sd = sl == VCT_P_BW ? scale->bw_sd : scale->p_sd[sl];
    s->mean[j] = (float)mean;
    s->inv_sd[j] = sd > 0.0 ? (float)(1.0 / sd) : 0.0f;
  }
  for (int j = 15; j < NF; ++j) {
    s->mean[j] = 0.0f;
    s->inv_sd[j] = (float)(1.0 / std::log(3.0));
  }
  const int64_t B = desc->batch;
  const int sp = splits_for(B);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = al(off + bytes); return o; };
  const size_t o_w = take(sizeof(float) * kNParams), o_m = take(sizeof(float) * kNParams),
               o_v = take(sizeof(float) * kNParams), o_g = take(sizeof(float) * kNParams);
  const size_t o_w1 = take(sizeof(bf16) * H * KF), o_w2 = take(sizeof(bf16) * H * H),
               o_w3 = take(sizeof(bf16) * NOK * H);
  const size_t o_b1 = take(sizeof(float) * H), o_b2 = take(sizeof(float) * H), o_b3 = take(sizeof(float) * NOP);
  const size_t o_xb = take(sizeof(bf16) * B * KF), o_h1 = take(sizeof(bf16) * B * H),
               o_h2 = take(sizeof(bf16) * B * H), o_dz3 = take(sizeof(bf16) * B * NOK),
               o_dz2 = take(sizeof(bf16) * B * H), o_dz1 = take(sizeof(bf16) * B * H);
  const size_t o_t = take(sizeof(float) * B * NO), o_lg = take(sizeof(float) * B * NOP),
               o_rl = take(sizeof(float) * B), o_p = take(sizeof(float) * sp * H * H);
  const size_t o_err = take(sizeof(int));
  cudaError_t e = cudaMalloc(&s->mem, off);
  if (e != cudaSuccess) {
    delete s;
    return sfail(VCT_ERR_OOM, "surrogate buffers (%zu B): %s", off, cudaGetErrorString(e));
  }
  char *b = (char *)s->mem;
  s->w = (float *)(b + o_w);
  s->m = (float *)(b + o_m);
  s->v = (float *)(b + o_v);
  s->g = (float *)(b + o_g);
  s->W1b = (bf16 *)(b + o_w1);
  s->W2b = (bf16 *)(b + o_w2);
  s->W3b = (bf16 *)(b + o_w3);
  s->b1 = (float *)(b + o_b1);
  s->b2 = (float *)(b + o_b2);
  s->b3 = (float *)(b + o_b3);
  s->xb = (bf16 *)(b + o_xb);
  s->h1 = (bf16 *)(b + o_h1);
  s->h2 = (bf16 *)(b + o_h2);
  s->dz3 = (bf16 *)(b + o_dz3);
  s->dz2 = (bf16 *)(b + o_dz2);
  s->dz1 = (bf16 *)(b + o_dz1);
  s->tgt = (float *)(b + o_t);
  s->logits = (float *)(b + o_lg);
  s->row_loss = (float *)(b + o_rl);
  s->partial = (float *)(b + o_p);
  s->err = (int *)(b + o_err);
  // He-uniform initial weights (host RNG, seeded), zero biases and moments
  std::vector<float> w((size_t)kNParams, 0.0f);
  std::mt19937_64 rng(desc->seed);
  auto fill = [&](int64_t o, int64_t count, int fan_in) {
    const double lim = std::sqrt(6.0 / fan_in);
    std::uniform_real_distribution<double> u(-lim, lim);
    for (int64_t i = 0; i < count; ++i) w[(size_t)(o + i)] = (float)u(rng);
  };
  fill(kOffW1, (int64_t)H * NF, NF);
  fill(kOffW2, (int64_t)H * H, H);
  fill(kOffW3, (int64_t)NO * H, H);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  e = cudaMemsetAsync(s->mem, 0, off, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->w, w.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = refresh_bf16(s, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(s->mem);
    delete s;
    return sfail(VCT_ERR_CUDA, "surrogate init: %s", cudaGetErrorString(e));
  }
  *out = s;
  return VCT_OK;
}

vct_status vct_surrogate_destroy(vct_surrogate *s) {
  if (!s) return VCT_OK;
  cudaError_t e = cudaFree(s->mem);
  delete s;
  if (e != cudaSuccess) return sfail(VCT_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
  return VCT_OK;
}

size_t vct_surrogate_n_params(void) { return (size_t)kNParams; }

vct_status vct_surrogate_get(const vct_surrogate *s, float *weights, float *grads) {
  if (!s) return sfail(VCT_ERR_ARG, "surrogate is NULL");
  if (weights) S_CUDA(cudaMemcpy(weights, s->w, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  if (grads) S_CUDA(cudaMemcpy(grads, s->g, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
  return VCT_OK;
}

vct_status vct_surrogate_set(vct_surrogate *s, const float *weights, void *cuda_stream) {
  if (!s || !weights) return sfail(VCT_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  S_CUDA(cudaMemcpyAsync(s->w, weights, sizeof(float) * kNParams, cudaMemcpyHostToDevice, st));
  S_CUDA(refresh_bf16(s, st));
  S_CUDA(cudaStreamSynchronize(st));
  return VCT_OK;
}

vct_status vct_surrogate_features(const vct_surrogate *s, const vct_population *pop,
                                  const vct_scenario *scenarios, int32_t n_scen, float *dev_x,
                                  void *cuda_stream) {
  if (!s || !pop || (n_scen > 0 && (!scenarios || !dev_x))) return sfail(VCT_ERR_ARG, "NULL argument");
  if (n_scen <= 0 || pop->n == 0) return VCT_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *gains = nullptr;
  vct_status rc = upload_gains(scenarios, n_scen, st, &gains);
  if (rc) return rc;
  vct::FeatArgs f = feat_args(s, pop);
  f.gains = gains;
  f.n_scen = n_scen;
  f.n_rows = (int64_t)n_scen * pop->n;
  f.xf = dev_x;
  vct::features_kernel<<<blocks_for(f.n_rows, 256), 256, 0, st>>>(f);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(gains, st);
  if (e != cudaSuccess) return sfail(VCT_ERR_CUDA, "features: %s", cudaGetErrorString(e));
  return VCT_OK;
}

vct_status vct_surrogate_step(vct_surrogate *s, const float *dev_x, const float *dev_t, int64_t n_rows,
                              int32_t update, double *host_loss, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_surrogate_step");
  if (!s || !dev_x || !dev_t) return sfail(VCT_ERR_ARG, "NULL argument");
  vct_status rc = ensure_batch(s, n_rows);
  if (rc) return rc;
  if (n_rows < 1) return sfail(VCT_ERR_ARG, "n_rows < 1");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  vct::to_bf16_kernel<<<blocks_for(n_rows * KF, 256), 256, 0, st>>>(dev_x, n_rows * KF, KF, KF, s->xb);
  S_CUDA(cudaMemcpyAsync(s->tgt, dev_t, sizeof(float) * n_rows * NO, cudaMemcpyDeviceToDevice, st));
  if ((rc = train_rows(s, n_rows, update != 0, st))) return rc;
  if (host_loss && (rc = loss_of_rows(s, n_rows, st, host_loss))) return rc;
  return check_err(s, st);
}

vct_status vct_surrogate_train(vct_surrogate *s, const vct_population *pop, const vct_scenario *scenarios,
                               int32_t n_scen, const vct_patient_stats *dev_stats, int32_t epochs,
                               uint64_t shuffle_seed, double *host_epoch_loss, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_surrogate_train");
  if (!s || !pop || !scenarios || !dev_stats) return sfail(VCT_ERR_ARG, "NULL argument");
  if (n_scen < 1 || epochs < 0) return sfail(VCT_ERR_ARG, "n_scen >= 1 and epochs >= 0 required");
  const int64_t total = (int64_t)n_scen * pop->n;
  const int64_t B = s->batch;
  if (total < B) return sfail(VCT_ERR_ARG, "fewer samples (%lld) than one batch", (long long)total);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *gains = nullptr;
  vct_status rc = upload_gains(scenarios, n_scen, st, &gains);
  if (rc) return rc;
  int64_t *ids = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&ids, sizeof(int64_t) * total, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(gains, st);
    return sfail(VCT_ERR_OOM, "sample ids: %s", cudaGetErrorString(e));
  }
  std::vector<int64_t> perm((size_t)total);
  std::mt19937_64 rng(shuffle_seed);
  const int64_t steps = total / B;  // whole batches only
  for (int ep = 0; ep < epochs && rc == VCT_OK; ++ep) {
    for (int64_t i = 0; i < total; ++i) perm[(size_t)i] = i;
    std::shuffle(perm.begin(), perm.end(), rng);
    e = cudaMemcpyAsync(ids, perm.data(), sizeof(int64_t) * total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      rc = sfail(VCT_ERR_CUDA, "ids upload: %s", cudaGetErrorString(e));
      break;
    }
    double ep_loss = 0.0;
    for (int64_t b = 0; b < steps && rc == VCT_OK; ++b) {
      vct::FeatArgs f = feat_args(s, pop);
      f.gains = gains;
      f.n_scen = n_scen;
      f.ids = ids + b * B;
      f.n_rows = B;
      f.xb = s->xb;
      f.stats = dev_stats;
      f.t = s->tgt;
      vct::features_kernel<<<blocks_for(B, 256), 256, 0, st>>>(f);
      rc = train_rows(s, B, true, st);
      if (rc == VCT_OK && host_epoch_loss) {
        double l = 0.0;
        rc = loss_of_rows(s, B, st, &l);
        ep_loss += l;
      }
    }
    if (host_epoch_loss) host_epoch_loss[ep] = ep_loss / (double)steps;
  }
  cudaFreeAsync(ids, st);
  cudaFreeAsync(gains, st);
  if (rc != VCT_OK) return rc;
  return check_err(s, st);
}

vct_status vct_surrogate_inject_stall(vct_surrogate *s, int32_t on) {
  if (!s) return sfail(VCT_ERR_ARG, "surrogate is NULL");
  s->stall_test = on ? 1 : 0;
  return VCT_OK;
}

vct_status vct_surrogate_status(const vct_surrogate *s, void *cuda_stream) {
  if (!s) return sfail(VCT_ERR_ARG, "surrogate is NULL");
  return check_err(s, (cudaStream_t)cuda_stream);
}

vct_status vct_surrogate_predict(const vct_surrogate *s, const float *dev_x, int64_t n_rows, float *dev_p,
                                 void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_surrogate_predict");
  if (!s || (n_rows > 0 && (!dev_x || !dev_p))) return sfail(VCT_ERR_ARG, "NULL argument");
  if (n_rows <= 0) return VCT_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  bf16 *xb = nullptr;
  S_CUDA(cudaMallocAsync((void **)&xb, sizeof(bf16) * n_rows * KF, st));
  vct::to_bf16_kernel<<<blocks_for(n_rows * KF, 256), 256, 0, st>>>(dev_x, n_rows * KF, KF, KF, xb);
  vct::FwdArgs a = fwd_args(s);
  a.x = xb;
  a.n_rows = n_rows;
  a.p = dev_p;
  cudaError_t e = vct::launch_forward(a, vct::MODE_PREDICT, row_tiles(n_rows), st);
  cudaFreeAsync(xb, st);
  if (e != cudaSuccess) return sfail(VCT_ERR_CUDA, "predict: %s", cudaGetErrorString(e));
  return VCT_OK;
}

}  // extern "C"

namespace {
// Screening with the candidates' standardized log gains already in device memory.
vct_status screen_lg(const vct_surrogate *s, const vct_population *panel, const float *dev_lg,
                     int64_t n_cand, int32_t bin, float *dev_scores, cudaStream_t st) {
  const double one[3] = {1.0, 1.0, 1.0};
  double *gdev = nullptr;
  float *px = nullptr;
  S_CUDA(cudaMallocAsync((void **)&gdev, sizeof(one), st));
  S_CUDA(cudaMallocAsync((void **)&px, sizeof(float) * panel->n * KF, st));
  cudaError_t e = cudaMemcpyAsync(gdev, one, sizeof(one), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    // panel features (the gain slots are replaced per candidate)
    vct::FeatArgs f = feat_args(s, panel);
    f.gains = gdev;
    f.n_scen = 1;
    f.n_rows = panel->n;
    f.xf = px;
    vct::features_kernel<<<blocks_for(panel->n, 256), 256, 0, st>>>(f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    vct::FwdArgs a = fwd_args(s);
    a.panel_x = px;
    a.panel = (int32_t)panel->n;
    a.cand_lg = dev_lg;
    a.n_cand = n_cand;
    a.bin = bin;
    a.scores = dev_scores;
    e = vct::launch_forward(a, vct::MODE_SCREEN, n_cand, st);
  }
  cudaFreeAsync(gdev, st);
  cudaFreeAsync(px, st);
  if (e != cudaSuccess) return sfail(VCT_ERR_CUDA, "screen: %s", cudaGetErrorString(e));
  return VCT_OK;
}

vct_status screen_check(const vct_surrogate *s, const vct_population *panel, int64_t n_cand,
                        int32_t bin) {
  if (!s || !panel) return sfail(VCT_ERR_ARG, "NULL argument");
  if (bin < 0 || bin >= NO) return sfail(VCT_ERR_ARG, "bin must be in 0..4");
  if (panel->n < 1) return sfail(VCT_ERR_ARG, "empty panel");
  if (n_cand < 0) return sfail(VCT_ERR_ARG, "n_cand < 0");
  return VCT_OK;
}
}  // namespace

extern "C" {

vct_status vct_surrogate_screen(const vct_surrogate *s, const vct_population *panel, const double *host_gains,
                                int64_t n_cand, int32_t bin, float *dev_scores, void *cuda_stream) {
  vct_status rc = screen_check(s, panel, n_cand, bin);
  if (rc) return rc;
  if (n_cand == 0) return VCT_OK;
  if (!host_gains || !dev_scores) return sfail(VCT_ERR_ARG, "NULL argument");
  for (int64_t c = 0; c < 3 * n_cand; ++c)
    if (!(host_gains[c] > 0.0) || !std::isfinite(host_gains[c]))
      return sfail(VCT_ERR_ARG, "candidate %lld: gains must be > 0", (long long)(c / 3));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *g = nullptr;
  S_CUDA(cudaMallocAsync((void **)&g, sizeof(double) * 3 * n_cand, st));
  cudaError_t e = cudaMemcpyAsync(g, host_gains, sizeof(double) * 3 * n_cand, cudaMemcpyHostToDevice, st);
  rc = e == cudaSuccess ? vct_surrogate_screen_device(s, panel, g, n_cand, bin, dev_scores, cuda_stream)
                        : sfail(VCT_ERR_CUDA, "screen: %s", cudaGetErrorString(e));
  cudaFreeAsync(g, st);
  return rc;
}

vct_status vct_surrogate_screen_device(const vct_surrogate *s, const vct_population *panel,
                                       const double *dev_gains, int64_t n_cand, int32_t bin,
                                       float *dev_scores, void *cuda_stream) {
  vct::NvtxRange nvtx_range_("vct_surrogate_screen");
  vct_status rc = screen_check(s, panel, n_cand, bin);
  if (rc) return rc;
  if (n_cand == 0) return VCT_OK;
  if (!dev_gains || !dev_scores) return sfail(VCT_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float *lg = nullptr;
  S_CUDA(cudaMallocAsync((void **)&lg, sizeof(float) * 3 * n_cand, st));
  vct::cand_lg_kernel<<<blocks_for(3 * n_cand, 256), 256, 0, st>>>(
      dev_gains, n_cand, s->inv_sd[15], s->inv_sd[16], s->inv_sd[17], lg, s->err);
  cudaError_t e = cudaGetLastError();
  rc = e == cudaSuccess ? screen_lg(s, panel, lg, n_cand, bin, dev_scores, st)
                        : sfail(VCT_ERR_CUDA, "screen: %s", cudaGetErrorString(e));
  cudaFreeAsync(lg, st);
  return rc;
}

}  // extern "C"
