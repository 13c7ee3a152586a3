// vct_mlp_train.cu -- the surrogate network: features -> 256 -> 256 -> 5 range
// fractions (softmax), BF16 operands with FP32 accumulation on the tensor
// cores, trained on the simulator's own runs and used to screen controller
// tunings (the hyperparameters of the controller, Sec. III-B Eq. 3) before the
// closed-loop simulation (Sec. III) picks the best.  Not in the paper.
//
// Kernels
//   features_kernel    standardized features of (patient, scenario) pairs
//   forward (vct_mlp_fwd.cu) fused 3-layer forward on tcgen05, weights resident
//                      in shared memory (train: keeps H1, H2 and takes the softmax
//                      cross-entropy, the row losses, dZ3 and dZ2; predict:
//                      softmax; screen: mean range fraction per candidate)
//   tc_gemm (vct_mlp_gemm.cu) strided BF16 GEMM on tcgen05, split-K partials
//                      of a weight gradient with its bias gradient's, or
//                      ReLU-masked BF16 outputs (backward pass)
//   adamw_kernel       the split-K sums in a fixed order, then AdamW on FP32
//                      master weights and BF16 copies for the GEMMs
//                      (grad_kernel: the sums alone)
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
constexpr int kMaxSplits = 64;       // split-K factor of the weight gradients, at most
// Column-tile widths of the backward GEMMs: tiles narrower than the 256 a
// CTA could hold put more of these latency-bound launches on the SMs (128
// CTAs instead of 64; measured 0.158 -> 0.142 ms per training step call)
constexpr int kNTWeight = 128;       // weight gradients (split-K partials)
constexpr int kNTInput = 64;         // ReLU-masked input gradients

typedef __nv_bfloat16 bf16;

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

// Gather the rows ids[0 .. rows) of the precomputed feature and target tables
// into the batch buffers (16-byte chunks: KF BF16 features = 4 chunks).
// step (device, or null): the training call's step counter; the batch is then
// rows [(step mod steps) rows, +rows) of the epoch's shuffled ids (a CUDA graph
// of one step replays with the counter, not the arguments, advancing).
// coef (device, or null): thread 0 also writes the bias corrections of AdamW
// step t = base + step + 1 there, c1 = 1 / (1 - b1^t) and c2 = 1 / (1 - b2^t)
// (FP64), for the step's AdamW launch.
__global__ void gather_rows_kernel(const int64_t *ids, int64_t rows, const uint4 *x_all,
                                   const float *t_all, uint4 *xb, float *t, const int64_t *step,
                                   int64_t steps, double b1, double b2, int64_t base, float *coef) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (coef && i == 0) {
    const double tt = (double)(base + *step + 1);
    coef[0] = (float)(1.0 / (1.0 - pow(b1, tt)));
    coef[1] = (float)(1.0 / (1.0 - pow(b2, tt)));
  }
  if (step) ids += (*step % steps) * rows;
  constexpr int XC = KF * 2 / 16;  // chunks per feature row
  if (i < rows * XC) {
    const int64_t r = i / XC;
    xb[i] = x_all[ids[r] * XC + i % XC];
  }
  if (i < rows * NO) {
    const int64_t r = i / NO;
    t[i] = t_all[ids[r] * NO + i % NO];
  }
}

// The mean loss of a step's rows, in a fixed order, into out[*step] by one
// block of 256 threads; thread 0 then advances the step counter (the last
// write of a training step: the AdamW launch's extra block runs this).
__device__ void step_loss_block(const float *row_loss, int64_t rows, double *out, int64_t *step) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 256) s += (double)row_loss[r];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[*step] = sh[0] / (double)rows;
    *step += 1;
  }
}

// ------------------------------------------------------------------ AdamW
// One AdamW launch over the six parameter segments (W1, b1, W2, b2, W3, b3).
// Each gradient is the sum, in split order, of its weight-gradient GEMM's
// split-K partials (the bias gradients are partials of the same launch); the
// launch stores it in g as well.
struct AdamSeg {
  int64_t off, count;   // into the flat w, m, v, g arrays
  int cols, ld_b;       // master is [count / cols][cols]; BF16 copy is [rows][ld_b]
  bf16 *wb;             // BF16 copy for the kernels, or null
  float *wf;            // FP32 copy for the kernels (biases), or null
  int decay;
  const float *part;    // the segment's partials: element j of split z at part[z pstride + j]
  int splits;
  int64_t pstride;
  bf16 *wc;             // BF16 canonical image (canon_index, row length ld_b), or null
};
struct AdamArgs {
  float *w, *m, *v;
  float *g;
  AdamSeg seg[6];
  int n_seg;
  float lr, b1, b2, eps, wd, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
  const float *coef;                  // device (c1, c2) of the step, or null: c1, c2 above
  // a step whose count lives on the device: one extra block (the last) takes
  // the mean of the rows' losses into loss[*step] and advances the counter
  const float *row_loss;
  int64_t loss_rows;
  double *loss;                       // or null: no extra block
  int64_t *step;
};

// g = the sum over z, in order, of a segment's split-K partials at element j
__device__ __forceinline__ float split_sum(const AdamSeg &sg, int64_t j) {
  float g = 0.0f;
#pragma unroll 8
  for (int z = 0; z < sg.splits; ++z) g += sg.part[(int64_t)z * sg.pstride + j];  // loads batched, sum in order
  return g;
}

// The gradients alone (a step without an update).
__global__ void grad_kernel(AdamArgs a) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int s = 0;
  while (s < a.n_seg && j >= a.seg[s].count) j -= a.seg[s++].count;
  if (s >= a.n_seg) return;
  a.g[a.seg[s].off + j] = split_sum(a.seg[s], j);
}

__global__ void adamw_kernel(AdamArgs a) {
  if (a.loss && blockIdx.x == gridDim.x - 1) {
    step_loss_block(a.row_loss, a.loss_rows, a.loss, a.step);
    return;
  }
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int s = 0;
  while (s < a.n_seg && j >= a.seg[s].count) j -= a.seg[s++].count;
  if (s >= a.n_seg) return;
  const AdamSeg &sg = a.seg[s];
  const int64_t i = sg.off + j;
  const float g = split_sum(sg, j);
  a.g[i] = g;
  const float m = a.b1 * a.m[i] + (1.0f - a.b1) * g;
  const float v = a.b2 * a.v[i] + (1.0f - a.b2) * g * g;
  a.m[i] = m;
  a.v[i] = v;
  float w = a.w[i];
  if (sg.decay) w -= a.lr * a.wd * w;
  const float c1 = a.coef ? a.coef[0] : a.c1, c2 = a.coef ? a.coef[1] : a.c2;
  w -= a.lr * (m * c1) / (sqrtf(v * c2) + a.eps);
  a.w[i] = w;
  if (sg.wb) {
    const bf16 wv = __float2bfloat16_rn(w);
    sg.wb[(j / sg.cols) * sg.ld_b + j % sg.cols] = wv;
    sg.wc[canon_index((int)(j / sg.cols), (int)(j % sg.cols), sg.ld_b)] = wv;
  }
  if (sg.wf) sg.wf[j] = w;
}

__global__ void to_bf16_kernel(const float *w, int64_t count, int cols, int ld_b, bf16 *wb, bf16 *wc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const bf16 v = __float2bfloat16_rn(w[i]);
  wb[(i / cols) * ld_b + i % cols] = v;
  if (wc) wc[canon_index((int)(i / cols), (int)(i % cols), ld_b)] = v;
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
  // the same in the forward kernel's shared-memory layout (canon_index)
  __nv_bfloat16 *W1c, *W2c, *W3c;
  float *b1, *b2, *b3;  // padded copies for the forward (b3: [8])
  int64_t step;
  // training buffers (batch rows): xb [batch][KF], dz3 [batch][16], dz1 [batch][H];
  // h1, h2, dz2 chunk-major (act_cs)
  __nv_bfloat16 *xb, *h1, *h2, *dz3, *dz2, *dz1;
  float *tgt, *row_loss;
  float *part[3];  // split-K partials of the weight and bias gradients of layers 1, 2, 3
  int64_t batch;
  int *err;  // device: set by the forward kernel if a bounded wait gives up
  int stall_test;  // test hook (vct_surrogate_inject_stall)
  // the backward pass's second stream: two weight-gradient GEMMs run beside the
  // main stream's two GEMMs (fork and join through the two events)
  cudaStream_t side;
  cudaEvent_t ev[2];
};

namespace {

using vct::H;
using vct::KF;
using vct::NF;
using vct::NO;
using vct::NOK;
using vct::NOP;
using vct::kMaxSplits;
using vct::kNTInput;
using vct::kNTWeight;
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
  // padded BF16 copies, plain and as canonical images: W1 [H][KF] (cols >= NF
  // zero), W2 [H][H], W3 [NOK][H] (rows >= NO zero; the padding stays zero)
  vct::to_bf16_kernel<<<blocks_for((int64_t)H * NF, 256), 256, 0, st>>>(s->w + kOffW1, (int64_t)H * NF, NF, KF,
                                                                        s->W1b, s->W1c);
  vct::to_bf16_kernel<<<blocks_for((int64_t)H * H, 256), 256, 0, st>>>(s->w + kOffW2, (int64_t)H * H, H, H, s->W2b,
                                                                       s->W2c);
  vct::to_bf16_kernel<<<blocks_for((int64_t)NO * H, 256), 256, 0, st>>>(s->w + kOffW3, (int64_t)NO * H, H, H,
                                                                        s->W3b, s->W3c);
  cudaError_t e = cudaMemcpyAsync(s->b1, s->w + kOffB1, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->b2, s->w + kOffB2, sizeof(float) * H, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->b3, s->w + kOffB3, sizeof(float) * NO, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

vct::FwdArgs fwd_args(const vct_surrogate *s) {
  vct::FwdArgs a;
  std::memset(&a, 0, sizeof(a));
  a.W1 = s->W1c;
  a.W2 = s->W2c;
  a.W3 = s->W3c;
  a.b1 = s->b1;
  a.b2 = s->b2;
  a.b3 = s->b3;
  a.error = s->err;
  a.stall_test = s->stall_test;
  return a;
}

int64_t row_tiles(int64_t rows) { return (rows + 127) / 128; }

// H1, H2 and dZ2 are stored chunk-major for the batch capacity: unit u of row r
// at (u / 8) act_cs + 8 r + u % 8, so that the forward's epilogue stores
// coalesce (its lanes hold consecutive rows)
int64_t act_cs(const vct_surrogate *s) { return 8 * s->batch; }

// C (split-K partials or masked BF16) = A B with strided operands, on tcgen05:
// tiles of 128 rows x NT columns (NT = N rounded up to 16, at most kNTWeight for
// the split-K partials and kNTInput for the masked outputs, which have no
// split-K), split z covering k in [z kc, (z+1) kc) with kc a multiple of 64.
// Operand and mask layouts as TcGemmArgs describes them: Mat gives a plainly
// stored or chunk-major matrix.
// A matrix X[r][c] with one unit stride: at p[r sr + (c / 8) cs + c % 8] when
// sc == 1 (cs = 8 when stored plainly), at p[c sc + (r / 8) cs + r % 8] when sr == 1.
struct Mat {
  const bf16 *p;
  int64_t sr, sc, cs;
};
Mat plain(const bf16 *p, int64_t sr, int64_t sc) { return Mat{p, sr, sc, 8}; }

cudaError_t gemm(int mode, Mat A, Mat B, int M, int N, int64_t K, float *partial, int splits, bf16 *out,
                 Mat mask, int *err, cudaStream_t st, int64_t pstride = 0, float *bias_partial = nullptr) {
  // a K-contiguous operand is staged in 16-byte chunks along K (K a multiple of
  // 8); the other form reads one K row at a time (any K); chunk strides and the
  // other stride are multiples of 8 elements (16-byte chunks)
  auto mat_ok = [](const Mat &x) {
    return ((x.sc == 1 && x.sr % 8 == 0) || (x.sr == 1 && x.sc % 8 == 0)) && x.cs % 8 == 0 &&
           !((uintptr_t)x.p & 15);
  };
  const bool k_ok = (A.sc != 1 && B.sr != 1) || K % 8 == 0;
  if (!mat_ok(A) || !mat_ok(B) || !k_ok || M < 1 || N < 1 || K < 1) return cudaErrorInvalidValue;
  if (mode == 0 && (pstride < (int64_t)M * N || (bias_partial && A.sr != 1))) return cudaErrorInvalidValue;
  if (mode == 1 && (mask.sc != 1 || mask.cs % 8 != 0)) return cudaErrorInvalidValue;
  vct::TcGemmArgs g;
  std::memset(&g, 0, sizeof(g));
  g.A = A.p;
  g.sam = A.sr;
  g.sak = A.sc;
  g.acs = A.cs;
  g.B = B.p;
  g.sbk = B.sr;
  g.sbn = B.sc;
  g.bcs = B.cs;
  g.M = M;
  g.N = N;
  g.NT = std::min((N + 15) / 16 * 16, mode == 0 ? kNTWeight : kNTInput);
  g.K = K;
  g.kc = ((K + splits - 1) / splits + 63) / 64 * 64;
  g.mode = mode;
  g.partial = partial;
  g.pstride = pstride;
  g.bias_partial = bias_partial;
  g.out = out;
  g.mask = mask.p;
  g.mrs = mask.sr;
  g.mcs = mask.cs;
  g.error = err;
  const int sp = (int)((K + g.kc - 1) / g.kc);
  return vct::launch_tc_gemm(g, (N + g.NT - 1) / g.NT, (M + 127) / 128, sp, st);
}

// split-K factor of a weight gradient: about 128 CTAs, K slices of >= 64
int splits_for(int64_t K, int M, int N) {
  const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + kNTWeight - 1) / kNTWeight);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(kMaxSplits, K / 64),
                                                       std::max<int64_t>(1, 128 / tiles)));
}

// Weight and bias gradients of one layer, dW [M][N] = dZ^T [M][B] X [B][N] and
// db [M] = dZ^T 1, as split-K partials: split z's dW at part + z (M N + M), its
// db right behind (the parameter vector's layout, W then b).  dzt is dZ^T
// (stored along M), x is X.  Returns the splits in *splits; AdamW (or
// grad_kernel) adds them up.
cudaError_t weight_grad(vct_surrogate *s, Mat dzt, int M, Mat x, int N, int64_t B, float *part, int *splits,
                        cudaStream_t st) {
  int sp = splits_for(B, M, N);
  const int64_t kc = ((B + sp - 1) / sp + 63) / 64 * 64;
  sp = (int)((B + kc - 1) / kc);  // the splits the launch makes
  *splits = sp;
  const int64_t pstride = (int64_t)M * N + M;
  return gemm(0, dzt, x, M, N, B, part, sp, nullptr, Mat{}, s->err, st, pstride, part + (int64_t)M * N);
}

// Floats of one layer's split-K partials for batches of up to B rows.
int64_t partial_floats(int64_t B, int M, int N) {
  const int sp = splits_for(B, M, N);
  const int64_t kc = ((B + sp - 1) / sp + 63) / 64 * 64;
  return ((B + kc - 1) / kc) * ((int64_t)M * N + M);
}

vct_status ensure_batch(vct_surrogate *s, int64_t B) {
  if (B <= s->batch) return VCT_OK;
  return sfail(VCT_ERR_ARG, "batch %lld exceeds the surrogate's batch capacity %lld", (long long)B,
               (long long)s->batch);
}

// The device step counter of a graph-captured training step (null: host-driven):
// AdamW takes its bias corrections from coef, computed on the device for step
// base + *step + 1.
struct DevStep {
  int64_t *step;   // steps done in this call
  float *coef;     // the step's AdamW bias corrections (written by the gather)
  double *loss;    // the mean loss of every step of the call
};

// forward + loss + backward on the rows already in s->xb / s->tgt; then AdamW if update
vct_status train_rows(vct_surrogate *s, int64_t B, bool update, cudaStream_t st,
                      const DevStep *ds = nullptr) {
  vct::FwdArgs a = fwd_args(s);
  a.x = s->xb;
  a.n_rows = B;
  a.h1 = s->h1;
  a.h2 = s->h2;
  a.act_cs = act_cs(s);
  // the forward's last epilogue also takes the softmax cross-entropy (row losses
  // and dZ3 = (p sum(t) - t) / B) and dZ2 = (dZ3 W3) * [Z2 > 0]
  a.tgt = s->tgt;
  a.dz3 = s->dz3;
  a.dz2 = s->dz2;
  a.row_loss = s->row_loss;
  a.inv_b = 1.0f / (float)B;
  S_CUDA(vct::launch_forward(a, vct::MODE_TRAIN, row_tiles(B), st));
  // Two chains of two GEMMs each from the forward's outputs: dZ1 = (dZ2 W2) *
  // [H1 > 0], then layer 1's weight and bias gradients on the main stream;
  // layers 2 and 3's on the side stream (they read what the forward wrote and
  // write only their partials), which rejoins before the split-K sums.
  cudaStream_t sd = s->side;
  int sp[3];
  S_CUDA(cudaEventRecord(s->ev[0], st));
  S_CUDA(cudaStreamWaitEvent(sd, s->ev[0], 0));
  // layer 2: dW2 = dZ2^T H1, db2 = dZ2^T 1; layer 3: dW3 = dZ3^T H2, db3 = dZ3^T 1 (partials);
  // H1, H2 and dZ2 chunk-major (row r of a chunk 8 elements on), dZ3 [B][16]
  const int64_t cs = act_cs(s);
  S_CUDA(weight_grad(s, Mat{s->dz2, 1, 8, cs}, H, Mat{s->h1, 8, 1, cs}, H, B, s->part[1], &sp[1], sd));
  S_CUDA(weight_grad(s, plain(s->dz3, 1, NOK), NO, Mat{s->h2, 8, 1, cs}, H, B, s->part[2], &sp[2], sd));
  // layer 1: dZ1 = (dZ2 W2) * [H1 > 0] ([B][H]), dW1 = dZ1^T X, db1 = dZ1^T 1
  S_CUDA(gemm(1, Mat{s->dz2, 8, 1, cs}, plain(s->W2b, H, 1), (int)B, H, H, nullptr, 1, s->dz1,
              Mat{s->h1, 8, 1, cs}, s->err, st));
  S_CUDA(weight_grad(s, plain(s->dz1, 1, H), H, plain(s->xb, KF, 1), NF, B, s->part[0], &sp[0], st));
  S_CUDA(cudaEventRecord(s->ev[1], sd));
  S_CUDA(cudaStreamWaitEvent(st, s->ev[1], 0));
  S_CUDA(cudaGetLastError());
  // the six segments and their partials (W then b of each layer)
  const int lay_m[3] = {H, H, NO}, lay_n[3] = {NF, H, H};
  const vct::AdamSeg segs[6] = {{kOffW1, (int64_t)H * NF, NF, KF, s->W1b, nullptr, 1},
                                {kOffB1, H, H, H, nullptr, s->b1, 0},
                                {kOffW2, (int64_t)H * H, H, H, s->W2b, nullptr, 1},
                                {kOffB2, H, H, H, nullptr, s->b2, 0},
                                {kOffW3, (int64_t)NO * H, H, H, s->W3b, nullptr, 1},
                                {kOffB3, NO, NO, NO, nullptr, s->b3, 0}};
  vct::AdamArgs A;
  std::memset(&A, 0, sizeof(A));
  A.w = s->w;
  A.m = s->m;
  A.v = s->v;
  A.g = s->g;
  A.n_seg = 6;
  int64_t total = 0;
  for (int j = 0; j < 6; ++j) {
    const int l = j / 2;
    A.seg[j] = segs[j];
    A.seg[j].part = s->part[l] + (j % 2 ? (int64_t)lay_m[l] * lay_n[l] : 0);
    A.seg[j].splits = sp[l];
    A.seg[j].pstride = (int64_t)lay_m[l] * lay_n[l] + lay_m[l];
    A.seg[j].wc = j % 2 ? nullptr : (l == 0 ? s->W1c : (l == 1 ? s->W2c : s->W3c));
    total += segs[j].count;
  }
  if (!update) {
    vct::grad_kernel<<<blocks_for(total, 256), 256, 0, st>>>(A);
    S_CUDA(cudaGetLastError());
  } else {
    const vct_surrogate_desc &d = s->desc;
    A.lr = (float)d.lr;
    A.b1 = (float)d.beta1;
    A.b2 = (float)d.beta2;
    A.eps = (float)d.eps;
    A.wd = (float)d.weight_decay;
    if (ds) {  // the step count lives on the device (graph replay)
      A.coef = ds->coef;
      A.row_loss = s->row_loss;
      A.loss_rows = B;
      A.loss = ds->loss;
      A.step = ds->step;
    } else {
      s->step += 1;
      A.c1 = (float)(1.0 / (1.0 - std::pow(d.beta1, (double)s->step)));
      A.c2 = (float)(1.0 / (1.0 - std::pow(d.beta2, (double)s->step)));
    }
    vct::adamw_kernel<<<blocks_for(total, 256) + (A.loss ? 1 : 0), 256, 0, st>>>(A);
    S_CUDA(cudaGetLastError());
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
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = al(off + bytes); return o; };
  const size_t o_w = take(sizeof(float) * kNParams), o_m = take(sizeof(float) * kNParams),
               o_v = take(sizeof(float) * kNParams), o_g = take(sizeof(float) * kNParams);
  const size_t o_w1 = take(sizeof(bf16) * H * KF), o_w2 = take(sizeof(bf16) * H * H),
               o_w3 = take(sizeof(bf16) * NOK * H);
  const size_t o_w1c = take(sizeof(bf16) * H * KF), o_w2c = take(sizeof(bf16) * H * H),
               o_w3c = take(sizeof(bf16) * NOK * H);
  const size_t o_b1 = take(sizeof(float) * H), o_b2 = take(sizeof(float) * H), o_b3 = take(sizeof(float) * NOP);
  const size_t o_xb = take(sizeof(bf16) * B * KF), o_h1 = take(sizeof(bf16) * B * H),
               o_h2 = take(sizeof(bf16) * B * H), o_dz3 = take(sizeof(bf16) * B * NOK),
               o_dz2 = take(sizeof(bf16) * B * H), o_dz1 = take(sizeof(bf16) * B * H);
  const size_t o_t = take(sizeof(float) * B * NO),
               o_rl = take(sizeof(float) * B);
  const size_t o_p1 = take(sizeof(float) * partial_floats(B, H, NF)),
               o_p2 = take(sizeof(float) * partial_floats(B, H, H)),
               o_p3 = take(sizeof(float) * partial_floats(B, NO, H));
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
  s->W1c = (bf16 *)(b + o_w1c);
  s->W2c = (bf16 *)(b + o_w2c);
  s->W3c = (bf16 *)(b + o_w3c);
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
  s->row_loss = (float *)(b + o_rl);
  s->part[0] = (float *)(b + o_p1);
  s->part[1] = (float *)(b + o_p2);
  s->part[2] = (float *)(b + o_p3);
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
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaEventCreateWithFlags(&s->ev[j], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    for (int j = 0; j < 2; ++j)
      if (s->ev[j]) cudaEventDestroy(s->ev[j]);
    if (s->side) cudaStreamDestroy(s->side);
    cudaFree(s->mem);
    delete s;
    return sfail(VCT_ERR_CUDA, "surrogate init: %s", cudaGetErrorString(e));
  }
  *out = s;
  return VCT_OK;
}

vct_status vct_surrogate_destroy(vct_surrogate *s) {
  if (!s) return VCT_OK;
  for (int j = 0; j < 2; ++j) cudaEventDestroy(s->ev[j]);
  cudaStreamDestroy(s->side);
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
  vct::to_bf16_kernel<<<blocks_for(n_rows * KF, 256), 256, 0, st>>>(dev_x, n_rows * KF, KF, KF, s->xb, nullptr);
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
  const int64_t steps = total / B;  // whole batches only
  // Device memory of the call: the sample ids of one epoch, every sample's
  // feature row (BF16) and target row, computed once and gathered per step, and
  // the loss of every step (read once at the end: no synchronisation per step).
  double *gains = nullptr;
  vct_status rc = upload_gains(scenarios, n_scen, st, &gains);
  if (rc) return rc;
  int64_t *ids = nullptr;
  bf16 *x_all = nullptr;
  float *t_all = nullptr;
  double *step_loss = nullptr;
  int64_t *pinned[2] = {nullptr, nullptr};
  cudaEvent_t copied[2] = {nullptr, nullptr};
  const int64_t n_loss = std::max<int64_t>(1, (int64_t)epochs * steps);
  int64_t *dstep = nullptr;  // [0]: steps done in this call; then two floats of AdamW coefficients
  cudaError_t e = cudaMallocAsync((void **)&ids, sizeof(int64_t) * total, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&x_all, sizeof(bf16) * KF * total, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&t_all, sizeof(float) * NO * total, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&step_loss, sizeof(double) * n_loss, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&dstep, 256, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dstep, 0, 256, st);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
    e = cudaMallocHost((void **)&pinned[j], sizeof(int64_t) * total);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copied[j], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) rc = sfail(VCT_ERR_OOM, "training buffers: %s", cudaGetErrorString(e));
  if (rc == VCT_OK) {
    vct::FeatArgs f = feat_args(s, pop);
    f.gains = gains;
    f.n_scen = n_scen;
    f.ids = nullptr;  // every sample, in id order
    f.n_rows = total;
    f.xb = x_all;
    f.stats = dev_stats;
    f.t = t_all;
    vct::features_kernel<<<blocks_for(total, 256), 256, 0, st>>>(f);
    if ((e = cudaGetLastError()) != cudaSuccess) rc = sfail(VCT_ERR_CUDA, "features: %s", cudaGetErrorString(e));
  }
  // One training step (gather the batch, forward, loss, backward, AdamW, the
  // step's loss and the counter's advance) captured once in a CUDA graph and
  // replayed for every batch: the arguments are fixed, the device counter
  // selects the batch rows, the AdamW bias corrections and the loss slot.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (rc == VCT_OK && epochs > 0) {
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // buffers ready before the capture
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const DevStep ds{dstep, (float *)(dstep + 1), step_loss};
      vct::gather_rows_kernel<<<blocks_for(B * NO, 256), 256, 0, cap>>>(
          ids, B, (const uint4 *)x_all, t_all, (uint4 *)s->xb, s->tgt, dstep, steps, s->desc.beta1,
          s->desc.beta2, s->step, ds.coef);
      vct_status r2 = train_rows(s, B, true, cap, &ds);
      cudaError_t ec = cudaStreamEndCapture(cap, &graph);
      e = r2 != VCT_OK ? cudaErrorUnknown : (ec != cudaSuccess ? ec : cudaGetLastError());
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) rc = sfail(VCT_ERR_CUDA, "training step graph: %s", cudaGetErrorString(e));
  }
  std::mt19937_64 rng(shuffle_seed);
  for (int ep = 0; ep < epochs && rc == VCT_OK; ++ep) {
    // the epoch's shuffle, written into the pinned buffer whose previous copy is done
    int64_t *perm = pinned[ep & 1];
    if ((e = cudaEventSynchronize(copied[ep & 1])) != cudaSuccess) {
      rc = sfail(VCT_ERR_CUDA, "ids buffer: %s", cudaGetErrorString(e));
      break;
    }
    for (int64_t i = 0; i < total; ++i) perm[i] = i;
    std::shuffle(perm, perm + total, rng);
    e = cudaMemcpyAsync(ids, perm, sizeof(int64_t) * total, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(copied[ep & 1], st);
    if (e != cudaSuccess) {
      rc = sfail(VCT_ERR_CUDA, "ids upload: %s", cudaGetErrorString(e));
      break;
    }
    for (int64_t b = 0; b < steps && rc == VCT_OK; ++b) {
      if ((e = cudaGraphLaunch(exec, st)) != cudaSuccess)
        rc = sfail(VCT_ERR_CUDA, "training step: %s", cudaGetErrorString(e));
    }
  }
  if (rc == VCT_OK) s->step += (int64_t)epochs * steps;  // AdamW steps taken on the device
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (rc == VCT_OK && host_epoch_loss && epochs > 0) {
    std::vector<double> l((size_t)n_loss);
    e = cudaMemcpyAsync(l.data(), step_loss, sizeof(double) * n_loss, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = sfail(VCT_ERR_CUDA, "epoch losses: %s", cudaGetErrorString(e));
    for (int ep = 0; ep < epochs && rc == VCT_OK; ++ep) {
      double sum = 0.0;
      for (int64_t b = 0; b < steps; ++b) sum += l[(size_t)(ep * steps + b)];
      host_epoch_loss[ep] = sum / (double)steps;
    }
  }
  // the pinned buffers may still feed a copy: wait before freeing them
  cudaStreamSynchronize(st);
  for (int j = 0; j < 2; ++j) {
    if (copied[j]) cudaEventDestroy(copied[j]);
    if (pinned[j]) cudaFreeHost(pinned[j]);
  }
  cudaFreeAsync(dstep, st);
  cudaFreeAsync(step_loss, st);
  cudaFreeAsync(t_all, st);
  cudaFreeAsync(x_all, st);
  cudaFreeAsync(ids, st);
  cudaFreeAsync(gains, st);
  if (rc != VCT_OK) return rc;
  return check_err(s, st);
}

vct_status vct_surrogate_set_lr(vct_surrogate *s, double lr) {
  if (!s) return sfail(VCT_ERR_ARG, "surrogate is NULL");
  if (!(lr > 0.0) || !std::isfinite(lr)) return sfail(VCT_ERR_ARG, "lr must be finite and > 0");
  s->desc.lr = lr;
  return VCT_OK;
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
  vct::to_bf16_kernel<<<blocks_for(n_rows * KF, 256), 256, 0, st>>>(dev_x, n_rows * KF, KF, KF, xb, nullptr);
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
