// vct_mlp_fwd.cu -- the surrogate's fused forward pass on the 5th-generation
// tensor cores (tcgen05): one CTA of 128 threads per SM keeps all three weight
// matrices in shared memory, takes 128 rows at a time, and runs
//   layer 1: D1 = X W1^T       (TMEM columns   0..255, K = 32)
//   layer 2: D2 = H1 W2^T      (TMEM columns 256..511, K = 256)
//   layer 3: D3 = H2 W3^T      (TMEM columns   0..15,  K = 256, N = 16 >= 5)
// with BF16 operands from shared memory and FP32 accumulators in TMEM; one
// thread issues the MMAs and commits them to an mbarrier, the epilogues read
// TMEM with tcgen05.ld (thread t owns row t), add the bias, apply ReLU and
// write the BF16 activations back into shared memory for the next layer.
// Operands use the canonical K-major layout without swizzle: element (r, k)
// of an R x K operand sits at (r/8)(16 K) + (k/8) 128 + (r%8) 16 + (k%8) 2
// bytes, i.e. 8 x 16-byte core matrices, contiguous along K.
#include "vct_mlp.cuh"

namespace vct {
namespace {

constexpr int TM = 128;       // rows per tile = TMEM lanes
constexpr int THREADS = 256;  // 8 warps: warps w and w + 4 share TMEM lanes 32w..32w+31 and
                              // split the columns of a row between them
constexpr int H = kSurrH, KF = kSurrKF, NO = kSurrNO, NOP = kSurrNOP;
constexpr int N3 = 16;        // layer-3 MMA width
constexpr uint32_t kTmemCols = 512;
constexpr long kWaitLimit = 1L << 24;

// shared memory map (bytes)
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + H * KF * 2;
constexpr int OFF_W3 = OFF_W2 + H * H * 2;
constexpr int OFF_X = OFF_W3 + N3 * H * 2;
constexpr int OFF_H = OFF_X + TM * KF * 2;
constexpr int OFF_B1 = OFF_H + TM * H * 2;
constexpr int OFF_B2 = OFF_B1 + H * 4;
constexpr int OFF_B3 = OFF_B2 + H * 4;
constexpr int OFF_BAR = OFF_B3 + N3 * 4;
constexpr int OFF_TMEM = OFF_BAR + 8;
constexpr int OFF_RED = OFF_TMEM + 8;
constexpr int SMEM_BYTES = OFF_RED + 8 * 4;
static_assert(SMEM_BYTES <= 232448, "shared memory");

__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int K) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;                // K-direction core-matrix step
  d |= (uint64_t)(((uint32_t)(K * 16) >> 4) & 0x3FFF) << 32;  // 8-row group step
  d |= (uint64_t)1 << 46;                                      // descriptor version
  return d;                                                    // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// Bounded wait for the mbarrier phase; the block agrees on the outcome.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t phase) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
  const bool ok = __syncthreads_and(done != 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Make this thread's shared-memory writes visible to the tensor cores, then
// meet at the block barrier.
__device__ __forceinline__ void publish_smem() {
  asm volatile("tcgen05.fence::before_thread_sync;");
  asm volatile("fence.proxy.async.shared::cta;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ uint4 pack8(const float *f) {
  __nv_bfloat162 p0 = __floats2bfloat162_rn(f[0], f[1]), p1 = __floats2bfloat162_rn(f[2], f[3]),
                 p2 = __floats2bfloat162_rn(f[4], f[5]), p3 = __floats2bfloat162_rn(f[6], f[7]);
  uint4 u;
  u.x = *reinterpret_cast<uint32_t *>(&p0);
  u.y = *reinterpret_cast<uint32_t *>(&p1);
  u.z = *reinterpret_cast<uint32_t *>(&p2);
  u.w = *reinterpret_cast<uint32_t *>(&p3);
  return u;
}

// copy a row-major BF16 [rows][K] matrix into the canonical layout
__device__ void stage_matrix(unsigned char *dst, const __nv_bfloat16 *src, int rows, int K) {
  const int chunks = rows * (K / 8);
  for (int c = threadIdx.x; c < chunks; c += THREADS) {
    const int r = c / (K / 8), k = (c % (K / 8)) * 8;
    *reinterpret_cast<uint4 *>(dst + cm_off(r, k, K)) =
        *reinterpret_cast<const uint4 *>(src + (int64_t)r * K + k);
  }
}

// hidden-layer epilogue: thread (row, half) takes 128 of the row's 256 columns
// from TMEM, 32 per load, adds the bias, applies ReLU and stores BF16
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, uint32_t col0, const float *bias,
                                                unsigned char *hs, __nv_bfloat16 *glob, int row,
                                                int64_t grow, bool store_glob) {
  const int half = threadIdx.x >> 7;
  const uint32_t lane_addr = tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + col0;
#pragma unroll 1
  for (int c0 = half * (H / 2); c0 < (half + 1) * (H / 2); c0 += 32) {
    float v[32];
    tmem_ld32(lane_addr + c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + bias[c0 + j], 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 u = pack8(v + 8 * q);
      *reinterpret_cast<uint4 *>(hs + cm_off(row, c0 + 8 * q, H)) = u;
      if (store_glob) *reinterpret_cast<uint4 *>(glob + grow * H + c0 + 8 * q) = u;
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) forward_tc_kernel(FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float *b1 = reinterpret_cast<float *>(smem + OFF_B1);
  float *b2 = reinterpret_cast<float *>(smem + OFF_B2);
  float *b3 = reinterpret_cast<float *>(smem + OFF_B3);
  float *red = reinterpret_cast<float *>(smem + OFF_RED);
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = s_base + OFF_BAR;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_TMEM);

  stage_matrix(smem + OFF_W1, a.W1, H, KF);
  stage_matrix(smem + OFF_W2, a.W2, H, H);
  stage_matrix(smem + OFF_W3, a.W3, N3, H);
  for (int e = tid; e < H; e += THREADS) {
    b1[e] = a.b1[e];
    b2[e] = a.b2[e];
  }
  if (tid < N3) b3[tid] = tid < NO ? a.b3[tid] : 0.0f;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + OFF_TMEM),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  publish_smem();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;
  bool ok = true;

  const uint64_t dW1 = smem_desc(s_base + OFF_W1, KF), dW2 = smem_desc(s_base + OFF_W2, H),
                 dW3 = smem_desc(s_base + OFF_W3, H), dX = smem_desc(s_base + OFF_X, KF),
                 dH = smem_desc(s_base + OFF_H, H);
  const int64_t tiles_per_item = MODE == MODE_SCREEN ? (a.panel + TM - 1) / TM : 1;
  const int64_t n_items = MODE == MODE_SCREEN ? a.n_cand : (a.n_rows + TM - 1) / TM;
  const bool panel_cached = MODE == MODE_SCREEN && tiles_per_item == 1;
  float pf[16];  // this thread's 16 panel features (screening)

  for (int64_t item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
    float score = 0.0f;
    for (int64_t tile = 0; tile < tiles_per_item && ok; ++tile) {
      const int64_t row0 = MODE == MODE_SCREEN ? tile * TM : item * TM;
      const int64_t limit = MODE == MODE_SCREEN ? (int64_t)a.panel : a.n_rows;
      const int row = tid & (TM - 1), half = tid >> 7;
      const bool valid = row0 + row < limit;
      const int64_t grow = row0 + row;
      // input row, canonical layout: each of the row's two threads owns two
      // 8-feature chunks (half 0: features 0-15, half 1: 16-31)
      unsigned char *xs = smem + OFF_X;
      if (MODE != MODE_SCREEN) {
        if (valid) {
          const uint4 *src = reinterpret_cast<const uint4 *>(a.x + grow * KF);
#pragma unroll
          for (int c = 2 * half; c < 2 * half + 2; ++c)
            *reinterpret_cast<uint4 *>(xs + cm_off(row, 8 * c, KF)) = src[c];
        } else {
          const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
          for (int c = 2 * half; c < 2 * half + 2; ++c) *reinterpret_cast<uint4 *>(xs + cm_off(row, 8 * c, KF)) = z;
        }
      } else {
        // panel features of this row (the same for every candidate): loaded once
        // when the panel fits one tile, per tile otherwise
        if (!panel_cached || (item == blockIdx.x && tile == 0)) {
          if (valid) {
            const float4 *src = reinterpret_cast<const float4 *>(a.panel_x + grow * KF + 16 * half);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 v4 = src[q];
              pf[4 * q] = v4.x;
              pf[4 * q + 1] = v4.y;
              pf[4 * q + 2] = v4.z;
              pf[4 * q + 3] = v4.w;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) pf[q] = 0.0f;
          }
          *reinterpret_cast<uint4 *>(xs + cm_off(row, 16 * half, KF)) = pack8(pf);
          *reinterpret_cast<uint4 *>(xs + cm_off(row, 16 * half + 8, KF)) = pack8(pf + 8);
        }
        // the candidate's standardized log gains are features 15, 16, 17:
        // chunk 1 (half 0, slot 15) and chunk 2 (half 1, slots 16 and 17)
        float ch[8];
        if (half == 0) {
#pragma unroll
          for (int q = 0; q < 8; ++q) ch[q] = pf[8 + q];
          if (valid) ch[7] = a.cand_lg[item * 3];
          *reinterpret_cast<uint4 *>(xs + cm_off(row, 8, KF)) = pack8(ch);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) ch[q] = pf[q];
          if (valid) {
            ch[0] = a.cand_lg[item * 3 + 1];
            ch[1] = a.cand_lg[item * 3 + 2];
          }
          *reinterpret_cast<uint4 *>(xs + cm_off(row, 16, KF)) = pack8(ch);
        }
      }
      publish_smem();
      // layer 1
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < KF / 16; ++ks) mma(tmem, dX + 16 * ks, dW1 + 16 * ks, idesc_bf16(TM, H), ks > 0);
        commit(bar);
      }
      ok = wait_phase(bar, phase);
      phase ^= 1u;
      if (!ok) break;
      hidden_epilogue(tmem, 0, b1, smem + OFF_H, a.h1, row, grow, MODE == MODE_TRAIN && valid);
      publish_smem();
      // layer 2 (descriptor start addresses advance 256 B = 16 in >> 4 units per k step)
      if (tid == 0) {
#pragma unroll 1
        for (int ks = 0; ks < H / 16; ++ks) mma(tmem + 256, dH + 16 * ks, dW2 + 16 * ks, idesc_bf16(TM, H), ks > 0);
        commit(bar);
      }
      ok = wait_phase(bar, phase);
      phase ^= 1u;
      if (!ok) break;
      hidden_epilogue(tmem, 256, b2, smem + OFF_H, a.h2, row, grow, MODE == MODE_TRAIN && valid);
      publish_smem();
      // layer 3
      if (tid == 0) {
#pragma unroll 1
        for (int ks = 0; ks < H / 16; ++ks) mma(tmem, dH + 16 * ks, dW3 + 16 * ks, idesc_bf16(TM, N3), ks > 0);
        commit(bar);
      }
      ok = wait_phase(bar, phase);
      phase ^= 1u;
      if (!ok) break;
      float lg[16];
      tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16), lg);  // both halves read (aligned ld)
#pragma unroll
      for (int j = 0; j < NO; ++j) lg[j] += b3[j];
      float v = 0.0f;
      const bool out_thread = valid && half == 0;
      if (MODE == MODE_TRAIN) {
        if (out_thread) {
          float4 *o = reinterpret_cast<float4 *>(a.logits + grow * NOP);
          o[0] = make_float4(lg[0], lg[1], lg[2], lg[3]);
          o[1] = make_float4(lg[4], 0.0f, 0.0f, 0.0f);
        }
      } else if (out_thread) {
        float m = lg[0];
#pragma unroll
        for (int j = 1; j < NO; ++j) m = fmaxf(m, lg[j]);
        float ex[NO], sum = 0.0f;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          ex[j] = __expf(lg[j] - m);
          sum += ex[j];
        }
        const float inv = 1.0f / sum;
        if (MODE == MODE_PREDICT) {
#pragma unroll
          for (int j = 0; j < NO; ++j) a.p[grow * NO + j] = ex[j] * inv;
        } else {
          v = ex[a.bin] * inv;
        }
      }
      if (MODE == MODE_SCREEN) {
        // rows in a fixed order: lanes by shuffle, then the four warps
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) score += (red[0] + red[1]) + (red[2] + red[3]);  // warps 4..7 hold zeros
      }
      // TMEM columns 0..15 are rewritten by the next tile's layer 1
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (MODE == MODE_SCREEN && tid == 0 && ok) a.scores[item] = score / (float)a.panel;
  }
  if (!ok && tid == 0) atomicExch(a.error, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int MODE>
cudaError_t launch_mode(const FwdArgs &a, int64_t items, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(forward_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(items < sms ? (items > 0 ? items : 1) : sms);
  forward_tc_kernel<MODE><<<grid, THREADS, SMEM_BYTES, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward(const FwdArgs &a, int mode, int64_t items, cudaStream_t st) {
  switch (mode) {
    case MODE_TRAIN: return launch_mode<MODE_TRAIN>(a, items, st);
    case MODE_PREDICT: return launch_mode<MODE_PREDICT>(a, items, st);
    default: return launch_mode<MODE_SCREEN>(a, items, st);
  }
}

}  // namespace vct
