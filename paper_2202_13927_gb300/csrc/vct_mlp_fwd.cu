// vct_mlp_fwd.cu -- the surrogate's fused forward pass on the 5th-generation
// tensor cores (tcgen05): one CTA per SM keeps all three weight matrices in
// shared memory and takes 128 rows (one tile) at a time through
//   layer 1: D1 = X W1^T       (TMEM columns   0..255, K = 32)
//   layer 2: D2 = H1 W2^T      (TMEM columns 256..511, K = 256)
//   layer 3: D3 = H2 W3^T      (TMEM columns 256..271, K = 256, N = 16 >= 5)
// with BF16 operands from shared memory and FP32 accumulators in TMEM.
// Warp-specialised pipeline: one thread of warp 16 issues every MMA and
// commits it to an mbarrier; warps 0-15 run the epilogues (warp w reads TMEM
// lanes 32 (w % 4) .. + 31, i.e. rows, and 16 of each 64-column chunk), add
// the bias, apply ReLU and write BF16 activations back to shared memory.  The
// epilogue hands each 64-column chunk to the MMA thread through an mbarrier,
// so layer 2's K steps on chunk c run while chunk c + 1 is being written, and
// layer 3 follows layer 2's epilogue the same way; the next tile's layer 1 is
// issued as soon as its input is staged, during this tile's layer-2 epilogue.
// (Measured alternative: one 64-column load per warp and chunk, so that a
// chunk needs only four warps -- 17 % slower.)
// Operands use the canonical K-major layout without swizzle: element (r, k)
// of an R x K operand sits at (r/8)(16 K) + (k/8) 128 + (r%8) 16 + (k%8) 2
// bytes, i.e. 8 x 16-byte core matrices, contiguous along K.
#include "vct_mlp.cuh"

namespace vct {
namespace {

constexpr int TM = 128;       // rows per tile = TMEM lanes
constexpr int EPI_WARPS = 16; // epilogue warps: lane quadrant w % 4, column group w / 4
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int THREADS = EPI_THREADS + 32;  // + the MMA warp
constexpr int CHUNK = 64;     // columns per epilogue -> MMA hand-off
constexpr int NCHUNK = 256 / CHUNK;
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
// mbarriers: D1, D2, D3 committed; H1 chunk c ready; H2 chunk c ready; X staged; final
// (and the four row-quadrant partial scores written)
constexpr int BAR_D1 = 0, BAR_D2 = 1, BAR_D3 = 2, BAR_H1 = 3, BAR_H2 = BAR_H1 + NCHUNK,
              BAR_X = BAR_H2 + NCHUNK, BAR_FIN = BAR_X + 1, BAR_RED = BAR_FIN + 1, NBAR = BAR_RED + 1;
constexpr int OFF_BAR = OFF_B3 + N3 * 4;
constexpr int OFF_TMEM = OFF_BAR + 8 * NBAR;
constexpr int OFF_RED = OFF_TMEM + 8;
constexpr int OFF_ABORT = OFF_RED + 4 * 4;
constexpr int SMEM_BYTES = OFF_ABORT + 16;
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

// Bounded wait of a whole warp for an mbarrier phase; every lane polls (and so
// acquires), the warp agrees on the outcome.  A wait that runs out, or finds
// the CTA's abort flag set, returns false and sets the flag for everyone.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t phase, volatile int *abort) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (!done && (it & 1023) == 1023 && *abort) break;
  }
  const bool ok = __all_sync(0xffffffffu, done != 0);
  if (!ok) *abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok;
}

// The same for the single MMA-issuing thread.
__device__ __forceinline__ bool thread_wait(uint32_t bar, uint32_t phase, volatile int *abort) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (!done && (it & 1023) == 1023 && *abort) break;
  }
  if (!done) *abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return done != 0;
}

// A warp hands its part of a buffer on: its shared-memory writes become
// visible to the tensor cores' proxy, its TMEM reads are complete, then lane 0
// arrives on the mbarrier (count = the number of epilogue warps).
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if ((threadIdx.x & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// One 16-column piece of a hidden layer: thread = row of the tile, columns
// col .. col + 15 of D at TMEM address taddr: bias, ReLU, BF16 into the
// canonical layout of H (and to global memory when training).
__device__ __forceinline__ void hidden_piece(uint32_t taddr, int col, const float *bias,
                                             unsigned char *hs, __nv_bfloat16 *glob, int row,
                                             int64_t grow, bool store_glob) {
  float v[16];
  tmem_ld16(taddr, v);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + bias[col + j], 0.0f);
  const uint4 u0 = pack8(v), u1 = pack8(v + 8);
  *reinterpret_cast<uint4 *>(hs + cm_off(row, col, H)) = u0;
  *reinterpret_cast<uint4 *>(hs + cm_off(row, col + 8, H)) = u1;
  if (store_glob) {
    *reinterpret_cast<uint4 *>(glob + grow * H + col) = u0;
    *reinterpret_cast<uint4 *>(glob + grow * H + col + 8) = u1;
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
  volatile int *abort = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  auto bar = [&](int j) { return s_base + OFF_BAR + 8u * (uint32_t)j; };
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_TMEM);
  unsigned char *xs = smem + OFF_X;

  // weights and biases once per CTA
  stage_matrix(smem + OFF_W1, a.W1, H, KF);
  stage_matrix(smem + OFF_W2, a.W2, H, H);
  stage_matrix(smem + OFF_W3, a.W3, N3, H);
  for (int e = tid; e < H; e += THREADS) {
    b1[e] = a.b1[e];
    b2[e] = a.b2[e];
  }
  if (tid < N3) b3[tid] = tid < NO ? a.b3[tid] : 0.0f;
  if (tid == 0) {
    *abort = 0;
    for (int j = 0; j < NBAR; ++j) {
      // chunks and the next input are written by all sixteen epilogue warps
      const uint32_t count = (j >= BAR_H1 && j <= BAR_X) ? (uint32_t)EPI_WARPS : j == BAR_RED ? 4u : 1u;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(j)), "r"(count));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + OFF_TMEM),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  publish_smem();
  const uint32_t tmem = *tmem_slot;

  const uint64_t dW1 = smem_desc(s_base + OFF_W1, KF), dW2 = smem_desc(s_base + OFF_W2, H),
                 dW3 = smem_desc(s_base + OFF_W3, H), dX = smem_desc(s_base + OFF_X, KF),
                 dH = smem_desc(s_base + OFF_H, H);
  const int64_t tiles = MODE == MODE_SCREEN ? (a.panel + TM - 1) / TM : 1;
  const int64_t n_items = MODE == MODE_SCREEN ? a.n_cand : (a.n_rows + TM - 1) / TM;
  const int64_t my_items = blockIdx.x < n_items ? (n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_units = my_items * tiles;   // this CTA's tiles, in order
  const bool panel_cached = MODE == MODE_SCREEN && tiles == 1;
  auto unit_item = [&](int64_t u) { return blockIdx.x + (u / tiles) * (int64_t)gridDim.x; };

  if (warp == EPI_WARPS) {
    // ------------------------------------------------------------ MMA thread
    if (lane == 0 && n_units > 0) {
      bool ok = thread_wait(bar(BAR_X), 0u, abort);
      if (ok) {
#pragma unroll
        for (int ks = 0; ks < KF / 16; ++ks) mma(tmem, dX + 16 * ks, dW1 + 16 * ks, idesc_bf16(TM, H), ks > 0);
        commit(bar(BAR_D1));
      }
      for (int64_t u = 0; ok && u < n_units; ++u) {
        const uint32_t par = (uint32_t)(u & 1);
        for (int c = 0; ok && c < NCHUNK; ++c) {
          ok = thread_wait(bar(BAR_H1 + c), par, abort);
          if (!ok) break;
#pragma unroll
          for (int j = 0; j < CHUNK / 16; ++j) {
            const int ks = c * (CHUNK / 16) + j;
            mma(tmem + 256, dH + 16 * ks, dW2 + 16 * ks, idesc_bf16(TM, H), ks > 0);
          }
        }
        if (!ok) break;
        commit(bar(BAR_D2));
        if (u + 1 < n_units) {
          ok = thread_wait(bar(BAR_X), (uint32_t)((u + 1) & 1), abort);
          if (!ok) break;
#pragma unroll
          for (int ks = 0; ks < KF / 16; ++ks) mma(tmem, dX + 16 * ks, dW1 + 16 * ks, idesc_bf16(TM, H), ks > 0);
          commit(bar(BAR_D1));
        }
        for (int c = 0; ok && c < NCHUNK; ++c) {
          ok = thread_wait(bar(BAR_H2 + c), par, abort);
          if (!ok) break;
#pragma unroll
          for (int j = 0; j < CHUNK / 16; ++j) {
            const int ks = c * (CHUNK / 16) + j;
            mma(tmem + 256, dH + 16 * ks, dW3 + 16 * ks, idesc_bf16(TM, N3), ks > 0);
          }
        }
        if (!ok) break;
        commit(bar(BAR_D3));
      }
      // every MMA this thread issued has finished before TMEM is released
      commit(bar(BAR_FIN));
      thread_wait(bar(BAR_FIN), 0u, abort);
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int qd = warp & 3, grp = warp >> 2;
    const int row = 32 * qd + lane;               // TMEM lane = row of the tile
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    // staging: thread -> (row, 8-feature chunk) of X
    const int srow = tid & (TM - 1), sq = tid >> 7;
    float pf[8];                                  // this thread's 8 panel features (cached panel)
    float score = 0.0f;                           // warp 0 lane 0: the candidate's running sum

    auto stage_x = [&](int64_t u) {
      const int64_t item = unit_item(u), tile = u % tiles;
      if (MODE != MODE_SCREEN) {
        const int64_t grow = item * TM + srow;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (grow < a.n_rows) v = reinterpret_cast<const uint4 *>(a.x + grow * KF)[sq];
        *reinterpret_cast<uint4 *>(xs + cm_off(srow, 8 * sq, KF)) = v;
        return;
      }
      const int64_t prow = tile * TM + srow;
      const bool valid = prow < a.panel;
      if (!panel_cached || u == 0) {
        if (valid) {
          const float4 *src = reinterpret_cast<const float4 *>(a.panel_x + prow * KF + 8 * sq);
          const float4 v0 = src[0], v1 = src[1];
          pf[0] = v0.x; pf[1] = v0.y; pf[2] = v0.z; pf[3] = v0.w;
          pf[4] = v1.x; pf[5] = v1.y; pf[6] = v1.z; pf[7] = v1.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) pf[j] = 0.0f;
        }
        if (sq == 0 || sq == 3) *reinterpret_cast<uint4 *>(xs + cm_off(srow, 8 * sq, KF)) = pack8(pf);
      }
      // the candidate's standardized log gains are features 15, 16, 17:
      // slot 7 of chunk 1 and slots 0, 1 of chunk 2
      if (sq == 1 || sq == 2) {
        float ch[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) ch[j] = pf[j];
        if (valid) {
          if (sq == 1) {
            ch[7] = a.cand_lg[item * 3];
          } else {
            ch[0] = a.cand_lg[item * 3 + 1];
            ch[1] = a.cand_lg[item * 3 + 2];
          }
        }
        *reinterpret_cast<uint4 *>(xs + cm_off(srow, 8 * sq, KF)) = pack8(ch);
      }
    };

    bool ok = true;
    if (n_units > 0) {
      stage_x(0);
      warp_arrive(bar(BAR_X));
    }
    for (int64_t u = 0; ok && u < n_units; ++u) {
      const uint32_t par = (uint32_t)(u & 1);
      const int64_t item = unit_item(u), tile = u % tiles;
      const int64_t row0 = MODE == MODE_SCREEN ? tile * TM : item * TM;
      const int64_t limit = MODE == MODE_SCREEN ? (int64_t)a.panel : a.n_rows;
      const int64_t grow = row0 + row;
      const bool valid = grow < limit;
      const bool train = MODE == MODE_TRAIN && valid;
      // layer-1 epilogue, chunk by chunk
      ok = warp_wait(bar(BAR_D1), par, abort);
      if (!ok) break;
      for (int c = 0; c < NCHUNK; ++c) {
        const int col = c * CHUNK + 16 * grp;
        hidden_piece(lane_base + (uint32_t)col, col, b1, smem + OFF_H, a.h1, row, grow, train);
        warp_arrive(bar(BAR_H1 + c));
      }
      // the next tile's input (layer 1 of this tile has finished reading X)
      if (u + 1 < n_units) {
        stage_x(u + 1);
        warp_arrive(bar(BAR_X));
      }
      // layer-2 epilogue (H2 replaces H1 in shared memory: layer 2 has finished)
      ok = warp_wait(bar(BAR_D2), par, abort);
      if (!ok) break;
      for (int c = 0; c < NCHUNK; ++c) {
        const int col = c * CHUNK + 16 * grp;
        hidden_piece(lane_base + 256u + (uint32_t)col, col, b2, smem + OFF_H, a.h2, row, grow, train);
        warp_arrive(bar(BAR_H2 + c));
      }
      // layer 3 (all warps wait: the next tile's H1 overwrites what layer 3 reads)
      ok = warp_wait(bar(BAR_D3), par, abort);
      if (!ok) break;
      if (warp < 4) {
        float lg[16];
        tmem_ld16(lane_base + 256u, lg);
        asm volatile("tcgen05.fence::before_thread_sync;");
#pragma unroll
        for (int j = 0; j < NO; ++j) lg[j] += b3[j];
        float v = 0.0f;
        if (MODE == MODE_TRAIN) {
          if (valid) {
            float4 *o = reinterpret_cast<float4 *>(a.logits + grow * NOP);
            o[0] = make_float4(lg[0], lg[1], lg[2], lg[3]);
            o[1] = make_float4(lg[4], 0.0f, 0.0f, 0.0f);
          }
        } else if (valid) {
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
          if (lane == 0) {
            red[warp] = v;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(BAR_RED)) : "memory");
          }
          if (warp == 0) {
            ok = warp_wait(bar(BAR_RED), par, abort);
            if (ok && lane == 0) {
              score += (red[0] + red[1]) + (red[2] + red[3]);
              if (tile == tiles - 1) {
                a.scores[item] = score / (float)a.panel;
                score = 0.0f;
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort && tid == 0) atomicExch(a.error, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
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
