// vct_mlp_gemm.cu -- the surrogate's backward GEMMs on the tcgen05 tensor cores.
//
// C[M][N] = A[M][K] B[K][N] with BF16 operands given by strides (each operand
// stored contiguous along K or along its other dimension, plainly or in chunks
// of 8 elements a chunk stride apart) and FP32
// accumulation in TMEM.  One CTA of 256 threads computes a 128 x NT tile
// (NT <= 256, a multiple of 16) over one K range (split-K).  Its threads stage
// 64-deep K slices of both operands into shared memory in the canonical K-major
// layout -- a K-contiguous source as asynchronous 16-byte copies, the other as 8 x 8 blocks
// transposed in registers -- two slices in flight, while thread 0 issues the
// MMAs of the slice before.  Epilogue: the accumulators pass through a shared-
// memory tile, 32 columns at a time, so that whole rows are stored together:
// FP32 split-K partials, or the BF16 product masked by the ReLU pattern of the
// layer's activations.  A weight gradient dW = dZ^T X can also give its bias
// gradient db = dZ^T 1: the CTAs of the first column tile add up the rows of
// the A slices they stage (in registers, a fixed order) and write one partial
// per split beside the weight partials.
#include "vct_mlp.cuh"
#include "vct_tc.cuh"

namespace vct {
namespace {

constexpr int GM = 128;     // tile rows = TMEM lanes
constexpr int GKS = 64;     // K slice staged at a time
constexpr int GNMAX = 256;  // widest tile
constexpr int GTHR = 256;  // 8 warps: two per TMEM lane quadrant
constexpr int A_BYTES = GM * GKS * 2;
constexpr int B_BYTES = GNMAX * GKS * 2;
constexpr int OFF_A0 = 0, OFF_A1 = A_BYTES;
constexpr int OFF_B0 = 2 * A_BYTES, OFF_B1 = 2 * A_BYTES + B_BYTES;
// mbarriers: slice buffer 0 and 1 free again (their MMAs done), every MMA done
constexpr int OFF_BAR = 2 * A_BYTES + 2 * B_BYTES;
constexpr int BAR_DONE = 2;
constexpr int OFF_TMEM = OFF_BAR + 8 * 3;
constexpr int OFF_ABORT = OFF_TMEM + 8;
constexpr int SMEM_BYTES = OFF_ABORT + 8;
constexpr uint32_t kTmemCols = 256;
static_assert(2 * SMEM_BYTES <= 232448, "two CTAs per SM");
static_assert(GM * 65 * 4 <= 2 * A_BYTES + 2 * B_BYTES, "epilogue tile in the operand buffers");

// 8 x 8 BF16 transpose in registers: in[i] is row i (8 values), out[j] column j.
__device__ __forceinline__ void transpose8(const uint4 in[8], uint4 out[8]) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(in);  // w[4 i + c]: row i, columns 2c, 2c+1
  uint32_t *o = reinterpret_cast<uint32_t *>(out);             // o[4 j + c]: column j, rows 2c, 2c+1
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t a = w[4 * (2 * i) + c], b = w[4 * (2 * i + 1) + c];
      o[4 * (2 * c) + i] = __byte_perm(a, b, 0x5410);      // low halves: column 2c
      o[4 * (2 * c + 1) + i] = __byte_perm(a, b, 0x7632);  // high halves: column 2c + 1
    }
}

// v[j] <- v[(j + sh) % 8] for a per-thread shift sh in 0 .. 7: three
// conditional rotations by 1, 2 and 4 with constant register indices.  A
// transposed 8 x 8 block is one 128-byte core matrix, so the threads of a warp
// storing its row j at once all hit the same four banks; rotated by the lane,
// the eight lanes of each group store eight different rows (no conflicts).
__device__ __forceinline__ void rotate8(uint4 v[8], int sh) {
#pragma unroll
  for (int b = 1; b < 8; b <<= 1) {
    const bool on = (sh & b) != 0;
    uint4 t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = v[(j + b) & 7];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = on ? t[j] : v[j];
  }
}

// Stage the K slice [k0, k0 + GKS) of X[r][k] = src[r sr + k sk] as rows
// 0 .. rows-1 of a canonical K-major tile (tile row t is X's row r0 + t); rows
// >= R and k >= K read as zero.  The contiguous dimension is stored in chunks
// of 8 elements cs apart (cs = 8: plainly): sk == 1: X[r][k] = src[r sr + (k /
// 8) cs + k % 8], 16-byte chunks along k (K a multiple of 8); else sr == 1:
// X[r][k] = src[k sk + (r / 8) cs + r % 8], 8 x 8 blocks read along r, one k
// row at a time, and transposed.  (sr or sk, cs, r0 and the source address
// are multiples of 8 elements, checked by the host.)
__device__ void stage(unsigned char *dst, const __nv_bfloat16 *src, int64_t sr, int64_t sk, int64_t cs, int r0,
                      int R, int64_t k0, int64_t K, int rows) {
  if (sk == 1) {
    // asynchronous 16-byte copies, every one of the thread's in flight at once
    // (zero-filled outside the operand); the caller waits with cp.async.wait_all.
    // Copy c fills the c-th 16 bytes of the tile (row 8 (c / 64) + c % 8, k
    // 8 ((c / 8) % 8) ..): a warp writes 512 contiguous bytes of shared memory.
    const int chunks = rows * (GKS / 8);
    const uint32_t d0 = (uint32_t)__cvta_generic_to_shared(dst);
    for (int c = threadIdx.x; c < chunks; c += GTHR) {
      const int q = c >> 3, r = (q / (GKS / 8)) * 8 + (c & 7), kk = (q % (GKS / 8)) * 8;
      const int64_t gr = (int64_t)r0 + r, gk = k0 + kk;
      const bool in = gr < R && gk < K;
      const __nv_bfloat16 *g = in ? src + gr * sr + (gk >> 3) * cs : src;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d0 + 16u * (uint32_t)c), "l"(g),
                   "r"(in ? 16u : 0u)
                   : "memory");
    }
  } else {
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    const int blocks = (rows / 8) * (GKS / 8);
    for (int b = threadIdx.x; b < blocks; b += GTHR) {
      const int rb = (b / (GKS / 8)) * 8, kb = (b % (GKS / 8)) * 8;
      const int64_t gr = (int64_t)r0 + rb;
      const __nv_bfloat16 *col = src + (gr >> 3) * cs;
      uint4 in[8], out[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int64_t gk = k0 + kb + i;
        in[i] = (gr < R && gk < K) ? *reinterpret_cast<const uint4 *>(col + gk * sk) : zero;
      }
      transpose8(in, out);
      const int sh = b & 7;
      rotate8(out, sh);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int row = (j + sh) & 7;
        *reinterpret_cast<uint4 *>(dst + cm_off(rb + row, kb, GKS)) = gr + row < R ? out[j] : zero;
      }
    }
  }
}

// The transposed form of stage() for an A operand stored along M (sr == 1),
// adding up each staged row over the slice: thread t (< 128) stages the 8 x 8
// block of rows 8 (t / 8) .., k 8 (t % 8) .. and returns in sum[j] its row j's
// sum over those 8 k (in k order); the 8 threads of one block row are
// consecutive lanes of a warp.
__device__ __forceinline__ void stage_rows_summed(unsigned char *dst, const __nv_bfloat16 *src, int64_t sk,
                                                  int64_t cs, int r0, int R, int64_t k0, int64_t K, float sum[8]) {
  static_assert((GM / 8) * (GKS / 8) == 128, "one block per thread of warps 0-3");
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int j = 0; j < 8; ++j) sum[j] = 0.0f;
  const int b = threadIdx.x;
  if (b >= (GM / 8) * (GKS / 8)) return;
  const int rb = (b / (GKS / 8)) * 8, kb = (b % (GKS / 8)) * 8;
  const int64_t gr = (int64_t)r0 + rb;
  const __nv_bfloat16 *col = src + (gr >> 3) * cs;
  uint4 in[8], out[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gk = k0 + kb + i;
    in[i] = (gr < R && gk < K) ? *reinterpret_cast<const uint4 *>(col + gk * sk) : zero;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const uint32_t *w = reinterpret_cast<const uint32_t *>(&in[i]);  // rows 2c (low half), 2c + 1 (high)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sum[2 * c] += __uint_as_float(w[c] << 16);
      sum[2 * c + 1] += __uint_as_float(w[c] & 0xFFFF0000u);
    }
  }
  transpose8(in, out);
  const int sh = b & 7;
  rotate8(out, sh);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int row = (j + sh) & 7;
    *reinterpret_cast<uint4 *>(dst + cm_off(rb + row, kb, GKS)) = gr + row < R ? out[j] : zero;
  }
}

// (two CTAs per SM, as the shared memory allows: at most 128 registers a thread)
__global__ void __launch_bounds__(GTHR, 2) tc_gemm_kernel(const __grid_constant__ TcGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  auto bar = [&](int j) { return s_base + OFF_BAR + 8u * (uint32_t)j; };
  volatile int *abort = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * g.NT;
  const int64_t kb = (int64_t)blockIdx.z * g.kc;
  const int64_t ke = kb + g.kc < g.K ? kb + g.kc : g.K;
  const int n_slices = (int)((ke - kb + GKS - 1) / GKS);  // >= 1 (host)

  if (tid == 0) {
    *abort = 0;
    for (int j = 0; j < 3; ++j) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(j)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + OFF_TMEM),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  publish_smem();
  const uint32_t tmem = *reinterpret_cast<const uint32_t *>(smem + OFF_TMEM);
  const uint32_t idesc = idesc_bf16(GM, g.NT);
  // warp 0 issues the MMAs, converged, through one elected lane
  const uint32_t issue = warp == 0 ? elect_one() : 0u;
  // bias sums: the first column tile's CTAs, rows 8 (tid / 8) .. of the tile
  // (warps 0-3; after the butterfly every lane of a block row holds the sums)
  const bool bias = g.mode == 0 && g.bias_partial != nullptr && blockIdx.x == 0;
  float bsum[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) bsum[j] = 0.0f;

  bool ok = true;
  for (int s = 0; s < n_slices && ok; ++s) {
    const int buf = s & 1;
    // the buffer's previous slice (s - 2) has been consumed by its MMAs
    if (s >= 2) ok = warp_wait_spin(bar(buf), (uint32_t)(((s - 2) >> 1) & 1), abort);
    // every warp takes the same branch (the block barriers below need all of them)
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) break;
    const int off_a = buf ? OFF_A1 : OFF_A0, off_b = buf ? OFF_B1 : OFF_B0;
    const int64_t k0 = kb + (int64_t)s * GKS;
    if (bias) {  // CTA-uniform
      float part[8];
      stage_rows_summed(smem + off_a, g.A, g.sak, g.acs, m0, g.M, k0, ke, part);
      if (warp < 4) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float v = part[j];
          v += __shfl_xor_sync(0xFFFFFFFFu, v, 1);
          v += __shfl_xor_sync(0xFFFFFFFFu, v, 2);
          v += __shfl_xor_sync(0xFFFFFFFFu, v, 4);
          bsum[j] += v;
        }
      }
    } else {
      stage(smem + off_a, g.A, g.sam, g.sak, g.acs, m0, g.M, k0, ke, GM);
    }
    stage(smem + off_b, g.B, g.sbn, g.sbk, g.bcs, n0, g.N, k0, ke, g.NT);
    asm volatile("cp.async.wait_all;" ::: "memory");
    publish_smem();
    if (warp == 0) {
      const uint64_t da = smem_desc(s_base + off_a, GKS), db = smem_desc(s_base + off_b, GKS);
#pragma unroll
      for (int ks = 0; ks < GKS / 16; ++ks)
        mma(tmem, da + 16 * ks, db + 16 * ks, idesc, (s > 0 || ks > 0) ? 1u : 0u, issue);
      commit(bar(buf), issue);
    }
  }
  // every MMA issued has finished before TMEM is read or released
  if (warp == 0) commit(bar(BAR_DONE), issue);
  ok = warp_wait_spin(bar(BAR_DONE), 0u, abort) && ok;
  ok = __syncthreads_and(ok ? 1 : 0) != 0;

  if (ok) {
    // 64 columns at a time: the two warps of each TMEM lane quadrant move 32
    // columns each of their 32 rows into a padded shared-memory tile (the
    // operand buffers are free now), then every warp writes whole rows of it
    // (lane = column: coalesced stores)
    float *tile = reinterpret_cast<float *>(smem + OFF_A0);  // [GM][65]
    const int qd = warp & 3, half = warp >> 2;
    const uint32_t taddr = tmem + ((uint32_t)(32 * qd) << 16);
    for (int c0 = 0; c0 < g.NT; c0 += 64) {
      const int cc = c0 + 32 * half;
      if (cc < g.NT) {  // warp-uniform
        float v[32];
        tmem_ld32(taddr + (uint32_t)cc, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[(32 * qd + lane) * 65 + 32 * half + j] = v[j];
      }
      __syncthreads();
      if (g.mode == 0) {
#pragma unroll 4
        for (int r = warp; r < GM; r += GTHR / 32) {
          const int row = m0 + r;
          if (row >= g.M) continue;
          float *dst = g.partial + (int64_t)blockIdx.z * g.pstride + (int64_t)row * g.N;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = c0 + 32 * h + lane, n = n0 + c;
            if (c < g.NT && n < g.N) dst[n] = tile[r * 65 + 32 * h + lane];
          }
        }
      } else {
        // the warp's mask values first (independent loads), then the stores
        constexpr int RW = GM / (GTHR / 32);  // rows per warp
        bool on[RW][2];
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          const int row = m0 + warp + (GTHR / 32) * q;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = c0 + 32 * h + lane, n = n0 + c;
            on[q][h] = row < g.M && c < g.NT && n < g.N &&
                       __bfloat162float(g.mask[(int64_t)row * g.mrs + (int64_t)(n >> 3) * g.mcs + (n & 7)]) > 0.0f;
          }
        }
#pragma unroll
        for (int q = 0; q < RW; ++q) {
          const int r = warp + (GTHR / 32) * q, row = m0 + r;
          if (row >= g.M) continue;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = c0 + 32 * h + lane, n = n0 + c;
            if (c < g.NT && n < g.N)
              g.out[(int64_t)row * g.N + n] = __float2bfloat16_rn(on[q][h] ? tile[r * 65 + 32 * h + lane] : 0.0f);
          }
        }
      }
      __syncthreads();
    }
  }
  if (bias && ok && warp < 4 && (lane & 7) == 0) {
    float *dst = g.bias_partial + (int64_t)blockIdx.z * g.pstride;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int row = m0 + (tid >> 3) * 8 + j;
      if (row < g.M) dst[row] = bsum[j];
    }
  }
  __syncthreads();
  if (*abort && tid == 0) atomicOr(g.error, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

cudaError_t launch_tc_gemm(const TcGemmArgs &g, int tiles_n, int tiles_m, int splits, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<<<dim3(tiles_n, tiles_m, splits), GTHR, SMEM_BYTES, st>>>(g);
  return cudaGetLastError();
}

}  // namespace vct
