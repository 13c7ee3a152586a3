// vct_mlp_fwd.cu -- the surrogate's fused forward pass on the 5th-generation
// tensor cores (tcgen05).  One CTA per SM keeps the three weight matrices in
// shared memory (BF16, canonical K-major layout, copied in whole from images in
// that layout by the bulk-copy engine) and takes 128 rows (one tile = the 128
// TMEM lanes) at a time; the activations never leave tensor memory:
//   layer 1, two halves of 128 units: D1 = X W1[half]^T -> TMEM cols 0..127 (FP32);
//            the bias enters through input features 18 and 19 (both 1) and
//            W1's columns 18 and 19 (the BF16 high and low parts of b1)
//            epilogue: ReLU, BF16 pairs                   -> H1 in cols 384..511
//   layer 2: D2 = b2 + H1 W2^T, A operand read from TMEM   -> cols 128..383
//            epilogue, 64 units per warp, in place         -> H2 in the first 32
//                                                             columns of each 64
//   layer 3: D3 = H2 W3^T (N = 16 >= 5 outputs) as four independent partial
//            sums over 64 units each (no chain of dependent MMAs), in the
//            second half of H1 (cols 448..511, free while layer 3 runs), so
//            that the next tile's layer 2 waits for layer 3 alone, not for
//            the logits to be read
// training:  the softmax cross-entropy of each row from its logits (loss and
//            dZ3), then dZ2 = (dZ3 W3) where Z2 > 0 from an FP32 copy of W3
//            in shared memory (5 products per unit: too thin for the tensor
//            pipe), with the ReLU pattern kept as bits from the layer-2
//            epilogue; H1, H2 and dZ2 go to global memory chunk-major
//            (coalesced stores) for the backward GEMMs
// A BF16 activation pair (units 2j, 2j + 1) sits in one 32-bit TMEM column
// (even unit in the low half), so K step s of 16 units is 8 columns.
// Warp-specialised: warp 16 issues every MMA and commits it to an mbarrier
// (converged, through one elected lane: vct_tc.cuh); warps 0-15 run the
// epilogues (warp w owns TMEM lanes 32 (w % 4) .. + 31, i.e. rows, and column
// group w / 4).  Hand-offs go through mbarriers, so layer 2 starts on the
// first half of H1 while the second half of layer 1 is still in its epilogue,
// the next tile's first layer-1 half runs during this tile's layer-2
// epilogue, and its epilogue (H1 and H2 live in different columns) while
// layer 3 is on the tensor pipe.  Each epilogue step is a few TMEM loads and
// stores per warp (their latency, not the arithmetic, sets the pace).  Shared
// memory carries the MMAs' weight and input operands and, when training, the
// tile's dZ3 and W3 in FP32.
// Operands in shared memory use the canonical K-major layout (vct_tc.cuh).
#include "vct_mlp.cuh"
#include "vct_tc.cuh"

namespace vct {
namespace {

constexpr int TM = 128;       // rows per tile = TMEM lanes
constexpr int EPI_WARPS = 16; // epilogue warps: lane quadrant w % 4, column group w / 4
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int THREADS = EPI_THREADS + 32;  // + the MMA warp
constexpr int H = kSurrH, KF = kSurrKF, NO = kSurrNO;
constexpr int N3 = 16;        // layer-3 MMA width
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t COL_D1 = 0, COL_D2 = 128, COL_H = 384;
// layer 2's epilogue writes H2 in place: the BF16 pairs of units 64 g .. 64 g + 63
// into the first 32 of D2's columns 64 g .. 64 g + 63; layer 3's partial sum p
// (over those units) goes to 16 columns of H1's second half
__host__ __device__ constexpr uint32_t col_h2(int ks) { return COL_D2 + 64 * (ks / 4) + 8 * (ks % 4); }
__host__ __device__ constexpr uint32_t col_d3(int p) { return COL_H + 64 + 16 * p; }

// shared memory map (bytes)
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + H * KF * 2;
constexpr int OFF_W3 = OFF_W2 + H * H * 2;
constexpr int OFF_X = OFF_W3 + N3 * H * 2;
// layer 2's bias enters through one extra K step: A = ONES (128 x 16, columns
// 0 and 1 = 1), B = [hi(b), lo(b), 0 ...] per unit (256 x 16), so that D starts
// from hi(b) + lo(b) (two BF16 parts, about 16 significant bits).  Layer 1's
// input has room for the same in its padding: features KB1 and KB1 + 1 are 1
// and W1's columns KB1, KB1 + 1 hold hi(b1), lo(b1).
constexpr int BK = 16;
constexpr int KB1 = 18;
static_assert(KB1 % 2 == 0 && KB1 + 2 <= KF && KB1 / 8 == 2, "layer-1 bias features: word 1 of chunk 2");
constexpr int OFF_ONES = OFF_X + TM * KF * 2;
constexpr int OFF_BB2 = OFF_ONES + TM * BK * 2;
constexpr int OFF_B3 = OFF_BB2 + H * BK * 2;
// mbarriers: layer-1 halves, layer 2 and layer 3 committed; H1 halves written;
// H2 written; X staged; every MMA finished; the four partial scores written;
// the logits read; the rows' dZ3 written to shared memory (training); the
// weight images copied in
constexpr int BAR_D1A = 0, BAR_D1B = 1, BAR_D2 = 2, BAR_D3 = 3, BAR_H1A = 4, BAR_H1B = 5,
              BAR_H2 = 6, BAR_X = 7, BAR_FIN = 8, BAR_RED = 9, BAR_D3C = 10, BAR_DZ = 11, BAR_W = 12,
              NBAR = 13;
constexpr int OFF_BAR = OFF_B3 + N3 * 4;
constexpr int OFF_TMEM = OFF_BAR + 8 * NBAR;
constexpr int OFF_RED = OFF_TMEM + 8;           // screening: one value per row of the tile
constexpr int OFF_ABORT = OFF_RED + TM * 4;
constexpr int OFF_DZ = OFF_ABORT + 16;           // training: dZ3 of the tile, [5][TM] FP32
constexpr int OFF_W3F = (OFF_DZ + NO * TM * 4 + 15) / 16 * 16;   // training: W3 rows 0-4 in FP32, [5][H]
constexpr int SMEM_BYTES = OFF_W3F + NO * H * 4;
static_assert(SMEM_BYTES <= 232448, "shared memory");

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

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory with the bulk-copy engine, completing on mbarrier `bar`
// (whose expected transaction count the caller has raised by `bytes`).  A
// weight image in the canonical layout arrives in one copy: staged as 16-byte
// asynchronous copies by the threads, 155 KB took a third of a one-tile
// training launch (about 12 bytes per cycle, bounded by the copies an SM keeps
// in flight).
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// ReLU and BF16 rounding of two activations in one conversion; the even unit
// goes to the low half
__device__ __forceinline__ uint32_t relu_bf16_pair(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Store 8 units (one 16-byte chunk) of row grow, starting at unit, into a
// chunk-major activation array (unit u of row r at (u / 8) cs + 8 r + u % 8):
// the lanes of a warp hold consecutive rows, so one store instruction writes
// 512 contiguous bytes (row-major rows 512 bytes apart took one line each).
__device__ __forceinline__ void store_chunk(__nv_bfloat16 *glob, int64_t cs, int64_t grow, int unit, uint4 v) {
  *reinterpret_cast<uint4 *>(glob + (int64_t)(unit >> 3) * cs + grow * 8) = v;
}

// Layer 1's epilogue for 32 consecutive hidden units of this thread's row from
// FP32 TMEM at ld_addr (the bias is already in the accumulator): ReLU, BF16
// pairs into TMEM at st_addr (and to global memory when training); one TMEM
// load and one store.
__device__ __forceinline__ void hidden32(uint32_t ld_addr, uint32_t st_addr, int unit, __nv_bfloat16 *glob,
                                         int64_t cs, int64_t grow, bool store_glob) {
  float v[32];
  tmem_ld32(ld_addr, v);
  uint32_t p[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) p[j] = relu_bf16_pair(v[2 * j], v[2 * j + 1]);
  tmem_st16(st_addr, p);
  if (store_glob) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      store_chunk(glob, cs, grow, unit + 8 * q, make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]));
  }
}

// bit i set where the FP32 value with bits v[i] is > 0 (not -0, not NaN)
__device__ __forceinline__ uint32_t positive_bits(const uint32_t v[32]) {
  uint32_t m = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) m |= (v[i] - 1u < 0x7F800000u ? 1u : 0u) << i;
  return m;
}

// Layer 2's epilogue for 64 units of this thread's row, in place (the bias is
// already in the accumulators): ReLU and BF16 pairs of the first 32 units go
// to the group's first 16 columns while the second 32 units are loaded, then
// those to the next 16 (48 live registers instead of 64; the columns written
// are ones this warp has already read).  When training, the ReLU pattern
// [Z2 > 0] of the 64 units comes back as bits (unit 64 g + i: bit i % 32 of
// word i / 32).
__device__ __forceinline__ uint2 hidden64_in_place(uint32_t addr, int unit, __nv_bfloat16 *glob, int64_t cs,
                                                   int64_t grow, bool store_glob) {
  uint32_t v[32], pa[16], pb[16];
  uint2 on = make_uint2(0u, 0u);
  tmem_ld32_nowait(addr, v);
  tmem_wait_ld32(v);
#pragma unroll
  for (int j = 0; j < 16; ++j) pa[j] = relu_bf16_pair(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
  if (store_glob) on.x = positive_bits(v);
  tmem_ld32_nowait(addr + 32, v);
  tmem_st16_nowait(addr, pa);
  tmem_wait_ld32(v);
#pragma unroll
  for (int j = 0; j < 16; ++j) pb[j] = relu_bf16_pair(__uint_as_float(v[2 * j]), __uint_as_float(v[2 * j + 1]));
  if (store_glob) on.y = positive_bits(v);
  tmem_st16_nowait(addr + 16, pb);
  tmem_wait_st();
  if (store_glob) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      store_chunk(glob, cs, grow, unit + 8 * q, make_uint4(pa[4 * q], pa[4 * q + 1], pa[4 * q + 2], pa[4 * q + 3]));
#pragma unroll
    for (int q = 0; q < 4; ++q)
      store_chunk(glob, cs, grow, unit + 32 + 8 * q,
                  make_uint4(pb[4 * q], pb[4 * q + 1], pb[4 * q + 2], pb[4 * q + 3]));
  }
  return on;
}

// Two FP32 products, or two fmas, in one instruction (f32x2); each lane rounds
// as the scalar operation does.
__device__ __forceinline__ unsigned long long pack_f2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 unpack_f2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 mul_x2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack_f2(a)), "l"(pack_f2(b)));
  return unpack_f2(d);
}
__device__ __forceinline__ float2 fma_x2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pack_f2(a)), "l"(pack_f2(b)), "l"(pack_f2(c)));
  return unpack_f2(d);
}

// dZ2 of one row for the 64 units from `unit` on: (dZ3 W3)[u] where Z2 > 0,
// else 0.  d holds the row's dZ3 (BF16 values, as the weight gradient reads
// them); W3's rows 0-4, in FP32 in shared memory, are read 8 units at a time,
// the same address in every lane of the warp (broadcasts).  The products are
// exact in FP32 and summed in output order, two units per instruction.
__device__ __forceinline__ void dz2_row(const float *w3f, const float d[NO], uint2 on, __nv_bfloat16 *glob,
                                        int64_t cs, int64_t grow, int unit) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float2 acc2[4];
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const float4 *w = reinterpret_cast<const float4 *>(w3f + j * H + unit + 8 * c);
      const float4 w0 = w[0], w1 = w[1];
      const float2 wv[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                            make_float2(w1.z, w1.w)};
      const float2 dj = make_float2(d[j], d[j]);
#pragma unroll
      for (int i = 0; i < 4; ++i) acc2[i] = j == 0 ? mul_x2(dj, wv[i]) : fma_x2(dj, wv[i], acc2[i]);
    }
    float acc[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[2 * i] = acc2[i].x;
      acc[2 * i + 1] = acc2[i].y;
    }
    const uint32_t bits = (c < 4 ? on.x : on.y) >> (8 * (c & 3));
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = (bits >> i) & 1u ? acc[i] : 0.0f;
    store_chunk(glob, cs, grow, unit + 8 * c, pack8(acc));
  }
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) forward_tc_kernel(FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float *b3 = reinterpret_cast<float *>(smem + OFF_B3);
  float *red = reinterpret_cast<float *>(smem + OFF_RED);
  volatile int *abort = reinterpret_cast<volatile int *>(smem + OFF_ABORT);
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem);
  auto bar = [&](int j) { return s_base + OFF_BAR + 8u * (uint32_t)j; };
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_TMEM);
  unsigned char *xs = smem + OFF_X;

  // The weights once per CTA: their canonical images copied whole by the
  // bulk-copy engine (issued below, after the mbarriers are initialised), in
  // flight while the rest of the set-up runs (biases, constant operands, TMEM,
  // the first tile's input).
  static_assert(H <= THREADS && TM <= THREADS, "one bias unit, one ONES row per thread");
  // bias operands: (hi, lo) of unit u's bias in W1's columns KB1, KB1 + 1 (once
  // W1 has arrived) and in row u of the layer-2 bias operand; ONES row r = (1, 1, 0, ...)
  auto hi_lo = [](float b) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(b);
    const __nv_bfloat16 lo = __float2bfloat16_rn(b - __bfloat162float(hi));
    __nv_bfloat162 p0 = __halves2bfloat162(hi, lo);
    return *reinterpret_cast<uint32_t *>(&p0);
  };
  const float bias1 = tid < H ? a.b1[tid] : 0.0f;
  if (tid < H) {
    *reinterpret_cast<uint4 *>(smem + OFF_BB2 + cm_off(tid, 0, BK)) = make_uint4(hi_lo(a.b2[tid]), 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(smem + OFF_BB2 + cm_off(tid, 8, BK)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid < TM) {
    __nv_bfloat162 one2 = __floats2bfloat162_rn(1.0f, 1.0f);
    *reinterpret_cast<uint4 *>(smem + OFF_ONES + cm_off(tid, 0, BK)) =
        make_uint4(*reinterpret_cast<uint32_t *>(&one2), 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(smem + OFF_ONES + cm_off(tid, 8, BK)) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid < N3) b3[tid] = tid < NO ? a.b3[tid] : 0.0f;
  if (MODE == MODE_TRAIN) {
    float *w3f = reinterpret_cast<float *>(smem + OFF_W3F);
    for (int e = tid; e < NO * H; e += THREADS) w3f[e] = __bfloat162float(a.W3[canon_index(e / H, e % H, H)]);
  }
  if (tid == 0) {
    *abort = 0;
    for (int j = 0; j < NBAR; ++j) {
      // hand-offs from the epilogue come from all sixteen epilogue warps
      const uint32_t count = (j >= BAR_H1A && j <= BAR_X) ? (uint32_t)EPI_WARPS
                             : (j == BAR_RED || j == BAR_D3C || j == BAR_DZ) ? 4u : 1u;
      // (BAR_RED: the four row-quadrant warps have written their rows' values;
      //  BAR_D3C: they have read their rows' logits, which the next tile's second
      //  H1 half overwrites; BAR_DZ: they have written their rows' dZ3)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar(j)), "r"(count));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    constexpr uint32_t w1_bytes = H * KF * 2, w2_bytes = H * H * 2, w3_bytes = N3 * H * 2;
    static_assert(OFF_W2 == OFF_W1 + (int)w1_bytes && OFF_W3 == OFF_W2 + (int)w2_bytes && OFF_W1 % 16 == 0,
                  "weight images back to back in shared memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(BAR_W)),
                 "r"(w1_bytes + w2_bytes + w3_bytes)
                 : "memory");
    bulk_copy(s_base + OFF_W1, a.W1, w1_bytes, bar(BAR_W));
    bulk_copy(s_base + OFF_W2, a.W2, w2_bytes, bar(BAR_W));
    bulk_copy(s_base + OFF_W3, a.W3, w3_bytes, bar(BAR_W));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_base + OFF_TMEM),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the first tile's input chunk of this thread (train / predict; the
  // epilogue threads stage it)
  uint4 x_first = make_uint4(0u, 0u, 0u, 0u);
  if (MODE != MODE_SCREEN && tid < EPI_THREADS) {
    const int64_t grow = (int64_t)blockIdx.x * TM + (tid & (TM - 1));
    if (grow < a.n_rows) x_first = reinterpret_cast<const uint4 *>(a.x + grow * KF)[tid >> 7];
  }
  __syncthreads();   // the mbarriers are initialised
  // W1 has arrived before its bias columns are written over it (a wait that
  // runs out sets the abort flag: every later wait of the roles below then
  // gives up at once and the launch reports the timeout)
  const bool w_ok = warp_wait_spin(bar(BAR_W), 0u, abort);
  if (w_ok && tid < H) *reinterpret_cast<uint32_t *>(smem + OFF_W1 + cm_off(tid, KB1, KF)) = hi_lo(bias1);
  publish_smem();
  const uint32_t tmem = *tmem_slot;

  // W1 rows 128..255 start 16 row groups (of 8 rows x 16 K bytes) into the matrix
  const uint64_t dW1a = smem_desc(s_base + OFF_W1, KF), dW1b = smem_desc(s_base + OFF_W1 + 16 * KF * 16, KF),
                 dW2 = smem_desc(s_base + OFF_W2, H), dW3 = smem_desc(s_base + OFF_W3, H),
                 dX = smem_desc(s_base + OFF_X, KF), dOnes = smem_desc(s_base + OFF_ONES, BK),
                 dB2 = smem_desc(s_base + OFF_BB2, BK);
  const int64_t tiles = MODE == MODE_SCREEN ? (a.panel + TM - 1) / TM : 1;
  const int64_t n_items = MODE == MODE_SCREEN ? a.n_cand : (a.n_rows + TM - 1) / TM;
  const int64_t my_items = blockIdx.x < n_items ? (n_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_units = my_items * tiles;   // this CTA's tiles, in order
  const bool panel_cached = MODE == MODE_SCREEN && tiles == 1;

  if (warp == EPI_WARPS) {
    // ------------------------------------------------------------ MMA warp
    // (converged; the elected lane issues; every lane polls without suspending)
    if (n_units > 0) {
      const uint32_t e = elect_one();
      auto layer1 = [&](uint64_t dW, int bar_done) {
#pragma unroll
        for (int ks = 0; ks < KF / 16; ++ks)
          mma(tmem + COL_D1, dX + 16 * ks, dW + 16 * ks, idesc_bf16(TM, H / 2), ks > 0 ? 1u : 0u, e);
        commit(bar(bar_done), e);
      };
      bool ok = warp_wait_spin(bar(BAR_X), 0u, abort);
      // (test hook: without this first commit every wait of the CTA runs out)
      if (ok && !a.stall_test) layer1(dW1a, BAR_D1A);
      for (int64_t u = 0; ok && u < n_units; ++u) {
        const uint32_t par = (uint32_t)(u & 1);
        // second half of layer 1 once the first half's accumulators are read
        ok = warp_wait_spin(bar(BAR_H1A), par, abort);
        if (!ok) break;
        layer1(dW1b, BAR_D1B);
        // layer 2 overwrites D2: the previous tile's layer 3 has read H2 from it
        if (u > 0) {
          ok = warp_wait_spin(bar(BAR_D3), (uint32_t)((u - 1) & 1), abort);
          if (!ok) break;
        }
        // layer 2 (D2 = bias, then the first 128 units of H1 while their second half is written)
        mma(tmem + COL_D2, dOnes, dB2, idesc_bf16(TM, H), 0u, e);
#pragma unroll 1
        for (int ks = 0; ks < 8; ++ks)
          mma_ta(tmem + COL_D2, tmem + COL_H + 8 * ks, dW2 + 16 * ks, idesc_bf16(TM, H), 1u, e);
        ok = warp_wait_spin(bar(BAR_H1B), par, abort);
        if (!ok) break;
#pragma unroll 1
        for (int ks = 8; ks < 16; ++ks)
          mma_ta(tmem + COL_D2, tmem + COL_H + 8 * ks, dW2 + 16 * ks, idesc_bf16(TM, H), 1u, e);
        commit(bar(BAR_D2), e);
        // the next tile's first layer-1 half (its accumulator columns are free)
        if (u + 1 < n_units) {
          ok = warp_wait_spin(bar(BAR_X), (uint32_t)((u + 1) & 1), abort);
          if (!ok) break;
          layer1(dW1a, BAR_D1A);
        }
        // layer 3 once H2 is written.  Its partial sums overwrite the previous
        // tile's logits in H1's second half, which layer 2 has read by now; every
        // epilogue warp has seen those logits read before it arrives on H2
        // (warps 0-3 read them, column groups 1-3 wait for that before writing
        // this tile's second H1 half)
        ok = warp_wait_spin(bar(BAR_H2), par, abort);
        if (!ok) break;
        // four partial sums of four K steps each, interleaved so that no MMA waits
        // for the one before it
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int ks = 4 * p + j;
            mma_ta(tmem + col_d3(p), tmem + col_h2(ks), dW3 + 16 * ks, idesc_bf16(TM, N3), j > 0, e);
          }
        commit(bar(BAR_D3), e);
      }
      // every MMA this warp issued has finished before TMEM is released
      commit(bar(BAR_FIN), e);
      warp_wait(bar(BAR_FIN), 0u, abort);
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
    // Screening: the rows' values of a tile are summed by warp 0 one step later
    // (while the next tile's layer 2 runs), off the critical path, in a fixed order.
    auto finish_score = [&](int64_t pu, int64_t pitem, int64_t ptile) {
      if (!warp_wait_spin(bar(BAR_RED), (uint32_t)(pu & 1), abort)) return false;
      float v = (red[lane] + red[32 + lane]) + (red[64 + lane] + red[96 + lane]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        score += v;
        if (ptile == tiles - 1) {
          a.scores[pitem] = score / (float)a.panel;
          score = 0.0f;
        }
      }
      return true;
    };
    int64_t pend_u = -1, pend_item = 0, pend_tile = 0;   // a tile whose score sum is pending
    // Warps 0-3 read a tile's logits as soon as layer 3 is done (their TMEM
    // columns are the next layer 2's) but finish the softmax, and warp 0 the
    // candidate's score, only once the next tile's layer 2 is under way (the
    // epilogue warps wait for it anyway), off the critical path.
    float sm_lg[NO] = {};
    bool sm_pending = false, sm_valid = false;
    int64_t sm_grow = 0, sm_u = 0, sm_item = 0, sm_tile = 0;
    auto finish_softmax = [&]() {
      float v = 0.0f;
      if (sm_valid) {
        float m = sm_lg[0];
#pragma unroll
        for (int j = 1; j < NO; ++j) m = fmaxf(m, sm_lg[j]);
        float ex[NO], sum = 0.0f;
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          ex[j] = __expf(sm_lg[j] - m);
          sum += ex[j];
        }
        const float inv = 1.0f / sum;
        if (MODE == MODE_PREDICT) {
#pragma unroll
          for (int j = 0; j < NO; ++j) a.p[sm_grow * NO + j] = ex[j] * inv;
        } else {
          v = ex[a.bin] * inv;
        }
      }
      if (MODE == MODE_SCREEN) {
        red[row] = v;
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(BAR_RED)) : "memory");
        if (warp == 0) {
          pend_u = sm_u;
          pend_item = sm_item;
          pend_tile = sm_tile;
        }
      }
      sm_pending = false;
    };

    // A tile's input is fetched from global memory one tile ahead (into
    // registers) and written to shared memory once layer 1 has read the last one.
    struct Next {
      uint4 xv;        // train / predict: this thread's 16-byte chunk of X
      float g0, g1;    // screen: the candidate's log gains this thread places
    };
    auto fetch = [&](int64_t item, int64_t tile) {
      Next nx{make_uint4(0u, 0u, 0u, 0u), 0.0f, 0.0f};
      if (MODE != MODE_SCREEN) {
        const int64_t grow = item * TM + srow;
        if (grow < a.n_rows) nx.xv = reinterpret_cast<const uint4 *>(a.x + grow * KF)[sq];
      } else if (tile * TM + srow < a.panel) {
        if (sq == 1) nx.g0 = a.cand_lg[item * 3];
        if (sq == 2) {
          nx.g0 = a.cand_lg[item * 3 + 1];
          nx.g1 = a.cand_lg[item * 3 + 2];
        }
      }
      return nx;
    };
    // features KB1, KB1 + 1 (word 1 of chunk 2) are the layer-1 bias's ones
    const uint32_t ones = 0x3F803F80u;            // BF16 pair (1, 1)
    auto stage_x = [&](int64_t tile, bool first, const Next &nx) {
      if (MODE != MODE_SCREEN) {
        uint4 xv = nx.xv;
        if (sq == KB1 / 8) xv.y = ones;
        *reinterpret_cast<uint4 *>(xs + cm_off(srow, 8 * sq, KF)) = xv;
        return;
      }
      const int64_t prow = tile * TM + srow;
      const bool valid = prow < a.panel;
      if (!panel_cached || first) {
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
            ch[7] = nx.g0;
          } else {
            ch[0] = nx.g0;
            ch[1] = nx.g1;
          }
        }
        if (sq == KB1 / 8) ch[KB1 % 8] = ch[KB1 % 8 + 1] = 1.0f;
        *reinterpret_cast<uint4 *>(xs + cm_off(srow, 8 * sq, KF)) = pack8(ch);
      }
    };

    bool ok = true;
    const int64_t limit = MODE == MODE_SCREEN ? (int64_t)a.panel : a.n_rows;
    auto grow_of = [&](int64_t it, int64_t tl) { return (MODE == MODE_SCREEN ? tl * TM : it * TM) + row; };
    // Order per tile u: layer-1 second half, next input, the previous tile's
    // softmax and score, layer-2 epilogue (H2 in place of D2), then the NEXT
    // tile's layer-1 first half -- H1 and H2 live in different TMEM columns, so
    // it runs while layer 3 is on the tensor pipe -- and last this tile's logits.
    auto epi1a = [&](int64_t it, int64_t tl, uint32_t parity) {
      if (!warp_wait_spin(bar(BAR_D1A), parity, abort)) return false;
      const int64_t g = grow_of(it, tl);
      hidden32(lane_base + COL_D1 + 32 * grp, lane_base + COL_H + 16 * grp, 32 * grp, a.h1, a.act_cs, g,
                    MODE == MODE_TRAIN && g < limit);
      warp_arrive(bar(BAR_H1A));
      return true;
    };
    if (n_units > 0 && ok) {
      stage_x(0, true, MODE == MODE_SCREEN ? fetch(blockIdx.x, 0) : Next{x_first, 0.0f, 0.0f});
      warp_arrive(bar(BAR_X));
      ok = epi1a(blockIdx.x, 0, 0u);
    }
    int64_t item = blockIdx.x, tile = 0;          // unit u = (item, tile), advanced in order
    for (int64_t u = 0; ok && u < n_units; ++u) {
      const uint32_t par = (uint32_t)(u & 1);
      // the next unit, advanced without dividing
      const int64_t n_item = tile + 1 == tiles ? item + gridDim.x : item;
      const int64_t n_tile = tile + 1 == tiles ? 0 : tile + 1;
      const Next next = u + 1 < n_units ? fetch(n_item, n_tile) : Next{make_uint4(0u, 0u, 0u, 0u), 0.0f, 0.0f};
      const int64_t grow = grow_of(item, tile);
      const bool valid = grow < limit;
      const bool train = MODE == MODE_TRAIN && valid;
      // layer-1 epilogue, second half of 128 units (32 per warp); its columns
      // held the previous tile's logits, which warps 0-3 must have read
      ok = warp_wait_spin(bar(BAR_D1B), par, abort);
      if (!ok) break;
      if (grp > 0 && u > 0) {
        ok = warp_wait_spin(bar(BAR_D3C), (uint32_t)((u - 1) & 1), abort);
        if (!ok) break;
      }
      hidden32(lane_base + COL_D1 + 32 * grp, lane_base + COL_H + 64 + 16 * grp, 128 + 32 * grp, a.h1,
                    a.act_cs, grow, train);
      warp_arrive(bar(BAR_H1B));
      // the next tile's input (layer 1 of this tile has finished reading X)
      if (u + 1 < n_units) {
        stage_x(n_tile, false, next);
        warp_arrive(bar(BAR_X));
      }
      // the previous tile's softmax and score, while layer 2 runs (the epilogue
      // warps wait for it here anyway)
      if (MODE != MODE_TRAIN && warp < 4 && sm_pending) finish_softmax();
      if (MODE == MODE_SCREEN && warp == 0 && pend_u >= 0) {
        ok = finish_score(pend_u, pend_item, pend_tile);
        pend_u = -1;
        if (!ok) break;
      }
      // layer-2 epilogue, 64 units per warp, H2 written in place of their accumulators
      ok = warp_wait_spin(bar(BAR_D2), par, abort);
      if (!ok) break;
      const uint2 on = hidden64_in_place(lane_base + COL_D2 + 64 * grp, 64 * grp, a.h2, a.act_cs, grow, train);
      warp_arrive(bar(BAR_H2));
      // the next tile's first layer-1 half (H1 is free: layer 2 has finished)
      if (u + 1 < n_units) {
        ok = epi1a(n_item, n_tile, (uint32_t)((u + 1) & 1));
        if (!ok) break;
      }
      // this tile's logits: the four partial sums of layer 3
      ok = warp_wait_spin(bar(BAR_D3), par, abort);
      if (!ok) break;
      float dq[NO] = {};                         // training: the row's dZ3 as BF16 values
      float *dzs = reinterpret_cast<float *>(smem + OFF_DZ);
      if (warp < 4) {
        float part[4][16], lg[NO];
#pragma unroll
        for (int p = 0; p < 4; ++p) tmem_ld16(lane_base + col_d3(p), part[p]);
        warp_arrive(bar(BAR_D3C));               // the next H1 half may overwrite them
#pragma unroll
        for (int j = 0; j < NO; ++j) lg[j] = (part[0][j] + part[1][j]) + (part[2][j] + part[3][j]);
#pragma unroll
        for (int j = 0; j < NO; ++j) lg[j] += b3[j];
        if (MODE == MODE_TRAIN) {
          // softmax cross-entropy against the row's target fractions t:
          // loss = -sum t (z - lse), dLoss/dz = (p sum(t) - t) / rows
          if (valid) {
            float m = lg[0];
#pragma unroll
            for (int j = 1; j < NO; ++j) m = fmaxf(m, lg[j]);
            float ex[NO], t[NO], sum = 0.0f, ts = 0.0f;
#pragma unroll
            for (int j = 0; j < NO; ++j) {
              ex[j] = expf(lg[j] - m);
              sum += ex[j];
              t[j] = a.tgt[grow * NO + j];
              ts += t[j];
            }
            const float lse = m + logf(sum);
            float l = 0.0f, d[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) {
              l -= t[j] * (lg[j] - lse);
              d[j] = (ex[j] / sum * ts - t[j]) * a.inv_b;
            }
            const float zero8[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const float lo8[8] = {d[0], d[1], d[2], d[3], d[4], 0.0f, 0.0f, 0.0f};
            uint4 *o = reinterpret_cast<uint4 *>(a.dz3 + grow * N3);
            o[0] = pack8(lo8);
            o[1] = pack8(zero8);
            a.row_loss[grow] = l;
#pragma unroll
            for (int j = 0; j < NO; ++j) dq[j] = __bfloat162float(__float2bfloat16_rn(d[j]));
          }
          // the other column groups' warps take the row's dZ3 from shared memory
#pragma unroll
          for (int j = 0; j < NO; ++j) dzs[j * TM + row] = dq[j];
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(BAR_DZ)) : "memory");
        } else {
#pragma unroll
          for (int j = 0; j < NO; ++j) sm_lg[j] = lg[j];
          sm_pending = true;
          sm_valid = valid;
          sm_grow = grow;
          sm_u = u;
          sm_item = item;
          sm_tile = tile;
        }
      }
      // dZ2 of the row's 64 units of this column group.  The buffer is not
      // rewritten before every warp has read it: the next tile's dZ3 comes after
      // its layer 3, which waits for every warp's H2 of that tile.
      if (MODE == MODE_TRAIN) {
        if (warp >= 4) {
          ok = warp_wait_spin(bar(BAR_DZ), par, abort);
          if (!ok) break;
#pragma unroll
          for (int j = 0; j < NO; ++j) dq[j] = dzs[j * TM + row];
        }
        if (train) dz2_row(reinterpret_cast<const float *>(smem + OFF_W3F), dq, on, a.dz2, a.act_cs, grow, 64 * grp);
      }
      item = n_item;
      tile = n_tile;
    }
    if (MODE != MODE_TRAIN && warp < 4 && ok && sm_pending) finish_softmax();
    if (MODE == MODE_SCREEN && warp == 0 && ok && pend_u >= 0) finish_score(pend_u, pend_item, pend_tile);
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
