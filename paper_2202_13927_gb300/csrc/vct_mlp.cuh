// vct_mlp.cuh -- types shared by the surrogate's translation units.
#pragma once
#include <cuda_bf16.h>

#include "vct_internal.cuh"

namespace vct {

constexpr int kSurrH = VCT_SURR_HIDDEN;   // hidden width
constexpr int kSurrKF = VCT_SURR_KF;      // padded feature width
constexpr int kSurrNF = VCT_SURR_FEATURES;
constexpr int kSurrNO = VCT_NBINS;        // outputs
constexpr int kSurrNOP = 8;               // outputs padded (the layer-3 bias copy)

enum { MODE_TRAIN = 0, MODE_PREDICT = 1, MODE_SCREEN = 2 };

// Element (r, k) of a BF16 [rows][K] matrix in the canonical K-major layout of
// the tensor cores' shared-memory operands (core matrices of 8 rows x 8
// elements, 128 bytes; those of one 8-row group consecutive along k): the
// forward kernel copies a weight image in this layout into shared memory whole.
__host__ __device__ constexpr int64_t canon_index(int r, int k, int K) {
  return (int64_t)(r >> 3) * K * 8 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

struct FwdArgs {
  const __nv_bfloat16 *W1, *W2, *W3;  // canonical images (canon_index) of [H][KF], [H][H],
                                       // [16][H] (rows >= 5 zero); 16-byte aligned
  const float *b1, *b2, *b3;           // [H], [H], [>= 5]
  const __nv_bfloat16 *x;              // train / predict: [rows][KF]
  int64_t n_rows;
  __nv_bfloat16 *h1, *h2;              // train: [H / 8][act_rows][8] (see act_cs)
  const float *tgt;                    // train: [rows][5] target fractions
  __nv_bfloat16 *dz3;                  // train: [rows][16] dLoss/dlogits (BF16, columns >= 5 zero)
  __nv_bfloat16 *dz2;                  // train: dLoss/dZ2 = (dZ3 W3) where Z2 > 0 (BF16), as h1
  int64_t act_cs;                      // train: h1, h2 and dz2 are stored chunk-major, unit u of
                                       // row r at (u / 8) act_cs + 8 r + u % 8 (act_cs >= 8 rows):
                                       // a warp's 32 rows of one 8-unit chunk are 512 contiguous bytes
  float *row_loss;                     // train: [rows] cross-entropy of each row
  float inv_b;                         // train: 1 / rows (the loss is the mean over the rows)
  float *p;                            // predict: [rows][5]
  // screen
  const float *panel_x;                // [P][KF] features of the panel (gain slots ignored)
  int32_t panel;                       // P
  const float *cand_lg;                // [n_cand][3] standardized log gains
  int64_t n_cand;
  int32_t bin;
  float *scores;                       // [n_cand]
  int *error;                          // set to 1 if a bounded wait gives up
  int stall_test;                      // test hook: withhold the first commit (waits run out)
};

// Fused 3-layer forward on the tcgen05 tensor cores (vct_mlp_fwd.cu).
cudaError_t launch_forward(const FwdArgs &a, int mode, int64_t items, cudaStream_t st);

// C = A B on the tcgen05 tensor cores (vct_mlp_gemm.cu): A[m][k] = A[m sam + k sak],
// B[k][n] = B[k sbk + n sbn], one stride of each operand 1, the other a multiple
// of 8, K a multiple of 8 when an operand is K-contiguous, base addresses 16-byte
// aligned.  Each operand's contiguous dimension may be stored in chunks of 8
// elements acs (bcs) apart instead (8: stored plainly), e.g. A[m][k] =
// A[m sam + (k / 8) acs + k % 8] when sak == 1.  Grid (tiles_n, tiles_m, splits):
// tile 128 x NT (NT a multiple of 16, <= 256), split z covers k in [z kc, (z+1) kc).
struct TcGemmArgs {
  const __nv_bfloat16 *A;
  int64_t sam, sak, acs;
  const __nv_bfloat16 *B;
  int64_t sbk, sbn, bcs;
  int M, N, NT;
  int64_t K, kc;
  int mode;                      // 0: split z's FP32 partial [M][N] at partial + z pstride;
                                 // 1: out[M][N] = BF16(C) where mask > 0
  float *partial;
  int64_t pstride;               // mode 0: floats from one split's partial to the next (>= M N)
  float *bias_partial;           // mode 0, or null: split z's sums of A's rows over its K range at
                                 // bias_partial + z pstride (A stored along M: sam == 1)
  __nv_bfloat16 *out;
  const __nv_bfloat16 *mask;     // element (m, n) at m mrs + (n / 8) mcs + n % 8
  int64_t mrs, mcs;
  int *error;                    // bit 0 set if a bounded wait gives up
};
cudaError_t launch_tc_gemm(const TcGemmArgs &g, int tiles_n, int tiles_m, int splits, cudaStream_t st);

}  // namespace vct
