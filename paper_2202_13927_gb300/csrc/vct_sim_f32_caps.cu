// vct_sim_f32_caps.cu -- FP32 fast-form variants (m = 10) with capped register
// allocation: one patient per thread with 128, 112, 96 or 80 registers, two with
// 168 or 128; they trade a few spills for more resident warps.  The autotuner
// picks.
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_f32_caps(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                         cudaStream_t st) {
  if (!m10) return -1;
  if (ppt == 1) {
    switch (reg) {
      case 128: return run_variant<float, 10, 1, 128>(op, a, block, grid, st);
      case 112: return run_variant<float, 10, 1, 112>(op, a, block, grid, st);
      case 96: return run_variant<float, 10, 1, 96>(op, a, block, grid, st);
      case 80: return run_variant<float, 10, 1, 80>(op, a, block, grid, st);
      default: return -1;
    }
  }
  if (ppt == 2) {
    switch (reg) {
      case 168: return run_variant<float, 10, 2, 168>(op, a, block, grid, st);
      case 128: return run_variant<float, 10, 2, 128>(op, a, block, grid, st);
      default: return -1;
    }
  }
  return -1;
}
}  // namespace vct
