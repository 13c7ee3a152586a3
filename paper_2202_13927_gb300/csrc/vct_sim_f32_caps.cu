// vct_sim_f32_caps.cu -- FP32 fast-form variants (m = 10, one patient per
// thread) with capped register allocation: 112, 96 or 80 registers per thread
// trade a few spills for more resident warps.  The autotuner picks.
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_f32_caps(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                         cudaStream_t st) {
  if (!m10 || ppt != 1) return -1;
  switch (reg) {
    case 112: return run_variant<float, 10, 1, 112>(op, a, block, grid, st);
    case 96: return run_variant<float, 10, 1, 96>(op, a, block, grid, st);
    case 80: return run_variant<float, 10, 1, 80>(op, a, block, grid, st);
    default: return -1;
  }
}
}  // namespace vct
