// vct_sim_f32.cu -- FP32 fast-form variants of the closed-loop kernel with the
// natural register allocation (see vct_sim_body.cuh).
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_f32(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                    cudaStream_t st) {
  if (reg != 0) return -1;
  if (m10) {
    if (ppt == 1) return run_variant<float, 10, 1, 0>(op, a, block, grid, st);
    if (ppt == 2) return run_variant<float, 10, 2, 0>(op, a, block, grid, st);
  } else {
    if (ppt == 1) return run_variant<float, 0, 1, 0>(op, a, block, grid, st);
    if (ppt == 2) return run_variant<float, 0, 2, 0>(op, a, block, grid, st);
  }
  return -1;
}
}  // namespace vct
