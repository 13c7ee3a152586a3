// vct_sim_f64.cu -- the plain FP64 form of the closed-loop kernel.
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_f64(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                    cudaStream_t st) {
  if (reg != 0 || ppt != 1) return -1;
  return m10 ? run_variant<double, 10, 1, 0>(op, a, block, grid, st)
             : run_variant<double, 0, 1, 0>(op, a, block, grid, st);
}
}  // namespace vct
