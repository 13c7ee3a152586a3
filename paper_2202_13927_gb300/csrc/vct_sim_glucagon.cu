// vct_sim_glucagon.cu -- the closed-loop kernel with the two glucagon
// compartments and the AP's glucagon mode compiled in (Sec. IV-B, IV-C): FP64
// plain form and the FP32 fast form with one patient per thread (natural
// allocation, and 144- and 128-register caps for m = 10).  Scenarios without
// glucagon run bit-identically in these variants.
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_glucagon(int op, const SimArgs *a, int precision, bool m10, int ppt, int reg,
                         int block, int grid, cudaStream_t st) {
  if (ppt > 1) return -1;
  if (precision == VCT_FP64) {
    if (reg != 0) return -1;
    return m10 ? run_variant<double, 10, 1, 0, true>(op, a, block, grid, st)
               : run_variant<double, 0, 1, 0, true>(op, a, block, grid, st);
  }
  if (!m10) return reg == 0 ? run_variant<float, 0, 1, 0, true>(op, a, block, grid, st) : -1;
  switch (reg) {
    case 0: return run_variant<float, 10, 1, 0, true>(op, a, block, grid, st);
    case 144: return run_variant<float, 10, 1, 144, true>(op, a, block, grid, st);
    case 128: return run_variant<float, 10, 1, 128, true>(op, a, block, grid, st);
    default: return -1;
  }
}
}  // namespace vct
