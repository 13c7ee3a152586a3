// vct_sim_f32_lean.cu -- the FP32 fast form (m = 10, capped registers) with the
// trace, BG-histogram and protocol-meal branches compiled out: the kernel of a
// run that asks for none of them (fixed daily meals, indicators only), as the
// paper-scale trial does -- one patient per thread, or two in packed FP32
// pairs (vct_sim_pk2.cuh); and the same with the trace branch alone kept, for
// a traced run of that kind.  Results are bit for bit those of the full
// variants.
#include "vct_sim_body.cuh"

namespace vct {
int sim_variant_f32_lean(int op, const SimArgs *a, int ppt, int reg, int lean, int block, int grid,
                         cudaStream_t st) {
  if (lean == 2) {  // a traced run: the trace branch kept, one patient per thread, 128 registers
    return ppt == 1 && reg == 128 ? run_variant<float, 10, 1, 128, false, 2>(op, a, block, grid, st) : -1;
  }
  if (ppt == 2) {  // two patients per thread in packed FP32 pairs
    switch (reg) {
      case 192: return run_variant<float, 10, 2, 192, false, true, true>(op, a, block, grid, st);
      case 168: return run_variant<float, 10, 2, 168, false, true, true>(op, a, block, grid, st);
      default: return -1;
    }
  }
  if (ppt != 1) return -1;
  switch (reg) {
    case 128: return run_variant<float, 10, 1, 128, false, true>(op, a, block, grid, st);
    case 112: return run_variant<float, 10, 1, 112, false, true>(op, a, block, grid, st);
    case 96: return run_variant<float, 10, 1, 96, false, true>(op, a, block, grid, st);
    case 80: return run_variant<float, 10, 1, 80, false, true>(op, a, block, grid, st);
    default: return -1;
  }
}
}  // namespace vct
