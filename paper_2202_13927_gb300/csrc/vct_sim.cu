// vct_sim.cu -- dispatch to the compiled variants of the closed-loop kernel.
#include "vct_internal.cuh"

namespace vct {

int sim_variant_f32(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                    cudaStream_t st);
int sim_variant_f32_caps(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                         cudaStream_t st);
int sim_variant_f64(int op, const SimArgs *a, bool m10, int ppt, int reg, int block, int grid,
                    cudaStream_t st);
int sim_variant_glucagon(int op, const SimArgs *a, int precision, bool m10, int ppt, int reg,
                         int block, int grid, cudaStream_t st);
int sim_variant_f32_lean(int op, const SimArgs *a, int ppt, int reg, int lean, int block, int grid,
                         cudaStream_t st);

namespace {
// lean: 1 when the run has no trace, BG histogram, protocol or glucagon, 2 when
// it has a trace and none of the rest (the lean variants apply; with two
// patients per thread and a 192 / 168 cap only the packed lean form exists)
int dispatch(int op, const SimArgs *a, int precision, int m, int ppt, int reg, bool glu, int lean,
             int block, int grid, cudaStream_t st) {
  const bool m10 = m == 10;
  if (glu) return sim_variant_glucagon(op, a, precision, m10, ppt, reg, block, grid, st);
  if (precision == VCT_FP64) return sim_variant_f64(op, a, m10, ppt, reg, block, grid, st);
  if (reg == 0) return sim_variant_f32(op, a, m10, ppt, reg, block, grid, st);
  if (m10 && lean) {
    const int r = sim_variant_f32_lean(op, a, ppt, reg, lean, block, grid, st);
    if (r >= 0) return r;
  }
  return sim_variant_f32_caps(op, a, m10, ppt, reg, block, grid, st);
}
}  // namespace

bool sim_variant_exists(int precision, int m, int ppt, int reg, bool glu, int lean) {
  return dispatch(1, nullptr, precision, m, ppt, reg, glu, lean, 128, 0, nullptr) >= 0;
}

cudaError_t launch_simulation(const SimArgs &a, int precision, int block, int ppt, int reg,
                              int grid, cudaStream_t st) {
  int r = dispatch(0, &a, precision, a.m, ppt, reg, a.glucagon != 0, a.lean, block, grid, st);
  return r < 0 ? cudaErrorInvalidValue : (cudaError_t)r;
}

int sim_max_blocks_per_sm(int precision, int block, int ppt, int reg, int m, bool glu, int lean) {
  int r = dispatch(1, nullptr, precision, m, ppt, reg, glu, lean, block, 0, nullptr);
  return r < 0 ? 0 : r;
}

}  // namespace vct
