// Instances of the resident 2D kernel with the RK4P micro stepper: canvases of 48
// nodes (one CTA) and 64 nodes (a 2-CTA cluster), and the instances with strides
// taken from each box (any box size, both stencil orders).
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_rk4(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 48, 42, 1, micro_fp32_2d_kernel<3, kResTR, 48, 42, 1>, 0, 1},
      {3, 64, 29, 2, micro_fp32_2d_kernel<3, kResTR, 64, 29, 1>, 0, 1},
      {3, 0, 0, 0, micro_fp32_2d_kernel<3, kResTR, 0, 0, 1>, 0, 1},
      {1, 0, 0, 0, micro_fp32_2d_kernel<1, kResTR, 0, 0, 1>, 0, 1},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
