// Instances of the resident 2D kernel with strides taken from each box (any box
// size, both stencil orders); the cluster size is chosen per box.
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_any(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 0, 0, 0, micro_fp32_2d_kernel<3, kResTR, 0, 0>},
      {1, 0, 0, 0, micro_fp32_2d_kernel<1, kResTR, 0, 0>},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
