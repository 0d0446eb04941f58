// Instances of the resident 2D kernel with tiles of 2 rows (twice the threads of the
// 4-row tiles for the same slab): packs of 32..48-node boxes on one CTA, and 56..96-node
// boxes on clusters. The resident-plan autotuner times them beside the 4-row instances.
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_tr2(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 32, 26, 1, micro_fp32_2d_kernel<3, 2, 32, 26>, 0, 0, 2},
      {3, 40, 34, 1, micro_fp32_2d_kernel<3, 2, 40, 34>, 0, 0, 2},
      {3, 48, 42, 1, micro_fp32_2d_kernel<3, 2, 48, 42>, 0, 0, 2},
      {3, 56, 25, 2, micro_fp32_2d_kernel<3, 2, 56, 25>, 0, 0, 2},
      {3, 72, 22, 3, micro_fp32_2d_kernel<3, 2, 72, 22>, 0, 0, 2},
      {3, 80, 19, 4, micro_fp32_2d_kernel<3, 2, 80, 19>, 0, 0, 2},
      {3, 88, 21, 4, micro_fp32_2d_kernel<3, 2, 88, 21>, 0, 0, 2},
      {3, 96, 18, 5, micro_fp32_2d_kernel<3, 2, 96, 18>, 0, 0, 2},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
