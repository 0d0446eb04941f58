// Instances of the resident 2D kernel for packs of small boxes (order 4, one CTA
// per work item), canvases of 24..64 nodes per axis.
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_pack(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 24, 18, 1, micro_fp32_2d_kernel<3, kResTR, 24, 18>},
      {3, 32, 26, 1, micro_fp32_2d_kernel<3, kResTR, 32, 26>},
      {3, 40, 34, 1, micro_fp32_2d_kernel<3, kResTR, 40, 34>},
      {3, 48, 42, 1, micro_fp32_2d_kernel<3, kResTR, 48, 42>},
      {3, 56, 50, 1, micro_fp32_2d_kernel<3, kResTR, 56, 50>},
      {3, 64, 58, 1, micro_fp32_2d_kernel<3, kResTR, 64, 58>},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
