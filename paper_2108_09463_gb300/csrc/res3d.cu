// Instances of the 3D resident kernels (order 4). First the z-column kernel
// (micro_fp32_3d_col.cuh: boxes from 27^3 to 32^3, slabs of at most 3 planes, so 9 CTAs for
// 32^3; separable coefficients of at most two terms), then the z-slab kernel's
// canvases of 16, 24 and 32 nodes per axis with the cluster sizes whose slabs fit one
// SM (9 CTAs of 3 planes for 32^3), which also serve tabulated coefficients. Larger 3D
// boxes and the order-2 stencil in 3D run on the generic kernel.
#include "micro_fp32_3d_col.cuh"

namespace hmm {

int res3d_variants(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 32, kCol3S, 0, micro_fp32_3d_col_kernel<3>, -1},
      {3, 16, 10, 1, micro_fp32_3d_kernel<3, 4, 16, 10>, 4},
      {3, 24, 6, 3, micro_fp32_3d_kernel<3, 3, 24, 6>, 3},
      {3, 32, 3, 9, micro_fp32_3d_kernel<3, 3, 32, 3>, 3},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
