// Instances of the resident 2D kernel for boxes of 72..96 nodes per axis (order 4),
// each box split by rows over a thread-block cluster.
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_cluster_a(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 72, 33, 2, micro_fp32_2d_kernel<3, kResTR, 72, 33>},
      {3, 80, 37, 2, micro_fp32_2d_kernel<3, kResTR, 80, 37>},
      {3, 88, 28, 3, micro_fp32_2d_kernel<3, kResTR, 88, 28>},
      {3, 96, 30, 3, micro_fp32_2d_kernel<3, kResTR, 96, 30>},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
