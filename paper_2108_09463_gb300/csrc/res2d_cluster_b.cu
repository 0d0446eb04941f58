// Instances of the resident 2D kernel for boxes of 104..128 nodes per axis (order 4),
// each box split by rows over a thread-block cluster.
#include "micro_fp32_2d.cuh"

namespace hmm {

int res2d_variants_cluster_b(const ResVariant** v) {
  static const ResVariant t[] = {
      {3, 104, 33, 3, micro_fp32_2d_kernel<3, kResTR, 104, 33>},
      {3, 112, 27, 4, micro_fp32_2d_kernel<3, kResTR, 112, 27>},
      {3, 120, 23, 5, micro_fp32_2d_kernel<3, kResTR, 120, 23>},
      {3, 128, 25, 5, micro_fp32_2d_kernel<3, kResTR, 128, 25>},
  };
  *v = t;
  return (int)(sizeof(t) / sizeof(t[0]));
}

}  // namespace hmm
