// Kernel instantiation for the model shape n_max^R = 10, N_bas^R = 10, n_max^A = 6,
// N_bas^A = 6, N_neu = 30, l_max = 4 / 2 / 1 (3-body / 4-body / 5-body).
#include "nep_kernels.cuh"

namespace nep {
const ShapeOps *shape_pbte() {
  static const ShapeOps ops = make_ops<Shape<10, 10, 6, 6, 30, 4, 2, 1>>();
  return &ops;
}
}  // namespace nep
