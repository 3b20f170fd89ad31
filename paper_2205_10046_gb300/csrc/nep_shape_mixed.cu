// Kernel instantiation for the model shape n_max^R = 8, N_bas^R = 8, n_max^A = 4,
// N_bas^A = 4, N_neu = 40, l_max = 4 / 2 / 1 (3-body / 4-body / 5-body).
#include "nep_kernels.cuh"

namespace nep {
const ShapeOps *shape_mixed() {
  static const ShapeOps ops = make_ops<Shape<8, 8, 4, 4, 40, 4, 2, 1>>();
  return &ops;
}
}  // namespace nep
