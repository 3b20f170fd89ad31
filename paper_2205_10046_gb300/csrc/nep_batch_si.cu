// Kernel instantiation for the model shape n_max^R = 8, N_bas^R = 8, n_max^A = 4,
// N_bas^A = 4, N_neu = 50, l_max = 4 / 2 / 1 (3-body / 4-body / 5-body).
// Batched kernels (many structures, population members along grid.y) for this shape.
#define NEP_BATCH_KERNELS
#include "nep_kernels.cuh"

namespace nep {
template void attach_batch<Shape<8, 8, 4, 4, 50, 4, 2, 1>>(ShapeOps &o);
}  // namespace nep
