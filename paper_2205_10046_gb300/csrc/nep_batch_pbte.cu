// Kernel instantiation for the model shape n_max^R = 10, N_bas^R = 10, n_max^A = 6,
// N_bas^A = 6, N_neu = 30, l_max = 4 / 2 / 1 (3-body / 4-body / 5-body).
// Batched kernels (many structures, population members along grid.y) for this shape.
#define NEP_BATCH_KERNELS
#include "nep_kernels.cuh"

namespace nep {
template void attach_batch<Shape<10, 10, 6, 6, 30, 4, 2, 1>>(ShapeOps &o);
}  // namespace nep
