// Kernel instantiation for 4 points per direction (polynomial degree 3).
#include "dg_kernels.cuh"

namespace dg {
template struct Driver<4>;
}  // namespace dg
