// Kernel instantiation for 2 points per direction (polynomial degree 1).
#include "dg_kernels.cuh"

namespace dg {
template struct Driver<2>;
}  // namespace dg
