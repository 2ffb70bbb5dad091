// Kernel instantiation for 3 points per direction (polynomial degree 2).
#include "dg_kernels.cuh"

namespace dg {
template struct Driver<3>;
}  // namespace dg
