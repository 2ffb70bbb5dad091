// Kernel instantiation for 5 points per direction (polynomial degree 4).
#include "dg_kernels.cuh"

namespace dg {
template struct Driver<5>;
}  // namespace dg
