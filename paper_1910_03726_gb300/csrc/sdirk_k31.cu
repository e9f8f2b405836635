// SDIRK kernels for forward/backward recurrence orders (3, 1).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_INSTANTIATE(3, 1)
}  // namespace mg
