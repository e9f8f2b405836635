// SDIRK kernels for forward/backward recurrence orders (3, 2).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_INSTANTIATE(3, 2)
}  // namespace mg
