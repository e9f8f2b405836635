// SDIRK kernels for forward/backward recurrence orders (2, 1).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_INSTANTIATE(2, 1)
}  // namespace mg
