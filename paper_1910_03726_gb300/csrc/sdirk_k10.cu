// SDIRK kernels for forward/backward recurrence orders (1, 0).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_INSTANTIATE(1, 0)
}  // namespace mg
