// SDIRK level-1 FCF split over a cluster of two CTAs, recurrence orders (2, 1).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_SPLIT_INSTANTIATE(2, 1)
}  // namespace mg
