// SDIRK level-1 FCF split over a cluster of two CTAs, recurrence orders (3, 2).
#include "sdirk_impl.cuh"

namespace mg {
MG_SDIRK_SPLIT_INSTANTIATE(3, 2)
}  // namespace mg
