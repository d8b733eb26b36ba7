// gace_hot.h -- size of the hot-key cache that staged global histograms keep
// in shared memory after their stage buffers (host and device agree on it).
#pragma once

#include <stdint.h>

namespace gace {

// 2^kHotLog slots of (key, count), 8 bytes each.
#ifndef GACE_HOT_CACHE
#define GACE_HOT_CACHE 1
#endif
constexpr bool kHotCache = GACE_HOT_CACHE != 0;
constexpr uint32_t kHotLog = 10;

}  // namespace gace
