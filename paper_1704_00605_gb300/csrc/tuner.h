// Launch-shape selection for the batched kernels (per size bucket).
#pragma once

#include <cstdint>

#include "batch.h"

namespace gb64 {

// Shape for a batch of nmsg messages; total_bytes < 0 means "unknown".
BatchConfig tuned_batch_config(int decode, int64_t nmsg, int64_t total_bytes = -1);

}  // namespace gb64
