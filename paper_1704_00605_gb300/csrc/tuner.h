// Launch shapes of every kernel family, chosen per size bucket by an
// autotuner that times candidate shapes on the device (tuner.cpp).
#pragma once

#include <cstdint>

#include "batch.h"
#include "internal.h"

namespace gb64 {

enum Kind {
  kSingleEncode = 0,
  kSingleDecode = 1,
  kBatchEncode = 2,
  kBatchDecode = 3,
  kDecodeWs = 4,  // the line-model kernel of the whitespace-removing decode
  kKinds = 5
};

constexpr int kBuckets = 8;

// Size bucket. Single kinds: by input size (bytes or characters). Batch
// kinds: by mean message length (total / nmsg); total < 0 means unknown.
int bucket_of(int kind, int64_t total, int64_t nmsg);

// Shape used by a single-buffer launch of n bytes/characters.
TileConfig single_config(int decode, uint64_t n);

// Shape of the line-model kernel for m input characters (threads 256 or
// 512; units per thread; stages; blocks_per_sm unused).
TileConfig ws_lines_config(uint64_t m);
TileConfig default_ws_lines_config(uint64_t m);
bool ws_lines_config_valid(const TileConfig& c);
size_t ws_lines_smem_bytes(const TileConfig& c);

// Shape for a batch of nmsg messages; total_bytes < 0 means "unknown".
BatchConfig tuned_batch_config(int decode, int64_t nmsg, int64_t total_bytes = -1);

}  // namespace gb64
