// Launch-shape table of the batched kernels.
#include "tuner.h"

namespace gb64 {

BatchConfig tuned_batch_config(int decode, int64_t nmsg, int64_t total_bytes) {
  (void)nmsg;
  (void)total_bytes;
  return default_batch_config(decode);
}

}  // namespace gb64
