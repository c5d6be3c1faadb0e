// Internal interface of the batched kernels (batch.cu) used by the C ABI,
// the tuner and the serving loop.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace gb64 {

// Shape of a batched launch.
struct BatchConfig {
  int threads;        // 128, 256 or 512 threads per CTA
  int64_t tile;       // input bytes (encode, multiple of 384) or characters
                      // (decode, multiple of 512) per warp tile
  int blocks_per_sm;  // persistent CTAs per SM at most (0: as many as fit)
  int stages = 4;     // input stages per warp (2..6)
  int kernel = 0;     // 0 = short messages one thread each (packed batches)
                      // and staged per-warp tiles for the rest, 1 = staged
                      // tiles for every message, 2 = short messages one
                      // thread each and unstaged tiles (up to 64 rows),
                      // 3 = the flat decode (encode) of a packed batch whose
                      // encoded lengths are all multiples of 4 (padded
                      // output), else as 2
};

struct BatchArgs {
  int decode = 0;
  const uint8_t* src = nullptr;
  const int64_t* in_off = nullptr;
  int64_t nmsg = 0;
  uint8_t* dst = nullptr;
  int64_t* out_off = nullptr;
  int64_t* weight_off = nullptr;  // scratch: nmsg + 1 entries
  void* parts = nullptr;          // scratch: block totals of the scan
  int32_t* status = nullptr;    // decode only
  int64_t* first_bad = nullptr;
  int64_t* outlen = nullptr;
  cudaStream_t stream = nullptr;
  uint32_t flags = 0;  // variants of Section 2 / Appendix A (B64_FLAG_*)
};

// One message of a descriptor batch: its bytes anywhere in device memory and
// the offset of its output in the batch's output buffer.
struct MsgDesc {
  const uint8_t* src;
  int64_t len;
  int64_t out_off;
};

// Weight of a tile beyond its bytes when the tile kernels split a batch
// among warps: the bookkeeping a warp spends on a tile whatever its length,
// in bytes of coding that take the same time. A message of len bytes in
// t tiles weighs len + t * kBatchTileCost (0 with no tiles).
constexpr int64_t kBatchTileCost = 1024;

// Codes a batch described by host-built descriptors and weight offsets
// (weight_off[j] = sum over earlier messages of their weights above, every
// message of len > 0 being cut into ceil(len / cfg.tile) tiles), with no
// device scan: the persistent tile kernel (+ the decode finish kernel, + an
// initialisation of first_bad/outlen when init_results).
cudaError_t batch_launch_desc(int decode, const MsgDesc* desc, int64_t nmsg, uint8_t* dst,
                              const int64_t* weight_off, int32_t* status, int64_t* first_bad,
                              int64_t* outlen, const BatchConfig& cfg, bool init_results,
                              cudaStream_t stream, uint32_t flags = 0);

// Messages per block of the batch scan (its threads x items per thread).
constexpr int64_t kBatchScanPerBlock = 512 * 4;

// Bytes of scratch a batch of nmsg messages needs: weight_off (nmsg + 1
// int64) and per scan block its published totals (a flag and four int64; at
// least one block). Nothing in it needs clearing between calls: the scan
// tags what it writes with the call's number.
constexpr size_t batch_scratch_bytes(int64_t nmsg) {
  return (size_t)(nmsg + 1) * 8 +
         (size_t)((nmsg + kBatchScanPerBlock - 1) / kBatchScanPerBlock > 0
                      ? (nmsg + kBatchScanPerBlock - 1) / kBatchScanPerBlock
                      : 1) * 40;
}

// Splits a scratch block of batch_scratch_bytes(nmsg) into its arrays.
inline void batch_scratch_split(void* scratch, int64_t nmsg, int64_t** weight_off, void** parts) {
  *weight_off = static_cast<int64_t*>(scratch);
  *parts = *weight_off + (nmsg + 1);
}

// Output offsets of a batch, and its weight offsets (the prefix sums of the
// weights above, by which the tile kernels split the work among warps);
// first_bad/outlen (decode) are initialised when non-null.
// small_max > 0: messages of at most small_max bytes / characters get no
// tiles (threads code them one each).
cudaError_t batch_offsets(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                          int64_t* weight_off, int64_t tile, void* parts, int64_t* first_bad,
                          int64_t* outlen, cudaStream_t stream, uint32_t flags = 0,
                          int64_t small_max = 0);
int64_t batch_small_max(int decode);

// Offsets + the persistent tile kernel (+ the decode finish kernel).
cudaError_t batch_launch(const BatchArgs& a, const BatchConfig& cfg);

// Largest dynamic shared memory a valid batch shape may ask for: the
// opt-in limit of a CTA on sm_103 (227 KiB) less the kernel's static shared
// memory (tables, barriers and tile views): up to 9.5 KiB decoding, and up
// to 17.4 KiB encoding, whose table holds 8 KiB of character pairs (512
// threads). A launch still checks the device it runs on.
constexpr size_t kBatchSmemLimitDecode = 227 * 1024 - 10 * 1024;
constexpr size_t kBatchSmemLimitEncode = 227 * 1024 - 18 * 1024;

// Dynamic shared memory of a batched launch: per warp, `stages` input
// stages of a tile (and, decoding, one output buffer).
size_t batch_smem_bytes(int decode, const BatchConfig& c);

// Valid shapes and the defaults used when the tuner has no entry.
bool batch_config_valid(int decode, const BatchConfig& c);
BatchConfig default_batch_config(int decode, int64_t mean_len = -1);

}  // namespace gb64
