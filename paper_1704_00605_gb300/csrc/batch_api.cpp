// C ABI of the batched calls: argument checks, stream-ordered scratch, and
// the launch shape chosen by the tuner for the batch's size bucket.
#include <algorithm>

#include "batch.h"
#include "internal.h"
#include "tuner.h"

namespace gb64 {

bool batch_config_valid(int decode, const BatchConfig& c) {
  if (c.threads != 128 && c.threads != 256 && c.threads != 512) return false;
  if (c.blocks_per_sm < 0 || c.blocks_per_sm > 32) return false;
  if (c.stages < 2 || c.stages > 6) return false;
  if (c.kernel < 0 || c.kernel > 3) return false;
  const int64_t row = decode ? 512 : 384;  // one unit per lane of a warp
  const int64_t max_rows = c.kernel >= 2 ? 64 : 16;  // unstaged tiles need no shared memory
  if (c.tile < row || c.tile > max_rows * row || c.tile % row) return false;
  return batch_smem_bytes(decode, c) <= (decode ? kBatchSmemLimitDecode : kBatchSmemLimitEncode);
}

// Shapes measured fastest on GB300: mean message length below 1 KiB
// (262,144 messages of 256 B) and above (100,000 messages of 6.3 KiB on
// average, and 64 of 1 MiB). Decoding longer messages, unstaged tiles of 32
// rows beat staged ones (a shared-memory output buffer and its bulk store
// per tile, and tiles limited to 8 rows); encoding, the two are even and
// staged tiles stay. Decoding, the flat decode (kernel 3) takes every padded
// batch of messages of at least 1 Ki characters on average (and aligned
// buffers) and leaves the rest to the unstaged tiles: 1.2-1.4x faster on
// every mix measured. The flat encode is left to the shape table: the
// staged tiles beat it on every mix measured (equal 4 KiB - 1 MiB messages
// by 1.2-1.3x, the log-normal batch by 1.1x); one CTA of 16 warps per SM
// beats two of 8 by 2 % on the log-normal batch and ties elsewhere.
// mean_len < 0: unknown.
BatchConfig default_batch_config(int decode, int64_t mean_len) {
  const bool small = mean_len >= 0 && mean_len < 1024;
  if (decode) return small ? BatchConfig{128, 1024, 0, 2} : BatchConfig{128, 16384, 0, 2, 3};
  return small ? BatchConfig{256, 1536, 0, 2} : BatchConfig{512, 6144, 0, 2};
}

namespace {

int check_offsets_args(const int64_t* in_off, int64_t nmsg, const int64_t* out_off) {
  if (nmsg < 0) {
    set_error("nmsg must be >= 0");
    return B64_ERR_ARG;
  }
  if (!in_off || !out_off) {
    set_error("in_off and out_off must not be null");
    return B64_ERR_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(in_off) | reinterpret_cast<uintptr_t>(out_off)) & 7u) {
    set_error("offset arrays must be 8-byte aligned");
    return B64_ERR_ARG;
  }
  return B64_OK;
}

constexpr int kAllFlags = B64_FLAG_URL | B64_FLAG_NOPAD | B64_FLAG_STRICT_TAIL;

int check_flags(int flags) {
  if (flags & ~kAllFlags) {
    set_error("unknown flag bits 0x%x", flags & ~kAllFlags);
    return B64_ERR_ARG;
  }
  return B64_OK;
}

int run_batch(BatchArgs a) {
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, batch_scratch_bytes(a.nmsg), a.stream);
  if (e != cudaSuccess) return cuda_status(e, "batch: scratch");
  batch_scratch_split(scratch, a.nmsg, &a.weight_off, &a.parts);
  const BatchConfig cfg = tuned_batch_config(a.decode, a.nmsg);
  e = batch_launch(a, cfg);
  cudaError_t ef = cudaFreeAsync(scratch, a.stream);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return cuda_status(e, "batch: launch");
  return B64_OK;
}

}  // namespace
}  // namespace gb64

using namespace gb64;

extern "C" {

int b64_batch_out_offsets_ex(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                             int flags, gb64_stream_t stream) {
  clear_error();
  int rc = check_offsets_args(in_off, nmsg, out_off);
  if (rc == B64_OK) rc = check_flags(flags);
  if (rc != B64_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, batch_scratch_bytes(nmsg), s);
  if (e != cudaSuccess) return cuda_status(e, "batch_out_offsets: scratch");
  int64_t* weight_off;
  void* parts;
  batch_scratch_split(scratch, nmsg, &weight_off, &parts);
  e = batch_offsets(decode ? 1 : 0, in_off, nmsg, out_off, weight_off, 1 << 20, parts, nullptr,
                    nullptr, s, (uint32_t)flags);
  cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return cuda_status(e, "batch_out_offsets");
  return B64_OK;
}

int b64_batch_out_offsets(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                          gb64_stream_t stream) {
  return b64_batch_out_offsets_ex(decode, in_off, nmsg, out_off, 0, stream);
}

int b64_encode_batch_ex(const uint8_t* src, const int64_t* in_off, int64_t nmsg, char* dst,
                        int64_t* out_off, int flags, gb64_stream_t stream) {
  clear_error();
  int rc = check_offsets_args(in_off, nmsg, out_off);
  if (rc == B64_OK) rc = check_flags(flags);
  if (rc != B64_OK) return rc;
  if (nmsg > 0 && (!src || !dst)) {
    set_error("src and dst must not be null");
    return B64_ERR_ARG;
  }
  BatchArgs a;
  a.decode = 0;
  a.src = src;
  a.in_off = in_off;
  a.nmsg = nmsg;
  a.dst = reinterpret_cast<uint8_t*>(dst);
  a.out_off = out_off;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  a.flags = (uint32_t)flags;
  return run_batch(a);
}

int b64_encode_batch(const uint8_t* src, const int64_t* in_off, int64_t nmsg, char* dst,
                     int64_t* out_off, gb64_stream_t stream) {
  return b64_encode_batch_ex(src, in_off, nmsg, dst, out_off, 0, stream);
}

int b64_decode_batch_ex(const char* src, const int64_t* in_off, int64_t nmsg, uint8_t* dst,
                        int64_t* out_off, int32_t* status, int64_t* first_bad, int64_t* outlen,
                        int flags, gb64_stream_t stream) {
  clear_error();
  int rc = check_offsets_args(in_off, nmsg, out_off);
  if (rc == B64_OK) rc = check_flags(flags);
  if (rc != B64_OK) return rc;
  if (nmsg > 0 && (!src || !dst || !status || !first_bad || !outlen)) {
    set_error("src, dst, status, first_bad and outlen must not be null");
    return B64_ERR_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(first_bad) | reinterpret_cast<uintptr_t>(outlen)) & 7u ||
      reinterpret_cast<uintptr_t>(status) & 3u) {
    set_error("result arrays must be naturally aligned");
    return B64_ERR_ARG;
  }
  BatchArgs a;
  a.decode = 1;
  a.src = reinterpret_cast<const uint8_t*>(src);
  a.in_off = in_off;
  a.nmsg = nmsg;
  a.dst = dst;
  a.out_off = out_off;
  a.status = status;
  a.first_bad = first_bad;
  a.outlen = outlen;
  a.stream = reinterpret_cast<cudaStream_t>(stream);
  a.flags = (uint32_t)flags;
  return run_batch(a);
}

int b64_decode_batch(const char* src, const int64_t* in_off, int64_t nmsg, uint8_t* dst,
                     int64_t* out_off, int32_t* status, int64_t* first_bad, int64_t* outlen,
                     gb64_stream_t stream) {
  return b64_decode_batch_ex(src, in_off, nmsg, dst, out_off, status, first_bad, outlen, 0,
                             stream);
}

}  // extern "C"
