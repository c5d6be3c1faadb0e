// Batched decode that allocates no memory at all.
//
// b64_decode_batch takes its scratch (the weight offsets and the scan's block
// totals) from the stream-ordered allocator on every call. Some callers
// cannot do that: code that runs under a fixed device-memory budget or with
// its own pool (a serving loop that admits requests by free memory), hot
// paths that must never block (cudaMalloc and cudaFree can synchronize the
// whole device and stall other streams), and processes whose allocator is
// owned by another runtime. This variant runs the same kernels with its
// scratch in one file-scope device array of fixed size, so the call itself
// allocates nothing; the caller still passes every input and output buffer.
//
// Limits and sharing:
//   - at most kNoAllocMaxMsgs messages per call (larger batches are rejected
//     with B64_ERR_ARG before anything is enqueued);
//   - the array is loaded with the library on every GPU that uses it and
//     stays allocated there until the process exits (about 576 KiB);
//   - every call on a device uses the same array, so two calls whose work
//     overlaps on the GPU (different streams, no ordering) race and give
//     wrong results: order them on one stream or with events;
//   - nothing left from the previous call needs clearing: the kernels write
//     every offset and weight entry before reading it in the same call, and
//     the scan's per-block flags carry each call's number, so a flag left
//     by an earlier call is never taken for this call's;
//   - the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress); make that first call before any stream capture.
//     The address is kept for the life of the process, so the device must
//     not be reset (cudaDeviceReset) between calls.
#include <mutex>

#include "batch.h"
#include "internal.h"
#include "tuner.h"

namespace gb64 {
namespace {

constexpr int64_t kNoAllocMaxMsgs = 65536;
constexpr size_t kNoAllocScratchBytes = 576u << 10;

static_assert(batch_scratch_bytes(kNoAllocMaxMsgs) <= kNoAllocScratchBytes,
              "the fixed scratch must hold a batch of the largest accepted size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (looked up once
// per device with that device current; the host-side symbol is only a
// stand-in and must never be handed to a kernel).
void* noalloc_scratch(int device, cudaError_t* err) {
  static std::mutex mu;
  static void* addr[128] = {};
  std::lock_guard<std::mutex> g(mu);
  if (device < 0 || device >= 128) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
      return nullptr;
    }
    addr[device] = p;
  }
  return addr[device];
}

}  // namespace
}  // namespace gb64

using namespace gb64;

extern "C" int b64_decode_batch_noalloc(const char* src, const int64_t* in_off, int64_t nmsg,
                                        uint8_t* dst, int64_t* out_off, int32_t* status,
                                        int64_t* first_bad, int64_t* outlen,
                                        gb64_stream_t stream) {
  clear_error();
  if (nmsg < 0) {
    set_error("nmsg must be >= 0");
    return B64_ERR_ARG;
  }
  if (nmsg > kNoAllocMaxMsgs) {
    set_error("nmsg = %lld exceeds the %lld messages the fixed scratch of "
              "b64_decode_batch_noalloc holds; split the batch or use b64_decode_batch",
              (long long)nmsg, (long long)kNoAllocMaxMsgs);
    return B64_ERR_ARG;
  }
  if (!in_off || !out_off || (nmsg > 0 && (!src || !dst || !status || !first_bad || !outlen))) {
    set_error("in_off, out_off, src, dst, status, first_bad and outlen must not be null");
    return B64_ERR_ARG;
  }
  if ((reinterpret_cast<uintptr_t>(in_off) | reinterpret_cast<uintptr_t>(out_off) |
       reinterpret_cast<uintptr_t>(first_bad) | reinterpret_cast<uintptr_t>(outlen)) & 7u ||
      reinterpret_cast<uintptr_t>(status) & 3u) {
    set_error("offset and result arrays must be naturally aligned");
    return B64_ERR_ARG;
  }
  if (batch_scratch_bytes(nmsg) > kNoAllocScratchBytes) {
    set_error("internal: scratch of %lld messages does not fit the fixed array", (long long)nmsg);
    return B64_ERR_ARG;
  }
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return cuda_status(e, "decode_batch_noalloc: device query");
  void* scratch = noalloc_scratch(di->device, &e);
  if (!scratch) return cuda_status(e, "decode_batch_noalloc: scratch address");
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
  batch_scratch_split(scratch, nmsg, &a.weight_off, &a.parts);
  e = batch_launch(a, tuned_batch_config(1, nmsg));
  if (e != cudaSuccess) return cuda_status(e, "decode_batch_noalloc: launch");
  return B64_OK;
}
