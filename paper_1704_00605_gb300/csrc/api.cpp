// The C ABI of libgb64 (include/gb64.h): argument checks on the host, the
// per-thread error text, device facts, and the single-buffer calls.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "tuner.h"

namespace gb64 {

namespace {
thread_local std::string t_error;

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (na == 0 || nb == 0) return false;
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

// Device memory for the result of a synchronous decode, one per device and
// calling thread (the call waits for its stream before returning, so a
// thread never has two decodes in flight on it).
struct DecodeScratch {
  b64_result* dev = nullptr;
  b64_result* host = nullptr;  // pinned
};

DecodeScratch* decode_scratch(int device, cudaError_t* err) {
  thread_local std::vector<DecodeScratch> per_device;
  if ((int)per_device.size() <= device) per_device.resize(device + 1);
  DecodeScratch& s = per_device[device];
  if (!s.dev) {
    cudaError_t e = cudaMalloc(&s.dev, sizeof(b64_result));
    if (e == cudaSuccess) e = cudaMallocHost(&s.host, sizeof(b64_result));
    if (e != cudaSuccess) {
      *err = e;
      if (s.dev) cudaFree(s.dev);
      s.dev = nullptr;
      return nullptr;
    }
  }
  return &s;
}
}  // namespace

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_error = buf;
}

void clear_error() { t_error.clear(); }

int cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  cudaGetLastError();  // do not leave a non-sticky error for the caller's next CUDA call
  return e == cudaErrorMemoryAllocation ? B64_ERR_NOMEM : B64_ERR_CUDA;
}

const DeviceInfo* device_info(cudaError_t* err) {
  static std::mutex mu;
  static DeviceInfo infos[128];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    *err = e != cudaSuccess ? e : cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  DeviceInfo& d = infos[dev];
  if (d.device < 0) {
    DeviceInfo t;
    t.device = dev;
    e = cudaDeviceGetAttribute(&t.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&t.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&t.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&t.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    d = t;
  }
  return &d;
}

namespace {
constexpr uint64_t kDefaultWaitNs = 2000000000ull;
std::atomic<uint64_t> g_wait_limit_ns{kDefaultWaitNs};
std::atomic<uint32_t> g_stall{0};
}  // namespace

WaitTest wait_test() { return WaitTest{g_wait_limit_ns.load(), g_stall.load()}; }

int read_and_clear_faults() {
  unsigned a = 0, b = 0, c = 0;
  int rc = single_read_and_clear_fault(&a);
  if (rc) return rc;
  rc = batch_read_and_clear_fault(&b);
  if (rc) return rc;
  rc = ws_read_and_clear_fault(&c);
  if (rc) return rc;
  return (a | b | c) ? B64_ERR_TIMEOUT : B64_OK;
}

constexpr int kAllFlags = B64_FLAG_URL | B64_FLAG_NOPAD | B64_FLAG_STRICT_TAIL;
constexpr int kDecodeFlags = kAllFlags | B64_FLAG_SKIP_WS;

// Shared by the synchronous and host-buffer decodes: checks and enqueues.
int decode_enqueue(const char* src, size_t m, uint8_t* dst, b64_result* d_result,
                   cudaStream_t stream, int flags = 0) {
  if (flags & ~kDecodeFlags) {
    set_error("unknown flag bits 0x%x", flags & ~kDecodeFlags);
    return B64_ERR_ARG;
  }
  if (!d_result) {
    set_error("d_result is null");
    return B64_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(d_result) & 7u) {
    set_error("d_result must be 8-byte aligned");
    return B64_ERR_ARG;
  }
  const size_t cap = (size_t)decoded_cap_flags(m, (uint32_t)flags);
  if (m > 0 && !src) {
    set_error("src is null");
    return B64_ERR_ARG;
  }
  if (cap > 0 && !dst) {
    set_error("dst is null");
    return B64_ERR_ARG;
  }
  if (overlaps(src, m, dst, cap)) {
    set_error("src and dst overlap");
    return B64_ERR_ARG;
  }
  cudaError_t e = cudaMemsetAsync(d_result, 0xFF, sizeof(b64_result), stream);
  if (e != cudaSuccess) return cuda_status(e, "decode: clearing the result");
  if (flags & B64_FLAG_SKIP_WS) {
    if (m == 0) return decode_enqueue(src, m, dst, d_result, stream, flags & ~B64_FLAG_SKIP_WS);
    e = decode_ws_enqueue(reinterpret_cast<const uint8_t*>(src), m, dst, d_result,
                          (uint32_t)flags, stream);
    if (e != cudaSuccess) return cuda_status(e, "decode: whitespace launch");
    return B64_OK;
  }
  e = launch_decode(reinterpret_cast<const uint8_t*>(src), m, decode_body_end(m), dst, d_result,
                    stream, single_config(1, m), (uint32_t)flags);
  if (e != cudaSuccess) return cuda_status(e, "decode: launch");
  return B64_OK;
}

}  // namespace gb64

using namespace gb64;

extern "C" {

size_t b64_encoded_len(size_t n) {
  const size_t groups = n / 3 + (n % 3 != 0);
  if (groups > SIZE_MAX / 4) return SIZE_MAX;
  return 4 * groups;
}

size_t b64_decoded_cap(size_t m) { return 3 * (m / 4); }

size_t b64_encoded_len_ex(size_t n, int flags) {
  const size_t groups = n / 3 + (n % 3 != 0);
  if (groups > SIZE_MAX / 4) return SIZE_MAX;
  return (size_t)encoded_len_flags(n, (uint32_t)flags);
}

size_t b64_decoded_cap_ex(size_t m, int flags) { return (size_t)decoded_cap_flags(m, (uint32_t)flags); }

size_t b64_encode_ex(const uint8_t* src, size_t n, char* dst, int flags, gb64_stream_t stream) {
  clear_error();
  if (flags & ~kAllFlags) {
    set_error("unknown flag bits 0x%x", flags & ~kAllFlags);
    return SIZE_MAX;
  }
  if (n == 0) return 0;
  if (!src || !dst) {
    set_error("%s is null", src ? "dst" : "src");
    return SIZE_MAX;
  }
  const size_t m = b64_encoded_len_ex(n, flags);
  if (m == SIZE_MAX) {
    set_error("input length %zu overflows the output length", n);
    return SIZE_MAX;
  }
  if (overlaps(src, n, dst, m)) {
    set_error("src and dst overlap");
    return SIZE_MAX;
  }
  cudaError_t e = launch_encode(src, n, reinterpret_cast<uint8_t*>(dst),
                                reinterpret_cast<cudaStream_t>(stream), single_config(0, n),
                                (uint32_t)flags);
  if (e != cudaSuccess) {
    cuda_status(e, "encode: launch");
    return SIZE_MAX;
  }
  return m;
}

size_t b64_encode(const uint8_t* src, size_t n, char* dst, gb64_stream_t stream) {
  return b64_encode_ex(src, n, dst, 0, stream);
}

int b64_decode_async_ex(const char* src, size_t m, uint8_t* dst, b64_result* d_result, int flags,
                        gb64_stream_t stream) {
  clear_error();
  return decode_enqueue(src, m, dst, d_result, reinterpret_cast<cudaStream_t>(stream), flags);
}

int b64_decode_async(const char* src, size_t m, uint8_t* dst, b64_result* d_result,
                     gb64_stream_t stream) {
  clear_error();
  return decode_enqueue(src, m, dst, d_result, reinterpret_cast<cudaStream_t>(stream));
}

int b64_decode_ex(const char* src, size_t m, uint8_t* dst, size_t* outlen, size_t* first_bad,
                  int flags, gb64_stream_t stream) {
  clear_error();
  if (!outlen || !first_bad) {
    set_error("outlen and first_bad must not be null");
    return B64_ERR_ARG;
  }
  if (m == 0) {
    *outlen = 0;
    *first_bad = 0;
    return B64_OK;
  }
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return cuda_status(e, "decode: device query");
  DecodeScratch* sc = decode_scratch(di->device, &e);
  if (!sc) return cuda_status(e, "decode: result scratch");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = decode_enqueue(src, m, dst, sc->dev, s, flags);
  if (rc != B64_OK) return rc;
  e = cudaMemcpyAsync(sc->host, sc->dev, sizeof(b64_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e, "decode: reading the result");
  *outlen = (size_t)sc->host->outlen;
  *first_bad = (size_t)sc->host->first_bad;
  if (sc->host->status == B64_ERR_TIMEOUT) set_error("decode kernel timed out on a bounded wait");
  return sc->host->status;
}

int b64_decode(const char* src, size_t m, uint8_t* dst, size_t* outlen, size_t* first_bad,
               gb64_stream_t stream) {
  return b64_decode_ex(src, m, dst, outlen, first_bad, 0, stream);
}

const char* b64_status_str(int status) {
  switch (status) {
    case B64_OK: return "B64_OK";
    case B64_ERR_INVALID_CHAR: return "B64_ERR_INVALID_CHAR";
    case B64_ERR_BAD_LENGTH: return "B64_ERR_BAD_LENGTH";
    case B64_ERR_NONCANONICAL: return "B64_ERR_NONCANONICAL";
    case B64_ERR_ARG: return "B64_ERR_ARG";
    case B64_ERR_CUDA: return "B64_ERR_CUDA";
    case B64_ERR_NOMEM: return "B64_ERR_NOMEM";
    case B64_ERR_TIMEOUT: return "B64_ERR_TIMEOUT";
    default: return "B64_UNKNOWN_STATUS";
  }
}

const char* b64_last_error(void) { return t_error.c_str(); }

int b64_test_stall_copies(int stall, uint64_t wait_limit_ns) {
  clear_error();
  g_wait_limit_ns.store(wait_limit_ns ? wait_limit_ns : kDefaultWaitNs);
  g_stall.store(stall ? 1u : 0u);
  return B64_OK;
}

int b64_device_fault(void) {
  clear_error();
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e, "device fault query");
  return read_and_clear_faults();
}

int b64_release_scratch(void) {
  clear_error();
  const cudaError_t e = ws_release_scratch();
  if (e != cudaSuccess) return cuda_status(e, "releasing the whitespace scratch");
  return B64_OK;
}

}  // extern "C"
