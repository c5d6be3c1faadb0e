// Host-buffer forms of encode and decode: the input is moved to the device
// in chunks and the output moved back, with the host-to-device copy of one
// chunk overlapping the kernel and device-to-host copy of the previous ones
// (kStreams internal streams in rotation, all ordered after the caller's
// stream). The link, not the kernels, bounds these calls. Chunks are cut at
// multiples of 48 input bytes (encode) or 64 characters (decode) so every
// chunk's device buffers stay 16-byte aligned and take the TMA kernels.
#include <algorithm>
#include <vector>

#include "internal.h"
#include "tuner.h"

namespace gb64 {

int decode_enqueue(const char* src, size_t m, uint8_t* dst, b64_result* d_result,
                   cudaStream_t stream);

namespace {

constexpr int kStreams = 3;
constexpr size_t kEncChunk = (size_t)24 << 20;  // input bytes per chunk (multiple of 48)
constexpr size_t kDecChunk = (size_t)32 << 20;  // characters per chunk (multiple of 64)

struct Pipe {
  bool ready = false;
  cudaStream_t st[kStreams] = {};
  cudaEvent_t start = nullptr;
  uint8_t* in[kStreams] = {};
  uint8_t* out[kStreams] = {};
  size_t in_cap = 0, out_cap = 0;
  b64_result* res = nullptr;  // per-chunk decode results (device)
  b64_result* res_host = nullptr;
  size_t res_cap = 0;
};

Pipe* pipe_for_device(int device, cudaError_t* err) {
  thread_local std::vector<Pipe> pipes;
  if ((int)pipes.size() <= device) pipes.resize(device + 1);
  Pipe& p = pipes[device];
  if (!p.ready) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kStreams && e == cudaSuccess; ++i)
      e = cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      *err = e;
      return nullptr;
    }
    p.ready = true;
  }
  return &p;
}

cudaError_t sync_all(Pipe& p) {
  cudaError_t first = cudaSuccess;
  for (int i = 0; i < kStreams; ++i) {
    const cudaError_t e = cudaStreamSynchronize(p.st[i]);
    if (first == cudaSuccess) first = e;
  }
  return first;
}

cudaError_t ensure_buffers(Pipe& p, size_t in_bytes, size_t out_bytes) {
  if (p.in_cap >= in_bytes && p.out_cap >= out_bytes) return cudaSuccess;
  cudaError_t e = sync_all(p);
  if (e != cudaSuccess) return e;
  // grow to the larger of the old and new needs, so that alternating
  // encode (48 MiB in, 64 MiB out) and decode (64 MiB in, 48 MiB out) calls
  // stop reallocating after the first of each
  const size_t ic = std::max(in_bytes, p.in_cap), oc = std::max(out_bytes, p.out_cap);
  for (int i = 0; i < kStreams; ++i) {
    cudaFree(p.in[i]);
    cudaFree(p.out[i]);
    p.in[i] = p.out[i] = nullptr;
  }
  p.in_cap = p.out_cap = 0;
  for (int i = 0; i < kStreams; ++i) {
    e = cudaMalloc(&p.in[i], ic);
    if (e == cudaSuccess) e = cudaMalloc(&p.out[i], oc);
    if (e != cudaSuccess) return e;
  }
  p.in_cap = ic;
  p.out_cap = oc;
  return cudaSuccess;
}

cudaError_t ensure_results(Pipe& p, size_t n) {
  if (p.res_cap >= n) return cudaSuccess;
  cudaError_t e = sync_all(p);
  if (e != cudaSuccess) return e;
  cudaFree(p.res);
  cudaFreeHost(p.res_host);
  p.res = nullptr;
  p.res_host = nullptr;
  p.res_cap = 0;
  const size_t cap = std::max<size_t>(n, 64);
  e = cudaMalloc(&p.res, cap * sizeof(b64_result));
  if (e == cudaSuccess) e = cudaMallocHost(&p.res_host, cap * sizeof(b64_result));
  if (e != cudaSuccess) return e;
  p.res_cap = cap;
  return cudaSuccess;
}

// Orders both pipe streams after the caller's stream.
cudaError_t join_caller(Pipe& p, cudaStream_t caller) {
  cudaError_t e = cudaEventRecord(p.start, caller);
  for (int i = 0; i < kStreams && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(p.st[i], p.start, 0);
  return e;
}

}  // namespace
}  // namespace gb64

using namespace gb64;

extern "C" {

size_t b64_encode_host(const uint8_t* h_src, size_t n, char* h_dst, gb64_stream_t stream) {
  clear_error();
  if (n == 0) return 0;
  if (!h_src || !h_dst) {
    set_error("%s is null", h_src ? "h_dst" : "h_src");
    return SIZE_MAX;
  }
  const size_t m = b64_encoded_len(n);
  if (m == SIZE_MAX) {
    set_error("input length overflows the output length");
    return SIZE_MAX;
  }
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  Pipe* p = di ? pipe_for_device(di->device, &e) : nullptr;
  if (!p) {
    cuda_status(e, "encode_host: setup");
    return SIZE_MAX;
  }
  const size_t chunk = std::min(kEncChunk, (n + 47) / 48 * 48);
  e = ensure_buffers(*p, chunk, chunk / 3 * 4);
  if (e == cudaSuccess) e = join_caller(*p, reinterpret_cast<cudaStream_t>(stream));
  for (size_t off = 0, i = 0; e == cudaSuccess && off < n; off += chunk, ++i) {
    const int b = (int)(i % kStreams);
    const size_t len = std::min(chunk, n - off);
    e = cudaMemcpyAsync(p->in[b], h_src + off, len, cudaMemcpyHostToDevice, p->st[b]);
    if (e == cudaSuccess) e = launch_encode(p->in[b], len, p->out[b], p->st[b], single_config(0, len));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_dst + off / 3 * 4, p->out[b], b64_encoded_len(len),
                          cudaMemcpyDeviceToHost, p->st[b]);
  }
  const cudaError_t es = sync_all(*p);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) {
    cuda_status(e, "encode_host");
    return SIZE_MAX;
  }
  return m;
}

int b64_decode_host(const char* h_src, size_t m, uint8_t* h_dst, size_t* outlen,
                    size_t* first_bad, gb64_stream_t stream) {
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
  if (!h_src || (b64_decoded_cap(m) > 0 && !h_dst)) {
    set_error("null host buffer");
    return B64_ERR_ARG;
  }
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  Pipe* p = di ? pipe_for_device(di->device, &e) : nullptr;
  if (!p) return cuda_status(e, "decode_host: setup");
  const size_t chunk = std::min(kDecChunk, (m + 63) / 64 * 64);
  const size_t nchunks = (m + chunk - 1) / chunk;
  e = ensure_buffers(*p, chunk, chunk / 4 * 3);
  if (e == cudaSuccess) e = ensure_results(*p, nchunks);
  if (e == cudaSuccess) e = join_caller(*p, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "decode_host: buffers");
  const uint64_t body_end = decode_body_end(m);
  for (size_t i = 0; i < nchunks; ++i) {
    const int b = (int)(i % kStreams);
    const size_t off = i * chunk;
    const size_t len = std::min(chunk, m - off);
    const bool last = (i + 1 == nchunks);
    e = cudaMemcpyAsync(p->in[b], h_src + off, len, cudaMemcpyHostToDevice, p->st[b]);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->res + i, 0xFF, sizeof(b64_result), p->st[b]);
    if (e == cudaSuccess)
      e = launch_decode(p->in[b], len, last ? body_end - off : len, p->out[b], p->res + i,
                        p->st[b], single_config(1, len));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_dst + off / 4 * 3, p->out[b], b64_decoded_cap(len),
                          cudaMemcpyDeviceToHost, p->st[b]);
    if (e != cudaSuccess) break;
  }
  const cudaError_t es = sync_all(*p);
  if (e == cudaSuccess) e = es;
  if (e == cudaSuccess)
    e = cudaMemcpy(p->res_host, p->res, nchunks * sizeof(b64_result), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "decode_host");
  size_t total = 0;
  for (size_t i = 0; i < nchunks; ++i) {
    const b64_result& r = p->res_host[i];
    if (r.status != B64_OK) {
      *outlen = 0;
      *first_bad = (r.status == B64_ERR_TIMEOUT) ? m : (size_t)r.first_bad + i * chunk;
      return r.status;
    }
    total += (size_t)r.outlen;
  }
  *outlen = total;
  *first_bad = m;
  return B64_OK;
}

}  // extern "C"
