// Internal interfaces between the translation units of libgb64 (not part of
// the public C ABI, which is include/gb64.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gb64.h"
#include "rules.h"

namespace gb64 {

// Records the calling thread's last error text (read by b64_last_error).
void set_error(const char* fmt, ...);
void clear_error();

// Maps a CUDA failure to B64_ERR_CUDA (or B64_ERR_NOMEM) and records it.
int cuda_status(cudaError_t e, const char* what);

// Per-device facts used to size grids (cached; current device).
struct DeviceInfo {
  int device = -1;
  int sm_count = 0;
  int max_smem_optin = 0;
  int cc_major = 0, cc_minor = 0;
};
const DeviceInfo* device_info(cudaError_t* err);

// Kernel shape of a pipelined single-buffer launch.
struct TileConfig {
  int threads;            // 128, 256 or 512
  int upt;                // units per thread per tile (encode unit 12 B, decode unit 16 chars)
  int stages;             // input stages in shared memory (2..8)
  int blocks_per_sm = 0;  // persistent CTAs per SM (0 = as many as fit)
};

// Default shapes for a buffer of n bytes / m characters (the tuner may pick
// others), and the dynamic shared memory a shape needs.
TileConfig default_encode_config(uint64_t n);
TileConfig default_decode_config(uint64_t m);
size_t single_smem_bytes(int decode, const TileConfig& c);

// Raises the kernel's dynamic shared-memory limit to the device maximum (once
// per device and kernel) and returns how many CTAs of `threads` threads and
// smem_bytes of dynamic shared memory fit per SM (cached). Fails with
// cudaErrorInvalidValue when smem_bytes does not fit the device.
cudaError_t kernel_prepare(const void* kernel, size_t smem_bytes, int threads, int* blocks_per_sm);

// Single-buffer encode of n >= 1 bytes; picks the TMA kernel when src and
// dst are 16-byte aligned, else the generic one.
cudaError_t launch_encode(const uint8_t* src, uint64_t n, uint8_t* dst, cudaStream_t stream,
                          const TileConfig& cfg, uint32_t flags = 0);

// Single-buffer decode of m characters. Characters [0, body_end) must be
// whole quads of the alphabet; [body_end, m) are the final characters
// (padding rules). The caller has set *res to all-ones bytes on stream.
cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint64_t body_end, uint8_t* dst,
                          b64_result* res, cudaStream_t stream, const TileConfig& cfg,
                          uint32_t flags = 0);

// Whitespace-removing decode (ws.cu): the launch into the device's kept
// scratch (or, under graph capture, a stream-ordered allocation), and the
// release of that scratch (waits for its last user).
cudaError_t decode_ws_enqueue(const uint8_t* src, uint64_t m, uint8_t* dst, b64_result* d_result,
                              uint32_t flags, cudaStream_t stream);
cudaError_t ws_release_scratch();

// Limit of the pipelined kernels' bounded waits and the test stall of
// b64_test_stall_copies (host state, passed to every launch).
struct WaitTest {
  uint64_t limit_ns;  // wait limit (default 2 s)
  uint32_t stall;     // leave out the first copy of the first CTA / warp
};
WaitTest wait_test();

// Reads and clears the fault words of every kernel file (current device).
int read_and_clear_faults();
int batch_read_and_clear_fault(unsigned int* out);
int single_read_and_clear_fault(unsigned int* out);
int ws_read_and_clear_fault(unsigned int* out);

}  // namespace gb64
