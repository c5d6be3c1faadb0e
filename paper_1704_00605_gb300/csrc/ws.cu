// Decode with whitespace removal (Appendix B): space, line feed and carriage
// return are dropped before decoding, and the first bad index is reported in
// offsets of the original input.
//
//   1. k_ws_count:    per tile of kWsTile characters, the number kept.
//   2. k_ws_scan_*:   exclusive prefix of the tile counts (three phases);
//                     prefix[ntiles] is the compacted length m'.
//   3. k_ws_compact:  every CTA packs its tile's kept characters at its
//                     prefix (warp ballots/popc + a block scan of the
//                     per-thread counts) into a scratch buffer.
//   4. the single-buffer decode kernels, reading m' from device memory.
//   5. k_ws_map_result: maps first_bad from compacted to original offsets
//                     (binary search over the tile prefix, then a warp scan
//                     inside the tile); on success first_bad = m.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tuner.h"

namespace gb64 {
namespace {

constexpr int kWsThreads = 256;
constexpr int64_t kWsTile = kWsThreads * 16;  // characters per tile
constexpr int kScanThreads = 256;
constexpr int64_t kScanChunk = kScanThreads * 4;

__device__ __forceinline__ bool is_ws(uint32_t x) { return x == 0x20 || x == 0x0A || x == 0x0D; }

// Keep-mask (bit k = character k is not whitespace) of 16 characters.
__device__ __forceinline__ uint32_t keep_mask16(const uint8_t* p, int64_t avail) {
  uint32_t mask = 0;
  for (int k = 0; k < 16; ++k)
    if (k < avail && !is_ws(p[k])) mask |= 1u << k;
  return mask;
}

// The 16 characters a thread owns, as four words, plus their keep-mask.
__device__ __forceinline__ uint32_t load_unit(const uint8_t* src, int64_t m, int64_t at,
                                              uint4* w) {
  const int64_t avail = m - at;
  if (avail >= 16) {
    *w = load16_any(src + at, src, src + m);
    uint32_t mask = 0;
    const uint32_t ws[4] = {w->x, w->y, w->z, w->w};
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (!is_ws((ws[k >> 2] >> (8 * (k & 3))) & 0xFFu)) mask |= 1u << k;
    return mask;
  }
  uint32_t b[16];
  for (int k = 0; k < 16; ++k) b[k] = (k < avail) ? src[at + k] : 0u;
  *w = make_uint4(b[0] | b[1] << 8 | b[2] << 16 | b[3] << 24, b[4] | b[5] << 8 | b[6] << 16 | b[7] << 24,
                  b[8] | b[9] << 8 | b[10] << 16 | b[11] << 24,
                  b[12] | b[13] << 8 | b[14] << 16 | b[15] << 24);
  return avail > 0 ? keep_mask16(src + at, avail) : 0u;
}

// Block-wide exclusive scan of one int per thread (kWsThreads threads).
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_sums[kWsThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kWsThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < kWsThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  *total = warp_sums[kWsThreads / 32 - 1];
  const int r = (warp ? warp_sums[warp - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kWsThreads)
    k_ws_count(const uint8_t* __restrict__ src, int64_t m, int64_t* __restrict__ counts) {
  const int64_t at = blockIdx.x * kWsTile + 16 * (int64_t)threadIdx.x;
  uint4 w;
  const int c = __popc(load_unit(src, m, at, &w));
  int total;
  block_excl_scan(c, &total);
  if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Exclusive scan of n int64 values in place (three phases).
__global__ void __launch_bounds__(kScanThreads)
    k_ws_scan_local(int64_t* __restrict__ v, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t ws[kScanThreads / 32];
  const int64_t base = blockIdx.x * kScanChunk + 4 * (int64_t)threadIdx.x;
  int64_t x[4], s = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    x[i] = base + i < n ? v[base + i] : 0;
    s += x[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t t = lane < kScanThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = t;
  }
  __syncthreads();
  int64_t run = (warp ? ws[warp - 1] : 0) + inc - s;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (base + i < n) v[base + i] = run;
    run += x[i];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = ws[kScanThreads / 32 - 1];
}

__global__ void k_ws_scan_sums(int64_t* __restrict__ sums, int64_t nb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t i = 0; i < nb; ++i) {
    const int64_t t = sums[i];
    sums[i] = run;
    run += t;
  }
  sums[nb] = run;
}

__global__ void k_ws_scan_add(int64_t* __restrict__ v, int64_t n, const int64_t* __restrict__ sums,
                              int64_t nb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] += sums[i / kScanChunk];
  if (i == 0) v[n] = sums[nb];
}

__global__ void __launch_bounds__(kWsThreads)
    k_ws_compact(const uint8_t* __restrict__ src, int64_t m, const int64_t* __restrict__ prefix,
                 uint8_t* __restrict__ out) {
  const int64_t at = blockIdx.x * kWsTile + 16 * (int64_t)threadIdx.x;
  uint4 w;
  const uint32_t mask = load_unit(src, m, at, &w);
  int total;
  int64_t o = prefix[blockIdx.x] + block_excl_scan(__popc(mask), &total);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int k = 0; k < 16; ++k)
    if (mask & (1u << k)) out[o++] = (uint8_t)(ws[k >> 2] >> (8 * (k & 3)));
}

// Original index of compacted character k (k < prefix[ntiles]).
__device__ int64_t original_index(const uint8_t* src, int64_t m, const int64_t* prefix,
                                  int64_t ntiles, int64_t k) {
  int64_t lo = 0, hi = ntiles;  // prefix[lo] <= k < prefix[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (prefix[mid] <= k) lo = mid; else hi = mid;
  }
  int64_t left = k - prefix[lo];
  const int64_t end = tmin<int64_t>(m, (lo + 1) * kWsTile);
  for (int64_t i = lo * kWsTile; i < end; ++i)
    if (!is_ws(src[i]) && left-- == 0) return i;
  return m;  // not reached for a valid k
}

__global__ void k_ws_map_result(b64_result* res, const uint8_t* __restrict__ src, int64_t m,
                                const int64_t* __restrict__ prefix, int64_t ntiles) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (res->status == B64_OK) {
    res->first_bad = m;
  } else if (res->status > 0 && res->first_bad < prefix[ntiles]) {
    res->first_bad = original_index(src, m, prefix, ntiles, res->first_bad);
  } else if (res->status > 0) {
    res->first_bad = m;
  }
}

}  // namespace

cudaError_t launch_decode_devlen(const uint8_t* src, uint64_t m_max, const uint64_t* m_dev,
                                 uint8_t* dst, b64_result* res, cudaStream_t stream,
                                 const TileConfig& cfg, uint32_t flags);

size_t ws_scratch_bytes(uint64_t m) {
  const int64_t ntiles = std::max<int64_t>(1, ((int64_t)m + kWsTile - 1) / kWsTile);
  const int64_t nb = (ntiles + kScanChunk - 1) / kScanChunk;
  return ((m + 255) & ~255ull) + (size_t)(ntiles + 1) * 8 + (size_t)(nb + 1) * 8;
}

// Enqueues the whitespace-removing decode; *d_result has been cleared.
cudaError_t decode_ws_launch(const uint8_t* src, uint64_t m, uint8_t* dst, b64_result* d_result,
                             void* scratch, uint32_t flags, cudaStream_t stream) {
  const int64_t ntiles = std::max<int64_t>(1, ((int64_t)m + kWsTile - 1) / kWsTile);
  const int64_t nb = (ntiles + kScanChunk - 1) / kScanChunk;
  uint8_t* packed = static_cast<uint8_t*>(scratch);
  int64_t* prefix = reinterpret_cast<int64_t*>(packed + ((m + 255) & ~255ull));
  int64_t* sums = prefix + ntiles + 1;
  k_ws_count<<<(unsigned)ntiles, kWsThreads, 0, stream>>>(src, (int64_t)m, prefix);
  k_ws_scan_local<<<(unsigned)nb, kScanThreads, 0, stream>>>(prefix, ntiles, sums);
  k_ws_scan_sums<<<1, 32, 0, stream>>>(sums, nb);
  k_ws_scan_add<<<(unsigned)((ntiles + 255) / 256), 256, 0, stream>>>(prefix, ntiles, sums, nb);
  k_ws_compact<<<(unsigned)ntiles, kWsThreads, 0, stream>>>(src, (int64_t)m, prefix, packed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_decode_devlen(packed, m, reinterpret_cast<const uint64_t*>(prefix + ntiles), dst,
                           d_result, stream, single_config(1, m), flags & ~(uint32_t)B64_FLAG_SKIP_WS);
  if (e != cudaSuccess) return e;
  k_ws_map_result<<<1, 32, 0, stream>>>(d_result, src, (int64_t)m, prefix, ntiles);
  return cudaGetLastError();
}

}  // namespace gb64
