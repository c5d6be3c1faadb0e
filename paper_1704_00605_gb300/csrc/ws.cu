// Decode with whitespace removal (Appendix B): space, line feed and carriage
// return are dropped before decoding, and the first bad index is reported in
// offsets of the original input.
//
//   1. k_ws_count:    per tile of kWsTile characters (64 per thread), the
//                     number kept; whitespace is found four bytes at a time.
//   2. k_ws_scan_*:   exclusive prefix of the tile counts (three phases);
//                     prefix[ntiles] is the compacted length m'.
//   3. k_ws_compact:  every CTA packs its tile's kept characters at its
//                     prefix (a block scan of the per-thread counts) in
//                     shared memory and writes them to a scratch buffer with
//                     one bulk store.
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
constexpr int kWsPerThread = 64;                          // characters per thread
constexpr int64_t kWsTile = kWsThreads * kWsPerThread;  // characters per tile
constexpr int kScanThreads = 256;
constexpr int64_t kScanChunk = kScanThreads * 4;

// High bit of every byte of x that is zero (exact, no carries between bytes).
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
  return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);
}

// Keep bits (bit k = byte k of w is not space, line feed or carriage return).
__device__ __forceinline__ uint32_t keep4(uint32_t w) {
  const uint32_t ws = zero_bytes(w ^ 0x20202020u) | zero_bytes(w ^ 0x0A0A0A0Au) |
                      zero_bytes(w ^ 0x0D0D0D0Du);
  const uint32_t keep = ~ws & 0x80808080u;
  return ((keep >> 7) * 0x10204080u) >> 28;  // bits 7, 15, 23, 31 -> bits 0..3
}

// The 64 characters [at, at + 64) a thread owns, as 16 words (characters
// past m read as space), and their keep-mask (bit k = character k kept).
__device__ __forceinline__ uint64_t load_chars(const uint8_t* src, int64_t m, int64_t at,
                                               uint32_t* w) {
  if (m - at >= kWsPerThread) {
    uint4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = load16_any(src + at + 16 * i, src, src + m);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[4 * i] = v[i].x;
      w[4 * i + 1] = v[i].y;
      w[4 * i + 2] = v[i].z;
      w[4 * i + 3] = v[i].w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      uint32_t x = 0;
      for (int k = 0; k < 4; ++k) {
        const int64_t q = at + 4 * i + k;
        x |= (q < m ? (uint32_t)src[q] : 0x20u) << (8 * k);
      }
      w[i] = x;
    }
  }
  uint64_t mask = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) mask |= (uint64_t)keep4(w[i]) << (4 * i);
  return mask;
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
  const int64_t at = blockIdx.x * kWsTile + (int64_t)kWsPerThread * threadIdx.x;
  uint32_t w[16];
  const int c = __popcll(load_chars(src, m, at, w));
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

// Packs the tile's kept characters in shared memory at the output's phase
// (shared position o2 + i holds output byte i, o2 = the output address mod
// 16), then writes them out: the aligned interior by one bulk store, the
// ragged ends (at most 15 bytes each) by byte stores.
__global__ void __launch_bounds__(kWsThreads)
    k_ws_compact(const uint8_t* __restrict__ src, int64_t m, const int64_t* __restrict__ prefix,
                 uint8_t* __restrict__ out) {
  __shared__ __align__(16) uint8_t buf[kWsTile + 32];
  // byte_perm selectors moving the kept bytes of a word (keep bits k4) to
  // its low end, in order
  __shared__ uint16_t sel[16];
  if (threadIdx.x < 16) {
    uint32_t v = 0, r = 0;
    for (uint32_t k = 0; k < 4; ++k)
      if (threadIdx.x & (1u << k)) v |= k << (4 * r++);
    sel[threadIdx.x] = (uint16_t)v;
  }
  const int64_t at = blockIdx.x * kWsTile + (int64_t)kWsPerThread * threadIdx.x;
  uint32_t w[16];
  const uint64_t mask = load_chars(src, m, at, w);
  int total;
  const int local = block_excl_scan(__popcll(mask), &total);  // also orders sel
  uint8_t* d = out + prefix[blockIdx.x];
  const uintptr_t da = reinterpret_cast<uintptr_t>(d);
  const uint32_t o2 = (uint32_t)(da & 15u);
  uint32_t p = o2 + (uint32_t)local;
  // branch-free, so that the lanes of a warp never split over a word with
  // whitespace: the word's kept bytes moved down by one byte_perm, then
  // stored under predicates
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t k4 = (uint32_t)(mask >> (4 * i)) & 15u;
    const uint32_t v = __byte_perm(w[i], 0u, sel[k4]);
    const uint32_t n = __popc(k4);
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (k < n) buf[p + k] = (uint8_t)(v >> (8 * k));
    p += n;
  }
  fence_proxy_async_smem();
  __syncthreads();
  const uint32_t olen = (uint32_t)total;
  const uintptr_t lo = (da + 15u) & ~(uintptr_t)15u, hi = (da + olen) & ~(uintptr_t)15u;
  if (threadIdx.x == 0 && hi > lo) {
    tma_store_1d(reinterpret_cast<void*>(lo), buf + (o2 ? 16u : 0u), (uint32_t)(hi - lo));
    bulk_commit();
  }
  const uint32_t head = (uint32_t)(tmin<uintptr_t>(lo, da + olen) - da);
  const uint32_t ie = hi > lo ? (uint32_t)(hi - da) : head;
  const uint32_t t = threadIdx.x;
  if (t < head) {
    d[t] = buf[o2 + t];
  } else if (t >= 32u && t - 32u < olen - ie) {
    d[ie + t - 32u] = buf[o2 + ie + t - 32u];
  }
  if (threadIdx.x == 0) bulk_wait_all();  // the CTA's shared memory outlives the copy
}

__device__ __forceinline__ bool is_ws(uint32_t x) { return x == 0x20 || x == 0x0A || x == 0x0D; }

// Original index of compacted character k (k < prefix[ntiles]), by one
// warp: the tile holding it (binary search of the tile prefix), then the
// kept characters of each lane's 1/32 of the tile counted and prefixed, then
// one lane's scan of its part.
__device__ int64_t original_index(const uint8_t* src, int64_t m, const int64_t* prefix,
                                  int64_t ntiles, int64_t k, uint32_t lane) {
  int64_t lo = 0, hi = ntiles;  // prefix[lo] <= k < prefix[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (prefix[mid] <= k) lo = mid; else hi = mid;
  }
  const int64_t part = kWsTile / 32;
  const int64_t b = lo * kWsTile + lane * part, e = tmin<int64_t>(m, b + part);
  int c = 0;
  for (int64_t i = b; i < e; ++i) c += !is_ws(src[i]);
  int incl = c;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if ((int)lane >= d) incl += y;
  }
  const int64_t left = k - prefix[lo];  // kept characters of the tile before k
  const bool mine = left >= incl - c && left < incl;
  int64_t r = m;
  if (mine) {
    int64_t n = left - (incl - c);
    for (int64_t i = b; i < e; ++i)
      if (!is_ws(src[i]) && n-- == 0) {
        r = i;
        break;
      }
  }
  const uint32_t who = __ballot_sync(0xFFFFFFFFu, mine);
  return who ? __shfl_sync(0xFFFFFFFFu, r, __ffs(who) - 1) : m;
}

__global__ void k_ws_map_result(b64_result* res, const uint8_t* __restrict__ src, int64_t m,
                                const int64_t* __restrict__ prefix, int64_t ntiles) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const uint32_t lane = threadIdx.x;
  const int32_t status = res->status;
  const int64_t fb = res->first_bad;
  int64_t out = m;
  if (status > 0 && fb < prefix[ntiles]) out = original_index(src, m, prefix, ntiles, fb, lane);
  __syncwarp();
  if (lane == 0 && status >= 0) res->first_bad = out;
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
