// Batched encode and decode of many packed messages in one kernel per
// direction.
//
//   1. k_scan_local / k_scan_parts / k_scan_add: a device prefix sum over the
//      messages of (output length, tile count). Output length is
//      4 * ceil(n / 3) (encode) or 3 * floor(m / 4) (decode capacity); the
//      tile count is ceil(length / tile). The exclusive sums become out_off
//      (returned to the caller) and tile_off (scratch).
//   2. k_batch_encode / k_batch_decode: a persistent grid; CTA b owns the
//      contiguous tile range [b*T/G, (b+1)*T/G) of the T tiles, finds the
//      owning message of its first tile by binary search in tile_off and
//      advances through the following messages by a forward scan. Every tile
//      is coded with the unit codecs of common.cuh; per-message padding
//      (encode) and final quad, error index and length rule (decode) are
//      handled in the tile that holds the message end.
//   3. k_batch_decode_finish: per-message status, first_bad and outlen.
// All launches have fixed shapes, so a call can be captured in a CUDA graph.
#include <algorithm>

#include "batch.h"
#include "common.cuh"
#include "internal.h"

namespace gb64 {

static __device__ unsigned int g_batch_fault;

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int64_t kScanPerBlock = (int64_t)kScanThreads * kScanItems;
constexpr int64_t kNoBad = INT64_MAX;

// ----------------------------------------------------------------- scan
__device__ __forceinline__ void msg_values(int decode, int64_t len, int64_t tile, uint32_t flags,
                                           int64_t& outv, int64_t& tiles) {
  if (len < 0) len = 0;
  outv = decode ? (int64_t)decoded_cap_flags((uint64_t)len, flags)
                : (int64_t)encoded_len_flags((uint64_t)len, flags);
  tiles = (len + tile - 1) / tile;
}

// Block-wide exclusive scan of a pair of int64 values; returns the block total.
__device__ __forceinline__ void block_exclusive_scan2(int64_t& a, int64_t& b, int64_t& tot_a,
                                                      int64_t& tot_b) {
  __shared__ int64_t wa[kScanThreads / 32], wb[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t ia = a, ib = b;  // inclusive within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t xa = __shfl_up_sync(0xFFFFFFFFu, ia, d);
    const int64_t xb = __shfl_up_sync(0xFFFFFFFFu, ib, d);
    if (lane >= d) {
      ia += xa;
      ib += xb;
    }
  }
  if (lane == 31) {
    wa[warp] = ia;
    wb[warp] = ib;
  }
  __syncthreads();
  if (warp == 0) {
    int64_t sa = lane < kScanThreads / 32 ? wa[lane] : 0;
    int64_t sb = lane < kScanThreads / 32 ? wb[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t xa = __shfl_up_sync(0xFFFFFFFFu, sa, d);
      const int64_t xb = __shfl_up_sync(0xFFFFFFFFu, sb, d);
      if (lane >= d) {
        sa += xa;
        sb += xb;
      }
    }
    if (lane < kScanThreads / 32) {
      wa[lane] = sa;  // inclusive over warps
      wb[lane] = sb;
    }
  }
  __syncthreads();
  const int64_t pa = warp ? wa[warp - 1] : 0, pb = warp ? wb[warp - 1] : 0;
  tot_a = wa[kScanThreads / 32 - 1];
  tot_b = wb[kScanThreads / 32 - 1];
  a = pa + ia - a;
  b = pb + ib - b;
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_local(const int64_t* __restrict__ in_off, int64_t nmsg, int decode, int64_t tile,
                 uint32_t flags, int64_t* __restrict__ out_off, int64_t* __restrict__ tile_off,
                 int64_t* __restrict__ part_out, int64_t* __restrict__ part_tiles) {
  const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)threadIdx.x * kScanItems;
  int64_t vo[kScanItems], vt[kScanItems];
  int64_t so = 0, st = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    vo[i] = vt[i] = 0;
    if (j < nmsg) msg_values(decode, in_off[j + 1] - in_off[j], tile, flags, vo[i], vt[i]);
    so += vo[i];
    st += vt[i];
  }
  int64_t eo = so, et = st, to, tt;
  block_exclusive_scan2(eo, et, to, tt);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    eo += vo[i];
    et += vt[i];
    if (j < nmsg) {
      out_off[j + 1] = eo;  // inclusive within the block; k_scan_add adds the block base
      tile_off[j + 1] = et;
    }
  }
  if (threadIdx.x == 0) {
    part_out[blockIdx.x] = to;
    part_tiles[blockIdx.x] = tt;
  }
}

// One CTA: exclusive scan of the block totals, in place.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_parts(int64_t* __restrict__ part_out, int64_t* __restrict__ part_tiles, int64_t nparts) {
  __shared__ int64_t carry_o, carry_t;
  if (threadIdx.x == 0) carry_o = carry_t = 0;
  __syncthreads();
  for (int64_t c = 0; c < nparts; c += kScanThreads) {
    const int64_t i = c + threadIdx.x;
    int64_t a = i < nparts ? part_out[i] : 0, b = i < nparts ? part_tiles[i] : 0;
    int64_t ta, tb;
    block_exclusive_scan2(a, b, ta, tb);
    if (i < nparts) {
      part_out[i] = a + carry_o;
      part_tiles[i] = b + carry_t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_o += ta;
      carry_t += tb;
    }
    __syncthreads();
  }
}

__global__ void k_scan_add(int64_t nmsg, int64_t* __restrict__ out_off,
                           int64_t* __restrict__ tile_off, const int64_t* __restrict__ part_out,
                           const int64_t* __restrict__ part_tiles, int64_t* __restrict__ first_bad,
                           int64_t* __restrict__ outlen) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {
    out_off[0] = 0;
    tile_off[0] = 0;
  }
  if (j >= nmsg) return;
  const int64_t p = j / kScanPerBlock;
  out_off[j + 1] += part_out[p];
  tile_off[j + 1] += part_tiles[p];
  if (first_bad) first_bad[j] = kNoBad;
  if (outlen) outlen[j] = 0;
}

// ------------------------------------------------------------ tile walk
// Largest j in [0, nmsg) with tile_off[j] <= t (tile_off non-decreasing).
__device__ __forceinline__ int64_t owner_of(const int64_t* tile_off, int64_t nmsg, int64_t t) {
  int64_t lo = 0, hi = nmsg;  // invariant: tile_off[lo] <= t < tile_off[hi]
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (__ldg(tile_off + mid) <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// One message as a tile sees it: its bytes, its output, and the bounds that
// aligned-word reads near its ends must stay within.
struct Msg {
  const uint8_t* src;
  int64_t len;
  uint8_t* out;
  const uint8_t* lo;
  const uint8_t* hi;
};

// Messages packed back to back in one buffer (the batched C ABI).
struct PackedMsgs {
  const uint8_t* src;
  const int64_t* in_off;
  uint8_t* dst;
  const int64_t* out_off;
  const uint8_t* src_hi;
  __device__ __forceinline__ Msg get(int64_t j) const {
    const int64_t m0 = __ldg(in_off + j);
    return Msg{src + m0, __ldg(in_off + j + 1) - m0, dst + __ldg(out_off + j), src, src_hi};
  }
  __device__ __forceinline__ int64_t len(int64_t j) const {
    return __ldg(in_off + j + 1) - __ldg(in_off + j);
  }
  __device__ __forceinline__ void prepare(int64_t nmsg) { src_hi = src + __ldg(in_off + nmsg); }
};

// Messages anywhere in device memory, one descriptor each (the server).
struct DescMsgs {
  const MsgDesc* desc;
  uint8_t* dst;
  __device__ __forceinline__ Msg get(int64_t j) const {
    const MsgDesc d = desc[j];
    return Msg{d.src, d.len, dst + d.out_off, d.src, d.src + d.len};
  }
  __device__ __forceinline__ int64_t len(int64_t j) const { return desc[j].len; }
  __device__ __forceinline__ void prepare(int64_t) {}
};

// Encodes tile [t0, t0 + tile) of message m (Algorithm 1 per unit; the
// message's last tile also codes the partial group with its padding).
template <int NT>
__device__ __forceinline__ void encode_tile(const Msg& m, int64_t t0, int64_t tile,
                                            const uint8_t* T, uint32_t flags) {
  const uint32_t tid = threadIdx.x;
  const uint32_t len = (uint32_t)tmin<int64_t>(tile, m.len - t0);
  const uint8_t* sp = m.src + t0;
  uint8_t* dp = m.out + t0 / 3 * 4;
  const uint32_t nu = len / 12;
#pragma unroll 2
  for (uint32_t u = tid; u < nu; u += NT) {
    const uint3 w = load12_any(sp + 12 * u, m.lo, m.hi);
    store16_any(dp + 16 * u, enc_unit(w.x, w.y, w.z, T));
  }
  const uint32_t rest = len - 12 * nu;
  const uint32_t ng = (rest + 2) / 3;
  if (tid < ng) {
    const uint8_t* p = sp + 12 * nu + 3 * tid;
    const uint32_t cnt = min(3u, rest - 3 * tid);
    const uint32_t b0 = p[0], b1 = cnt > 1 ? p[1] : 0u, b2 = cnt > 2 ? p[2] : 0u;
    store_tail_group(dp + 16 * nu + 4 * tid, enc_tail_group(b0, b1, b2, cnt, T), cnt, flags);
  }
}

// Decodes tile [t0, t0 + tile) of message m (Algorithm 2 per unit; the tile
// holding the message end also checks the final characters). Every thread
// of the CTA must call it (warp-wide error reduction).
template <int NT>
__device__ __forceinline__ void decode_tile(const Msg& m, uint64_t t0, int64_t tile,
                                            const uint8_t* D, unsigned long long* fb,
                                            int64_t* outlen_j, uint32_t flags) {
  const uint32_t tid = threadIdx.x;
  const uint64_t mlen = (uint64_t)m.len;
  const uint64_t body_end = decode_body_end(mlen);
  const uint32_t len = (uint32_t)tmin<uint64_t>(tile, mlen - t0);
  const uint32_t body = body_end > t0 ? (uint32_t)tmin<uint64_t>(len, body_end - t0) : 0u;
  const uint32_t nu = body / 16;
  unsigned long long bad = ~0ull;
  const uint32_t lane = tid & 31u;
  for (uint32_t base = 0; base < nu; base += NT) {
    // the lanes of a warp own consecutive units, so they store together
    const uint32_t u = base + tid;
    uint3 o = make_uint3(0, 0, 0);
    if (u < nu) {
      const uint4 w = load16_any(m.src + t0 + 16 * u, m.lo, m.hi);
      uint32_t err = 0;
      o = dec_unit(w, D, err);
      if ((err & kBadFlag) && bad == ~0ull) bad = t0 + 16 * u + dec_unit_first_bad(w, D);
    }
    const uint32_t u0 = base + (tid & ~31u);
    if (u0 < nu) store12_warp(m.out + t0 / 4 * 3 + 12 * u0, o, lane, min(32u, nu - u0));
  }
  warp_min_to(fb, bad);
  const uint32_t nq = (body - 16 * nu) / 4;
  if (tid < nq) {
    const uint64_t idx = t0 + 16 * nu + 4 * tid;
    const uint8_t* p = m.src + idx;
    const uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                       ((uint32_t)p[3] << 24);
    uint32_t err = 0;
    const uint32_t v = dec_quad(x, D, err);
    if (err & kBadFlag) {
      for (uint32_t q = 0; q < 4; ++q)
        if (D[(x >> (8 * q)) & 0xFFu] & kBadFlag) {
          atomicMin(fb, (unsigned long long)(idx + q));
          break;
        }
    } else {
      uint8_t* o = m.out + idx / 4 * 3;
      o[0] = (uint8_t)(v >> 16);
      o[1] = (uint8_t)(v >> 8);
      o[2] = (uint8_t)v;
    }
  }
  if (tid == NT - 1 && body_end >= t0 && body_end < t0 + len)
    *outlen_j = dec_final_group(m.src, mlen, body_end, m.out, D, fb, flags);
}

// Persistent tile walk: CTA b owns tiles [b*T/G, (b+1)*T/G) of the
// T = tile_off[nmsg] tiles, in order.
template <int NT, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_encode(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ tile_off, int64_t tile,
                   uint32_t flags) {
  __shared__ uint8_t T[64];
  init_tables(T, nullptr, flags & kFlagUrl);
  const int64_t total = tile_off[nmsg];
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  int64_t t = (int64_t)blockIdx.x * per;
  const int64_t t_end = min(total, t + per);
  if (t >= t_end) return;
  Msgs ms = msgs;
  ms.prepare(nmsg);
  int64_t j = owner_of(tile_off, nmsg, t);
  for (; t < t_end; ++t) {
    while (__ldg(tile_off + j + 1) <= t) ++j;
    encode_tile<NT>(ms.get(j), (t - __ldg(tile_off + j)) * tile, tile, T, flags);
  }
}

template <int NT, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_decode(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ tile_off, int64_t tile,
                   int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen,
                   uint32_t flags) {
  __shared__ uint8_t D[256];
  init_tables(nullptr, D, flags & kFlagUrl);
  const int64_t total = tile_off[nmsg];
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  int64_t t = (int64_t)blockIdx.x * per;
  const int64_t t_end = min(total, t + per);
  if (t >= t_end) return;
  Msgs ms = msgs;
  ms.prepare(nmsg);
  int64_t j = owner_of(tile_off, nmsg, t);
  for (; t < t_end; ++t) {
    while (__ldg(tile_off + j + 1) <= t) ++j;
    decode_tile<NT>(ms.get(j), (uint64_t)(t - __ldg(tile_off + j)) * tile, tile, D,
                    reinterpret_cast<unsigned long long*>(first_bad + j), outlen + j, flags);
  }
}

// Per-message status: first bad character wins, then the length rule, then
// Appendix A's check (decoder of the final group returned a negative code).
template <class Msgs>
__global__ void k_batch_decode_finish(Msgs msgs, int64_t nmsg, int32_t* __restrict__ status,
                                      int64_t* __restrict__ first_bad,
                                      int64_t* __restrict__ outlen, uint32_t flags) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nmsg) return;
  const uint64_t m = (uint64_t)max((long long)0, (long long)msgs.len(j));
  const uint64_t body_end = decode_body_end(m);
  const int64_t final = (body_end < m) ? outlen[j] : 0;
  const FinalStatus f = final_status(m, body_end, (unsigned long long)first_bad[j], final, flags);
  status[j] = f.status;
  first_bad[j] = f.first_bad;
  outlen[j] = f.outlen;
}

// Initial per-message decode results for descriptor batches.
__global__ void k_batch_decode_init(int64_t nmsg, int64_t* __restrict__ first_bad,
                                    int64_t* __restrict__ outlen) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nmsg) return;
  first_bad[j] = kNoBad;
  outlen[j] = 0;
}

// ------------------------------------------------------------------ host
size_t batch_scratch_bytes(int64_t nmsg) {
  const int64_t nparts = (nmsg + kScanPerBlock - 1) / kScanPerBlock;
  return (size_t)(nmsg + 1) * 8 + (size_t)std::max<int64_t>(nparts, 1) * 16;
}

cudaError_t batch_offsets(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                          int64_t* tile_off, int64_t tile, void* scratch_parts,
                          int64_t* first_bad, int64_t* outlen, cudaStream_t stream,
                          uint32_t flags) {
  const int64_t nparts = (nmsg + kScanPerBlock - 1) / kScanPerBlock;
  int64_t* part_out = static_cast<int64_t*>(scratch_parts);
  int64_t* part_tiles = part_out + std::max<int64_t>(nparts, 1);
  if (nparts > 0) {
    k_scan_local<<<(unsigned)nparts, kScanThreads, 0, stream>>>(in_off, nmsg, decode, tile, flags,
                                                                out_off, tile_off, part_out,
                                                                part_tiles);
    k_scan_parts<<<1, kScanThreads, 0, stream>>>(part_out, part_tiles, nparts);
  }
  const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
  k_scan_add<<<(unsigned)blocks, 256, 0, stream>>>(nmsg, out_off, tile_off, part_out, part_tiles,
                                                   first_bad, outlen);
  return cudaGetLastError();
}

namespace {
template <int NT, class Msgs>
cudaError_t launch_work(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* tile_off,
                        int32_t* status, int64_t* first_bad, int64_t* outlen,
                        const BatchConfig& cfg, const DeviceInfo* di, uint32_t flags,
                        cudaStream_t stream) {
  const int grid = di->sm_count * cfg.blocks_per_sm;
  if (!decode) {
    k_batch_encode<NT, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, tile_off, cfg.tile, flags);
    return cudaGetLastError();
  }
  k_batch_decode<NT, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, tile_off, cfg.tile, first_bad,
                                                    outlen, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
  k_batch_decode_finish<Msgs><<<(unsigned)blocks, 256, 0, stream>>>(msgs, nmsg, status, first_bad,
                                                                   outlen, flags);
  return cudaGetLastError();
}

template <class Msgs>
cudaError_t launch_work_any(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* tile_off,
                            int32_t* status, int64_t* first_bad, int64_t* outlen,
                            const BatchConfig& cfg, uint32_t flags, cudaStream_t stream) {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  switch (cfg.threads) {
    case 128:
      return launch_work<128>(decode, msgs, nmsg, tile_off, status, first_bad, outlen, cfg, di,
                              flags, stream);
    case 512:
      return launch_work<512>(decode, msgs, nmsg, tile_off, status, first_bad, outlen, cfg, di,
                              flags, stream);
    default:
      return launch_work<256>(decode, msgs, nmsg, tile_off, status, first_bad, outlen, cfg, di,
                              flags, stream);
  }
}
}  // namespace

cudaError_t batch_launch_desc(int decode, const MsgDesc* desc, int64_t nmsg, uint8_t* dst,
                              const int64_t* tile_off, int32_t* status, int64_t* first_bad,
                              int64_t* outlen, const BatchConfig& cfg, bool init_results,
                              cudaStream_t stream, uint32_t flags) {
  if (decode && init_results) {
    const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
    k_batch_decode_init<<<(unsigned)blocks, 256, 0, stream>>>(nmsg, first_bad, outlen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_work_any(decode, DescMsgs{desc, dst}, nmsg, tile_off, status, first_bad, outlen,
                         cfg, flags, stream);
}

cudaError_t batch_launch(const BatchArgs& a, const BatchConfig& cfg) {
  cudaError_t e = batch_offsets(a.decode, a.in_off, a.nmsg, a.out_off, a.tile_off, cfg.tile,
                                a.parts, a.decode ? a.first_bad : nullptr,
                                a.decode ? a.outlen : nullptr, a.stream, a.flags);
  if (e != cudaSuccess) return e;
  // src_hi (the end of the packed input, in_off[nmsg]) is read on the device
  PackedMsgs msgs{a.src, a.in_off, a.dst, a.out_off, nullptr};
  return launch_work_any(a.decode, msgs, a.nmsg, a.tile_off, a.status, a.first_bad, a.outlen, cfg,
                         a.flags, a.stream);
}

int batch_read_and_clear_fault(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_batch_fault, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_batch_fault, &zero, sizeof(zero));
  *out = v;
  return e == cudaSuccess ? 0 : cuda_status(e, "reading the fault word");
}

}  // namespace gb64
