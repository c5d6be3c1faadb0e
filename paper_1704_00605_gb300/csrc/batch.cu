// Batched encode and decode of many packed messages in one kernel per
// direction.
//
//   1. k_scan_local / k_scan_parts / k_scan_add: a device prefix sum over the
//      messages of (output length, tile count). Output length is
//      4 * ceil(n / 3) (encode) or 3 * floor(m / 4) (decode capacity); the
//      tile count is ceil(length / tile). The exclusive sums become out_off
//      (returned to the caller) and tile_off (scratch).
//   2. k_batch_code (encode or decode): a persistent grid in which every
//      warp owns a contiguous range of the T tiles, finds the owning message
//      of its first tile by binary search in tile_off and advances through
//      the following messages by a forward scan. Tiles reach shared memory
//      by bulk copies (TMA) several tiles ahead and are coded with the unit
//      codecs of common.cuh; outputs leave by bulk stores. Per-message
//      padding (encode) and final quad, error index and length rule
//      (decode) are handled in the tile that holds the message end.
//   3. k_batch_decode_finish: per-message status, first_bad and outlen.
// All launches have fixed shapes, so a call can be captured in a CUDA graph.
#include <algorithm>

#include "batch.h"
#include "common.cuh"
#include "internal.h"

namespace gb64 {

static __device__ unsigned int g_batch_fault;

constexpr int kMaxBatchStages = 6;

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int64_t kScanPerBlock = (int64_t)kScanThreads * kScanItems;
constexpr int64_t kNoBad = INT64_MAX;
constexpr int64_t kTileCost = kBatchTileCost;

// ----------------------------------------------------------------- scan
// Output length, tile count and weight of one message; messages of at most
// small_max bytes get no tiles (threads code them one each) and no weight.
// A message's weight, its length plus kTileCost per tile, is what the
// tile kernels divide evenly among their warps.
__device__ __forceinline__ void msg_values(int decode, int64_t len, int64_t tile, uint32_t flags,
                                           int64_t small_max, int64_t& outv, int64_t& tiles,
                                           int64_t& weight) {
  if (len < 0) len = 0;
  outv = decode ? (int64_t)decoded_cap_flags((uint64_t)len, flags)
                : (int64_t)encoded_len_flags((uint64_t)len, flags);
  tiles = len > small_max ? (len + tile - 1) / tile : 0;
  weight = tiles ? len + tiles * kTileCost : 0;
}

// Three int64 running sums (output, tiles, weight).
struct Sum3 {
  int64_t v[3];
};

__device__ __forceinline__ Sum3 shfl_up3(const Sum3& x, int d) {
  Sum3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i) r.v[i] = __shfl_up_sync(0xFFFFFFFFu, x.v[i], d);
  return r;
}

// Block-wide exclusive scan of x; tot receives the block total.
__device__ __forceinline__ void block_exclusive_scan3(Sum3& x, Sum3& tot) {
  __shared__ int64_t ws[3][kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Sum3 inc = x;  // inclusive within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const Sum3 y = shfl_up3(inc, d);
    if (lane >= d)
#pragma unroll
      for (int i = 0; i < 3; ++i) inc.v[i] += y.v[i];
  }
  if (lane == 31)
#pragma unroll
    for (int i = 0; i < 3; ++i) ws[i][warp] = inc.v[i];
  __syncthreads();
  if (warp == 0) {
    Sum3 w;
#pragma unroll
    for (int i = 0; i < 3; ++i) w.v[i] = lane < kScanThreads / 32 ? ws[i][lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const Sum3 y = shfl_up3(w, d);
      if (lane >= d)
#pragma unroll
        for (int i = 0; i < 3; ++i) w.v[i] += y.v[i];
    }
    if (lane < kScanThreads / 32)
#pragma unroll
      for (int i = 0; i < 3; ++i) ws[i][lane] = w.v[i];  // inclusive over warps
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int64_t before = warp ? ws[i][warp - 1] : 0;
    tot.v[i] = ws[i][kScanThreads / 32 - 1];
    x.v[i] = before + inc.v[i] - x.v[i];
  }
}

// The block totals: parts[i * nparts + p] for sum i of block p.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_local(const int64_t* __restrict__ in_off, int64_t nmsg, int decode, int64_t tile,
                 uint32_t flags, int64_t small_max, int64_t* __restrict__ out_off,
                 int64_t* __restrict__ tile_off, int64_t* __restrict__ weight_off,
                 int64_t* __restrict__ parts, int64_t nparts) {
  const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)threadIdx.x * kScanItems;
  Sum3 item[kScanItems];
  Sum3 sum = {{0, 0, 0}};
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t j = base + k;
    item[k] = Sum3{{0, 0, 0}};
    if (j < nmsg)
      msg_values(decode, in_off[j + 1] - in_off[j], tile, flags, small_max, item[k].v[0],
                 item[k].v[1], item[k].v[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) sum.v[i] += item[k].v[i];
  }
  Sum3 tot;
  block_exclusive_scan3(sum, tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t j = base + k;
#pragma unroll
    for (int i = 0; i < 3; ++i) sum.v[i] += item[k].v[i];
    if (j < nmsg) {  // inclusive within the block; k_scan_add adds the block base
      out_off[j + 1] = sum.v[0];
      tile_off[j + 1] = sum.v[1];
      weight_off[j + 1] = sum.v[2];
    }
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < 3; ++i) parts[i * nparts + blockIdx.x] = tot.v[i];
}

// One CTA: exclusive scan of the block totals, in place.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_parts(int64_t* __restrict__ parts, int64_t nparts) {
  __shared__ int64_t carry[3];
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t c = 0; c < nparts; c += kScanThreads) {
    const int64_t p = c + threadIdx.x;
    Sum3 x;
#pragma unroll
    for (int i = 0; i < 3; ++i) x.v[i] = p < nparts ? parts[i * nparts + p] : 0;
    Sum3 tot;
    block_exclusive_scan3(x, tot);
    if (p < nparts)
#pragma unroll
      for (int i = 0; i < 3; ++i) parts[i * nparts + p] = x.v[i] + carry[i];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < 3; ++i) carry[i] += tot.v[i];
    __syncthreads();
  }
}

__global__ void k_scan_add(int64_t nmsg, int64_t* __restrict__ out_off,
                           int64_t* __restrict__ tile_off, int64_t* __restrict__ weight_off,
                           const int64_t* __restrict__ parts, int64_t nparts,
                           int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {
    out_off[0] = 0;
    tile_off[0] = 0;
    weight_off[0] = 0;
  }
  if (j >= nmsg) return;
  const int64_t p = j / kScanPerBlock;
  out_off[j + 1] += parts[p];
  tile_off[j + 1] += parts[nparts + p];
  weight_off[j + 1] += parts[2 * nparts + p];
  if (first_bad) first_bad[j] = kNoBad;
  if (outlen) outlen[j] = 0;
}

// ------------------------------------------------------------ tile walk
// Largest j in [0, nmsg) with tile_off[j] <= t (tile_off non-decreasing,
// t < tile_off[nmsg]). The whole warp searches: each round its 32 lanes
// probe 32 evenly spaced offsets and the count of those <= t narrows the
// interval 33-fold (4 dependent loads for 10^5 messages, not 17).
__device__ __forceinline__ int64_t owner_of_warp(const int64_t* tile_off, int64_t nmsg, int64_t t,
                                                 uint32_t lane) {
  int64_t lo = 0, hi = nmsg;  // invariant: tile_off[lo] <= t < tile_off[hi]
  while (hi - lo > 1) {
    const int64_t span = hi - lo;
    // probes lo < p_0 <= p_1 <= ... <= p_31 < hi
    const int64_t p = lo + 1 + (span - 1) * (int64_t)lane / 32;
    const uint32_t le = __ballot_sync(0xFFFFFFFFu, __ldg(tile_off + p) <= t);
    const int c = __popc(le);  // the probes <= t are lanes [0, c)
    const int64_t below = __shfl_sync(0xFFFFFFFFu, p, c > 0 ? c - 1 : 0);
    const int64_t above = __shfl_sync(0xFFFFFFFFu, p, c < 32 ? c : 31);
    if (c > 0) lo = below;
    if (c < 32) hi = above;
  }
  return lo;
}

// The same search for two targets at once: lanes 0-15 find the owner of
// their x, lanes 16-31 of theirs (16 probes a round each).
__device__ __forceinline__ int64_t owner_of_halves(const int64_t* off, int64_t nmsg, int64_t x,
                                                   uint32_t lane) {
  const uint32_t h = lane >> 4, k = lane & 15u;
  int64_t lo = 0, hi = nmsg;  // invariant: off[lo] <= x < off[hi]
  while (__any_sync(0xFFFFFFFFu, hi - lo > 1)) {
    const int64_t span = hi - lo;
    // probes lo < p_0 <= ... <= p_15 < hi (p = hi <= nmsg once span is 1)
    const int64_t p = lo + 1 + (span - 1) * (int64_t)k / 16;
    const uint32_t le = __ballot_sync(0xFFFFFFFFu, __ldg(off + p) <= x);
    const int c = __popc((le >> (16u * h)) & 0xFFFFu);
    const int64_t below = __shfl_sync(0xFFFFFFFFu, p, (int)(16u * h) + (c > 0 ? c - 1 : 0));
    const int64_t above = __shfl_sync(0xFFFFFFFFu, p, (int)(16u * h) + (c < 16 ? c : 15));
    if (span > 1) {
      if (c > 0) lo = below;
      if (c < 16) hi = above;
    }
  }
  return lo;
}

// The tiles [t_begin, t_end) of warp w of the grid's nw warps. With weight
// offsets the warps split the total weight evenly, a warp taking the tiles
// that start (tile k of message j starts at weight_off[j] + k * (tile +
// kTileCost)) in its share: tiles of one message are equal but the last, and
// messages differ, so equal tile counts would not be equal work. Without
// them (host-built descriptor batches) every warp gets the same count.
// j_begin: a message at or before the one holding t_begin (the walk moves
// forward from it), when t_begin < t_end.
__device__ __forceinline__ void warp_tile_range(const int64_t* tile_off, const int64_t* weight_off,
                                                int64_t nmsg, int64_t tile, int64_t w, int64_t nw,
                                                uint32_t lane, int64_t& t_begin, int64_t& t_end,
                                                int64_t& j_begin) {
  const int64_t total = __ldg(tile_off + nmsg);
  if (!weight_off || total == 0) {
    const int64_t per = (total + nw - 1) / nw;
    t_begin = tmin<int64_t>(total, w * per);
    t_end = tmin<int64_t>(total, t_begin + per);
    j_begin = t_begin < t_end ? owner_of_warp(tile_off, nmsg, t_begin, lane) : 0;
    return;
  }
  const int64_t wt = __ldg(weight_off + nmsg);  // > 0 when there are tiles
  const bool last = w + 1 == nw;
  // lanes 0-15: the start of the share, 16-31: its end (the next share's start)
  const int64_t x = lane < 16 ? wt * w / nw : (last ? 0 : wt * (w + 1) / nw);
  const int64_t j = owner_of_halves(weight_off, nmsg, x, lane);
  const int64_t t0 = __ldg(tile_off + j), nt = __ldg(tile_off + j + 1) - t0;
  const int64_t k = (x - __ldg(weight_off + j) + tile + kTileCost - 1) / (tile + kTileCost);
  const int64_t t = t0 + tmin<int64_t>(k, nt);  // the first tile starting at or after x
  t_begin = __shfl_sync(0xFFFFFFFFu, t, 0);
  t_end = last ? total : __shfl_sync(0xFFFFFFFFu, t, 16);
  j_begin = __shfl_sync(0xFFFFFFFFu, j, 0);  // t_begin is in j or a later message
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

// ------------------------------------------------------ warp pipeline
// Every warp walks its own contiguous range of tiles. Tile t of message j
// holds input bytes [t0, t0 + len) of j (len <= tile). The tile's
// 16-byte-aligned interior is copied into the warp's input stage by one bulk
// copy, issued `stages` tiles ahead; stage position o + i holds input byte
// t0 + i, o being the tile start's address mod 16, so positions [ia, ib)
// are the copied ones. Units whose bytes reach outside [ia, ib) read global
// memory instead. Every unit's output goes to the warp's output stage at
// position o2 + i for output byte i (o2 = the output start's address mod
// 16); the aligned interior of the tile's output leaves by one bulk store,
// its two ragged ends (at most 15 bytes each) by byte stores.
struct TileView {
  const uint8_t* msrc;  // the message's input and output
  uint8_t* mout;
  const uint8_t* lo;    // bounds of aligned-word reads near the message ends
  const uint8_t* hi;
  uint8_t* dst;         // output of the tile's first unit
  int64_t t0;           // offset of the tile in its message
  int64_t mlen;
  int64_t j;            // message index
  uint32_t len;         // input bytes of the tile
  uint32_t o;           // stage position of input byte t0
  uint32_t ia, ib;
};

// The issuing lane's walk over its tiles: the current message is kept in
// the warp's slot of shared memory (not in registers, which every lane would
// pay for), so the offsets arrays are read only when the walk enters the
// next message (tile_off is non-decreasing; tiles are visited in order).
struct WalkState {
  Msg m;
  int64_t j;        // current message
  int64_t t_first;  // its first tile
  int64_t t_end;    // one past its last tile
};

template <class Msgs>
__device__ __forceinline__ void walk_load(WalkState& w, const Msgs& ms, const int64_t* tile_off) {
  w.m = ms.get(w.j);
  w.t_first = __ldg(tile_off + w.j);
  w.t_end = __ldg(tile_off + w.j + 1);
}

// The view of tile t (t >= the previous tile asked for).
template <class Msgs>
__device__ __forceinline__ TileView walk_view(WalkState& w, const Msgs& ms,
                                              const int64_t* tile_off, int64_t t, int64_t tile,
                                              int64_t out_tile) {
  while (t >= w.t_end) {
    ++w.j;
    walk_load(w, ms, tile_off);
  }
  const Msg m = w.m;
  const int64_t k = t - w.t_first;
  TileView v;
  v.msrc = m.src;
  v.mout = m.out;
  v.lo = m.lo;
  v.hi = m.hi;
  v.dst = m.out + k * out_tile;
  v.t0 = k * tile;
  v.mlen = m.len;
  v.j = w.j;
  v.len = (uint32_t)tmin<int64_t>(tile, m.len - v.t0);
  const uintptr_t s = reinterpret_cast<uintptr_t>(m.src + v.t0);
  const uintptr_t a = (s + 15u) & ~(uintptr_t)15u, b = (s + v.len) & ~(uintptr_t)15u;
  v.o = (uint32_t)(s & 15u);
  v.ia = v.o ? 16u : 0u;
  v.ib = b > a ? v.ia + (uint32_t)(b - a) : v.ia;
  return v;
}

// Issues the bulk copy of a tile's interior into its input stage (one lane;
// the arrive publishes the view written before it).
__device__ __forceinline__ void issue_tile(const TileView& v, uint8_t* in, uint64_t* bar) {
  fence_proxy_async_smem();  // earlier generic reads of this stage come first
  if (v.ib > v.ia) {
    mbar_arrive_expect_tx(bar, v.ib - v.ia);
    tma_load_1d(in + v.ia, v.msrc + v.t0 + (v.ia - v.o), v.ib - v.ia, bar);
  } else {
    mbar_arrive(bar);
  }
}

// Writes output bytes [0, olen) of a tile, staged at out + (d mod 16), to d:
// the aligned interior by one bulk store (always one commit group per
// tile), the ends by lanes 0-14 and 16-30. The warp has fenced and synced.
__device__ __forceinline__ void copy_out(uint8_t* d, uint32_t olen, const uint8_t* out,
                                         uint32_t lane) {
  const uintptr_t da = reinterpret_cast<uintptr_t>(d);
  const uint32_t o2 = (uint32_t)(da & 15u);
  const uintptr_t a = (da + 15u) & ~(uintptr_t)15u, b = (da + olen) & ~(uintptr_t)15u;
  if (lane == 0) {
    if (b > a) tma_store_1d(reinterpret_cast<void*>(a), out + (o2 ? 16u : 0u), (uint32_t)(b - a));
    bulk_commit();
  }
  const uint32_t head = (uint32_t)(tmin<uintptr_t>(a, da + olen) - da);
  const uint32_t ie = b > a ? (uint32_t)(b - da) : head;  // end of the interior
  if (lane < head) {
    d[lane] = out[o2 + lane];
  } else if (lane >= 16u && lane - 16u < olen - ie) {
    d[ie + lane - 16u] = out[o2 + ie + lane - 16u];
  }
}

// Input words of the 12 tile bytes at off: from the stage when they were
// all copied there, else from global memory (off + 12 <= the tile's length).
__device__ __forceinline__ uint3 enc_load(const TileView& v, const uint8_t* in, const uint8_t* sp,
                                          uint32_t off) {
  const uint32_t p = v.o + off;
  return (p >= v.ia && p + 12u <= v.ib) ? lds12(in + p) : load12_any(sp + off, v.lo, v.hi);
}

__device__ __forceinline__ uint32_t word_of(uint4 c, uint32_t k) {
  return k < 2 ? (k == 0 ? c.x : c.y) : (k == 2 ? c.z : c.w);
}

__device__ __forceinline__ uint32_t byte_of(uint4 c, uint32_t k) {
  return (word_of(c, k >> 2) >> (8u * (k & 3u))) & 0xFFu;
}

// cnt whole chunks: chunk i encodes the 12 stage bytes at sb + 12i (sb + 12i
// is R mod 4 for every i) and goes to the aligned 16 bytes at db + 16i.
template <int R>
__device__ __forceinline__ void enc_chunks(const uint8_t* sb, uint8_t* db, int32_t cnt,
                                           uint32_t lane, const uint8_t* T) {
  const uint32_t* wb = reinterpret_cast<const uint32_t*>(sb - R);
#pragma unroll 2
  for (int32_t i = (int32_t)lane; i < cnt; i += 32) {
    const uint32_t* q = wb + 3 * i;
    uint32_t x, y, z;
    if (R == 0) {
      x = q[0];
      y = q[1];
      z = q[2];
    } else {
      const uint32_t q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
      x = __funnelshift_r(q0, q1, 8 * R);
      y = __funnelshift_r(q1, q2, 8 * R);
      z = __funnelshift_r(q2, q3, 8 * R);
    }
    st_global_v4_cs(db + 16 * i, enc_unit(x, y, z, T));
  }
}

// The same chunks read straight from global memory (no staging): s is the
// input of the first chunk, s + 12i is R mod 4 for every i, and the aligned
// words covering each chunk's 12 bytes lie inside the input buffer. Each
// lane issues the loads of up to four chunks before coding them.
template <int R>
__device__ __forceinline__ void enc_chunks_global(const uint8_t* s, uint8_t* db, int32_t cnt,
                                                  uint32_t lane, const uint8_t* T) {
  constexpr int32_t kAhead = 4;
  const uint32_t* wb = reinterpret_cast<const uint32_t*>(s - R);
  for (int32_t i0 = 0; i0 < cnt; i0 += 32 * kAhead) {
    uint32_t q[kAhead][4];
#pragma unroll
    for (int32_t k = 0; k < kAhead; ++k) {
      const int32_t i = i0 + 32 * k + (int32_t)lane;
      if (i < cnt) {
        const uint32_t* p = wb + 3 * i;
        q[k][0] = __ldg(p);
        q[k][1] = __ldg(p + 1);
        q[k][2] = __ldg(p + 2);
        q[k][3] = R ? __ldg(p + 3) : 0u;
      }
    }
#pragma unroll
    for (int32_t k = 0; k < kAhead; ++k) {
      const int32_t i = i0 + 32 * k + (int32_t)lane;
      if (i < cnt) {
        const uint32_t x = R ? __funnelshift_r(q[k][0], q[k][1], 8 * R) : q[k][0];
        const uint32_t y = R ? __funnelshift_r(q[k][1], q[k][2], 8 * R) : q[k][1];
        const uint32_t z = R ? __funnelshift_r(q[k][2], q[k][3], 8 * R) : q[k][2];
        st_global_v4_cs(db + 16 * i, enc_unit(x, y, z, T));
      }
    }
  }
}

// Encodes one tile (Algorithm 1 per 12-byte unit) straight to global memory
// in aligned 16-byte stores; the message's last tile also codes the partial
// group with its padding.
//  - Output start d word-aligned (d mod 16 = 4q, always so for padded
//    output at a word-aligned base): the lane of aligned chunk c writes the
//    16 characters at d - 4q + 16c, which encode tile bytes
//    [12c - 3q, 12c - 3q + 12). With q > 0, chunk 0 keeps the first 4 - q
//    words of unit 0's characters and chunk nu the last q words of unit
//    nu - 1's.
//  - Otherwise (d mod 4 != 0): lanes code units, and the lane of unit u
//    builds aligned chunk u from unit u - 1 (the previous lane, or the
//    previous row's last lane) and unit u; the ends go out as bytes.
// DIRECT: nothing was staged (v.ia == v.ib); whole chunks read global memory.
template <bool DIRECT>
__device__ __forceinline__ void encode_tile(const TileView& v, const uint8_t* in,
                                            const uint8_t* T, uint32_t lane, uint32_t flags) {
  const uint32_t nu = v.len / 12u;
  const uint8_t* sp = v.msrc + v.t0;
  uint8_t* dp = v.dst;
  const uint32_t o2 = (uint32_t)(reinterpret_cast<uintptr_t>(dp) & 15u);
  uint8_t* abase = dp - o2;  // 16-byte aligned
  if ((o2 & 3u) == 0) {
    const uint32_t q = o2 >> 2;
    // whole chunks c in [cf, nu): input offset 12c - 3q, stage position
    // p0 + 12c; those whose 12 bytes were all copied, [c_lo, c_hi), take
    // the loop specialised on the stage's 4-byte phase
    const int32_t cf = q ? 1 : 0, n = (int32_t)nu;
    int32_t c_lo, c_hi;
    if (DIRECT) {
      // every whole chunk, but a chunk whose aligned words would reach
      // outside the input buffer (first or last only) goes with the edges
      c_lo = min(n, cf);
      c_hi = n;
      const uintptr_t s0 = reinterpret_cast<uintptr_t>(sp) + 12 * c_lo - 3 * q;
      const uint32_t r = (uint32_t)(s0 & 3u);
      if (r && c_hi > c_lo) {
        if (s0 - r < reinterpret_cast<uintptr_t>(v.lo)) ++c_lo;
        const uintptr_t sl = reinterpret_cast<uintptr_t>(sp) + 12 * (c_hi - 1) - 3 * q;
        if (sl - r + 16 > reinterpret_cast<uintptr_t>(v.hi)) --c_hi;
        c_hi = max(c_hi, c_lo);
      }
      if (c_hi > c_lo) {
        const uint8_t* s = sp + (12 * c_lo - 3 * (int32_t)q);
        uint8_t* db = abase + 16u * (uint32_t)c_lo;
        const int32_t cnt = c_hi - c_lo;
        switch (r) {
          case 0: enc_chunks_global<0>(s, db, cnt, lane, T); break;
          case 1: enc_chunks_global<1>(s, db, cnt, lane, T); break;
          case 2: enc_chunks_global<2>(s, db, cnt, lane, T); break;
          default: enc_chunks_global<3>(s, db, cnt, lane, T); break;
        }
      }
    } else {
      const int32_t p0 = (int32_t)v.o - 3 * (int32_t)q;
      c_lo = n > 0 ? min(n, max(cf, ((int32_t)v.ia - p0 + 11) / 12)) : 0;
      const int32_t room = (int32_t)v.ib - 12 - p0;  // last copied chunk start
      c_hi = room < 0 ? c_lo : max(c_lo, min(n, room / 12 + 1));
      if (c_hi > c_lo) {
        const uint8_t* sb = in + (p0 + 12 * c_lo);
        uint8_t* db = abase + 16u * (uint32_t)c_lo;
        const int32_t cnt = c_hi - c_lo;
        switch ((p0 + 12 * c_lo) & 3) {
          case 0: enc_chunks<0>(sb, db, cnt, lane, T); break;
          case 1: enc_chunks<1>(sb, db, cnt, lane, T); break;
          case 2: enc_chunks<2>(sb, db, cnt, lane, T); break;
          default: enc_chunks<3>(sb, db, cnt, lane, T); break;
        }
      }
    }
    // the rest: chunks outside the copied part, and with q > 0 the partial
    // chunks at both ends (chunk 0 keeps the first 4 - q words of unit 0's
    // characters, chunk nu the last q words of unit nu - 1's)
    const int32_t nedge = n == 0 ? 0 : (c_lo - cf) + (n - c_hi) + (q ? 2 : 0);
    for (int32_t k = (int32_t)lane; k < nedge; k += 32) {
      int32_t c;
      if (k < c_lo - cf) {
        c = cf + k;
      } else if (k < (c_lo - cf) + (n - c_hi)) {
        c = c_hi + (k - (c_lo - cf));
      } else {
        c = (k == nedge - 2) ? 0 : n;  // the two partial chunks
      }
      const bool head = q && c == 0, tail = q && c == n;
      const uint32_t off = head ? 0u : (tail ? 12u * (nu - 1u) : 12u * (uint32_t)c - 3u * q);
      const uint3 w = enc_load(v, in, sp, off);
      const uint4 e = enc_unit(w.x, w.y, w.z, T);
      if (!head && !tail) {
        st_global_v4_cs(abase + 16u * (uint32_t)c, e);
      } else {
        uint32_t* wd = reinterpret_cast<uint32_t*>(head ? dp : dp + 16u * nu - 4u * q);
        const uint32_t k0 = head ? 0u : 4u - q, nk = head ? 4u - q : q;
        for (uint32_t i = 0; i < nk; ++i) wd[i] = word_of(e, k0 + i);
      }
    }
  } else {
    uint4 carry = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t base = 0; base < nu; base += 32u) {
      const uint32_t u = base + lane;
      uint4 c = make_uint4(0u, 0u, 0u, 0u);
      if (u < nu) {
        const uint3 w = enc_load(v, in, sp, 12u * u);
        c = enc_unit(w.x, w.y, w.z, T);
      }
      uint4 prev;
      prev.x = __shfl_up_sync(0xFFFFFFFFu, c.x, 1);
      prev.y = __shfl_up_sync(0xFFFFFFFFu, c.y, 1);
      prev.z = __shfl_up_sync(0xFFFFFFFFu, c.z, 1);
      prev.w = __shfl_up_sync(0xFFFFFFFFu, c.w, 1);
      if (lane == 0) prev = carry;
      if (u < nu) {
        if (u > 0) {
          st_global_v4_cs(abase + 16u * u, realign16(prev, c, 16u - o2));
        } else {
          for (uint32_t k = 0; k < 16u - o2; ++k) dp[k] = (uint8_t)byte_of(c, k);
        }
        if (u == nu - 1) {
          uint8_t* t = dp + 16u * nu - o2;
          for (uint32_t k = 0; k < o2; ++k) t[k] = (uint8_t)byte_of(c, 16u - o2 + k);
        }
      }
      carry.x = __shfl_sync(0xFFFFFFFFu, c.x, 31);
      carry.y = __shfl_sync(0xFFFFFFFFu, c.y, 31);
      carry.z = __shfl_sync(0xFFFFFFFFu, c.z, 31);
      carry.w = __shfl_sync(0xFFFFFFFFu, c.w, 31);
    }
  }
  const uint32_t rest = v.len - 12u * nu;
  const uint32_t ng = (rest + 2u) / 3u;
  if (lane < ng) {
    const uint8_t* p = sp + 12u * nu + 3u * lane;
    const uint32_t cnt = min(3u, rest - 3u * lane);
    const uint32_t b0 = p[0], b1 = cnt > 1 ? p[1] : 0u, b2 = cnt > 2 ? p[2] : 0u;
    store_tail_group(dp + 16u * nu + 4u * lane, enc_tail_group(b0, b1, b2, cnt, T), cnt, flags);
  }
}

// Characters of decode unit u of a tile, from the stage or global memory.
__device__ __forceinline__ uint4 dec_load(const TileView& v, const uint8_t* in, uint32_t u) {
  const uint32_t p = v.o + 16u * u;
  if (p >= v.ia && p + 16u <= v.ib) {
    const uint4* q = reinterpret_cast<const uint4*>(in + (p & ~15u));
    return v.o ? realign16(q[0], q[1], v.o) : q[0];
  }
  return load16_any(v.msrc + v.t0 + 16u * u, v.lo, v.hi);
}

// Stages a row of decoded units (12 bytes each at o2 + 12u): word stores
// when o2 is word-aligned, else aligned words whose first one takes the
// last bytes of unit u - 1 (the previous lane, or `carry` from the previous
// row). Every lane of the warp calls it.
__device__ __forceinline__ void dec_store_row(uint8_t* out, uint32_t o2, uint32_t u, uint32_t nu,
                                              uint3 o, uint32_t& carry, uint32_t lane) {
  const uint32_t r2 = o2 & 3u;
  if (r2 == 0) {
    if (u < nu) {
      uint32_t* wq = reinterpret_cast<uint32_t*>(out + o2 + 12u * u);
      wq[0] = o.x;
      wq[1] = o.y;
      wq[2] = o.z;
    }
    return;
  }
  uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, o.z, 1);
  if (lane == 0) prev = carry;
  if (u < nu) {
    uint32_t* wq = reinterpret_cast<uint32_t*>(out + ((o2 + 12u * u) & ~3u));
    const uint32_t sh = 8u * (4u - r2);
    wq[0] = __funnelshift_r(prev, o.x, sh);
    wq[1] = __funnelshift_r(o.x, o.y, sh);
    wq[2] = __funnelshift_r(o.y, o.z, sh);
    if (u == nu - 1) wq[3] = __funnelshift_r(o.z, o.z, sh);
  }
  carry = __shfl_sync(0xFFFFFFFFu, o.z, 31);
}

// The same row written straight to the tile's output d (unit u at
// d + 12u): aligned word stores, the word shared with the unit before the
// tile and the one shared with the unit after it by bytes (other warps may
// be writing the rest of those words).
__device__ __forceinline__ void dec_store_row_global(uint8_t* d, uint32_t u, uint32_t nu, uint3 o,
                                                     uint32_t& carry, uint32_t lane) {
  const uint32_t r2 = (uint32_t)(reinterpret_cast<uintptr_t>(d) & 3u);
  if (r2 == 0) {
    if (u < nu) {
      uint32_t* wq = reinterpret_cast<uint32_t*>(d + 12u * u);
      wq[0] = o.x;
      wq[1] = o.y;
      wq[2] = o.z;
    }
    return;
  }
  uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, o.z, 1);
  if (lane == 0) prev = carry;
  if (u < nu) {
    uint8_t* q = d + 12u * u;
    uint32_t* wq = reinterpret_cast<uint32_t*>(q - r2);  // aligned word holding q[0]
    const uint32_t sh = 8u * (4u - r2);
    if (u == 0) {
      for (uint32_t k = 0; k < 4u - r2; ++k) q[k] = (uint8_t)(o.x >> (8u * k));
    } else {
      wq[0] = __funnelshift_r(prev, o.x, sh);
    }
    wq[1] = __funnelshift_r(o.x, o.y, sh);
    wq[2] = __funnelshift_r(o.y, o.z, sh);
    if (u == nu - 1)
      for (uint32_t k = 0; k < r2; ++k) q[12u - r2 + k] = (uint8_t)(o.z >> (sh + 8u * k));
  }
  carry = __shfl_sync(0xFFFFFFFFu, o.z, 31);
}

// Decodes one tile (Algorithm 2 per 16-character unit; whole quads after
// the last unit and, in the tile holding it, the message's final group go
// straight to global memory). DIRECT: the units are read from and written
// to global memory, four rows' loads issued before their decoding.
template <bool DIRECT>
__device__ __forceinline__ void decode_tile(const TileView& v, const uint8_t* in, uint8_t* out,
                                            const uint8_t* D, unsigned long long* fb,
                                            int64_t* outlen_j, uint32_t lane, uint32_t flags) {
  const uint64_t mlen = (uint64_t)v.mlen;
  const uint64_t body_end = decode_body_end(mlen);
  const uint64_t t0 = (uint64_t)v.t0;
  const uint32_t body = body_end > t0 ? (uint32_t)tmin<uint64_t>(v.len, body_end - t0) : 0u;
  const uint32_t nu = body / 16u;
  uint8_t* dp = v.dst;
  const uint32_t o2 = (uint32_t)(reinterpret_cast<uintptr_t>(dp) & 15u);
  unsigned long long bad = ~0ull;
  uint32_t carry = 0;  // last word of the previous row's last unit
  if (DIRECT) {
    constexpr uint32_t kAhead = 4;
    const uint8_t* s = v.msrc + v.t0;
    for (uint32_t base = 0; base < nu; base += 32u * kAhead) {
      uint4 w[kAhead];
#pragma unroll
      for (uint32_t k = 0; k < kAhead; ++k) {
        const uint32_t u = base + 32u * k + lane;
        w[k] = u < nu ? load16_any(s + 16u * u, v.lo, v.hi) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (uint32_t k = 0; k < kAhead; ++k) {
        if (base + 32u * k >= nu) break;  // the whole warp
        const uint32_t u = base + 32u * k + lane;
        uint32_t err = 0;
        const uint3 o = dec_unit(w[k], D, err);
        if ((err & kBadFlag) && u < nu && bad == ~0ull)
          bad = t0 + 16u * u + dec_unit_first_bad(w[k], D);
        dec_store_row_global(dp, u, nu, o, carry, lane);
      }
    }
  } else {
    for (uint32_t base = 0; base < nu; base += 32u) {
      const uint32_t u = base + lane;
      uint4 w = make_uint4(0u, 0u, 0u, 0u);
      if (u < nu) w = dec_load(v, in, u);
      uint32_t err = 0;
      const uint3 o = dec_unit(w, D, err);
      if ((err & kBadFlag) && u < nu && bad == ~0ull)
        bad = t0 + 16u * u + dec_unit_first_bad(w, D);
      dec_store_row(out, o2, u, nu, o, carry, lane);
    }
  }
  warp_min_to(fb, bad);
  const uint32_t nq = (body - 16u * nu) / 4u;
  if (lane < nq) {
    const uint64_t idx = t0 + 16u * nu + 4u * lane;
    const uint8_t* p = v.msrc + idx;
    const uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                       ((uint32_t)p[3] << 24);
    uint32_t err = 0;
    const uint32_t val = dec_quad(x, D, err);
    if (err & kBadFlag) {
      for (uint32_t q = 0; q < 4; ++q)
        if (D[(x >> (8 * q)) & 0xFFu] & kBadFlag) {
          atomicMin(fb, (unsigned long long)(idx + q));
          break;
        }
    } else {
      uint8_t* w = v.mout + idx / 4 * 3;
      w[0] = (uint8_t)(val >> 16);
      w[1] = (uint8_t)(val >> 8);
      w[2] = (uint8_t)val;
    }
  }
  if (lane == 31 && body_end >= t0 && body_end < t0 + v.len)
    *outlen_j = dec_final_group(v.msrc, mlen, body_end, v.mout, D, fb, flags);
  if (!DIRECT) {
    fence_proxy_async_smem();
    __syncwarp();
    copy_out(dp, 12u * nu, out, lane);
  }
}

// ------------------------------------------------------ short messages
// One thread codes a whole message of at most small_max bytes (encode) or
// characters (decode), straight between global memory and registers: a
// message of a few dozen bytes then costs its own groups only, not a tile.
__device__ __forceinline__ void encode_message(const uint8_t* p, int64_t n, uint8_t* d,
                                               const uint8_t* T, uint32_t flags,
                                               const uint8_t* lo, const uint8_t* hi) {
  const uint32_t nu = (uint32_t)(n / 12);
  for (uint32_t u0 = 0; u0 < nu; u0 += 4) {  // Algorithm 1 on 12-byte units, 4 loads ahead
    uint3 w[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (u0 + k < nu) w[k] = load12_any(p + 12 * (u0 + k), lo, hi);
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (u0 + k < nu) store16_any(d + 16 * (u0 + k), enc_unit(w[k].x, w[k].y, w[k].z, T));
  }
  const uint32_t rest = (uint32_t)n - 12 * nu;
  for (uint32_t g = 0; 3 * g < rest; ++g) {  // whole groups, then the partial one
    const uint8_t* q = p + 12 * nu + 3 * g;
    const uint32_t cnt = min(3u, rest - 3 * g);
    const uint32_t b0 = q[0], b1 = cnt > 1 ? q[1] : 0u, b2 = cnt > 2 ? q[2] : 0u;
    store_tail_group(d + 16 * nu + 4 * g, enc_tail_group(b0, b1, b2, cnt, T), cnt, flags);
  }
}

// Sequential byte output through aligned 32-bit stores: bytes are gathered
// in `word` until its aligned word is full; the first and last words of the
// output, shared with the neighbouring messages, are written byte by byte.
struct WordWriter {
  uint8_t* start;   // first output byte
  uint32_t* w;      // aligned word being filled
  uint32_t word = 0;
  uint32_t fill;    // bytes of *w before the next byte
  __device__ __forceinline__ explicit WordWriter(uint8_t* d)
      : start(d),
        w(reinterpret_cast<uint32_t*>(reinterpret_cast<uintptr_t>(d) & ~(uintptr_t)3)),
        fill((uint32_t)(reinterpret_cast<uintptr_t>(d) & 3u)) {}
  // appends the 4 bytes of x (little-endian)
  __device__ __forceinline__ void put4(uint32_t x) {
    if (fill == 0) {
      store_full(x);
      return;
    }
    const uint32_t sh = 8u * fill;
    store_full(word | (x << sh));
    word = x >> (32u - sh);
  }
  __device__ __forceinline__ void store_full(uint32_t v) {
    if (reinterpret_cast<uint8_t*>(w) < start) {  // the first word: our bytes only
      const uint32_t skip = (uint32_t)(start - reinterpret_cast<uint8_t*>(w));
      for (uint32_t k = skip; k < 4; ++k) reinterpret_cast<uint8_t*>(w)[k] = (uint8_t)(v >> (8 * k));
    } else {
      *w = v;
    }
    ++w;
  }
  // writes the bytes still held (fewer than 4)
  __device__ __forceinline__ void flush() {
    for (uint32_t k = 0; k < fill; ++k) {
      uint8_t* q = reinterpret_cast<uint8_t*>(w) + k;
      if (q >= start) *q = (uint8_t)(word >> (8 * k));
    }
  }
};

// Algorithm 2 over the body (stopping at the first invalid character, whose
// index goes to *fb), then the final characters; *outlen_j receives the
// final group's result as for the tile kernels.
__device__ __forceinline__ void decode_message(const uint8_t* p, int64_t m, uint8_t* d,
                                               const uint8_t* D, unsigned long long* fb,
                                               int64_t* outlen_j, uint32_t flags,
                                               const uint8_t* lo, const uint8_t* hi) {
  const uint64_t body_end = decode_body_end((uint64_t)m);
  const uint32_t nq = (uint32_t)(body_end / 4), nu = nq / 4;
  WordWriter out(d);
  for (uint32_t u0 = 0; u0 < nu; u0 += 4) {  // 16-character units, 4 loads ahead
    uint4 w[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (u0 + k < nu) w[k] = load16_any(p + 16 * (u0 + k), lo, hi);
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
      if (u0 + k >= nu) break;
      uint32_t err = 0;
      const uint3 o = dec_unit(w[k], D, err);
      if (err & kBadFlag) {
        *fb = 16ull * (u0 + k) + dec_unit_first_bad(w[k], D);
        return;
      }
      out.put4(o.x);
      out.put4(o.y);
      out.put4(o.z);
    }
  }
  out.flush();
  for (uint32_t k = 4 * nu; k < nq; ++k) {  // the last whole quads
    const uint8_t* c = p + 4 * k;
    const uint32_t x = (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) |
                       ((uint32_t)c[3] << 24);
    uint32_t err = 0;
    const uint32_t val = dec_quad(x, D, err);
    if (err & kBadFlag) {
      for (uint32_t i = 0; i < 4; ++i)
        if (D[(x >> (8 * i)) & 0xFFu] & kBadFlag) {
          *fb = 4ull * k + i;
          return;
        }
    }
    uint8_t* q = d + 3 * k;
    q[0] = (uint8_t)(val >> 16);
    q[1] = (uint8_t)(val >> 8);
    q[2] = (uint8_t)val;
  }
  if (m > 0) *outlen_j = dec_final_group(p, (uint64_t)m, body_end, d, D, fb, flags);
}

// The messages of at most small_max bytes / characters, one thread each, the
// grid's threads taking messages in turn (the tile kernel's first work).
template <int DECODE, class Msgs>
__device__ __noinline__ void code_short_messages(Msgs ms, int64_t nmsg, int64_t small_max,
                                                 const uint8_t* table, int64_t* first_bad,
                                                 int64_t* outlen, uint32_t flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nmsg; j += stride) {
    const int64_t len = ms.len(j);
    if (len <= 0 || len > small_max) continue;
    const Msg m = ms.get(j);
    if (DECODE) {
      decode_message(m.src, m.len, m.out, table,
                     reinterpret_cast<unsigned long long*>(first_bad + j), outlen + j, flags, m.lo,
                     m.hi);
    } else {
      encode_message(m.src, m.len, m.out, table, flags, m.lo, m.hi);
    }
  }
}

// Shared memory of a warp: `stages` input stages, and (decode) two output
// buffers, used by alternate tiles.
__host__ __device__ __forceinline__ uint32_t stage_in_bytes(int64_t tile) {
  return (uint32_t)tile + 32u;
}
__host__ __device__ __forceinline__ int64_t out_tile_bytes(int decode, int64_t tile) {
  return decode ? tile / 4 * 3 : tile / 3 * 4;
}
__host__ __device__ __forceinline__ uint32_t warp_smem_bytes(int decode, int64_t tile,
                                                             uint32_t stages) {
  return stages * stage_in_bytes(tile) + (decode ? (uint32_t)out_tile_bytes(1, tile) + 32u : 0u);
}

// The persistent kernel of both directions: warp w of the grid's G warps
// owns tiles [w*T/G, (w+1)*T/G) of the T = tile_off[nmsg] tiles, in order.
// Lane 0 of the warp computes each tile's view once, when it issues the
// tile's copy, and leaves it beside the stage.
template <int NT, int DECODE, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_code(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ tile_off,
                 const int64_t* __restrict__ weight_off, int64_t tile, uint32_t stages,
                 int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen, uint32_t flags,
                 int64_t small_max) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t table[DECODE ? 256 : 64];
  __shared__ __align__(8) uint64_t full[NT / 32][kMaxBatchStages];
  __shared__ TileView meta[NT / 32][kMaxBatchStages];
  __shared__ WalkState walks[NT / 32];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t S = stages;
  if (lane == 0) {
    for (uint32_t s = 0; s < S; ++s) mbar_init(&full[warp][s], 1);
    fence_mbar_init();
  }
  if (DECODE) {
    init_tables(nullptr, table, flags & kFlagUrl);
  } else {
    init_tables(table, nullptr, flags & kFlagUrl);
  }
  const int64_t out_tile = out_tile_bytes(DECODE, tile);
  const uint32_t in_b = stage_in_bytes(tile);
  uint8_t* wbase = smem + (size_t)warp * warp_smem_bytes(DECODE, tile, S);
  uint8_t* obase = wbase + S * in_b;  // decode: the output buffer

  int64_t t_begin, t_end, j_begin;
  warp_tile_range(tile_off, weight_off, nmsg, tile, (int64_t)blockIdx.x * (NT / 32) + warp,
                  (int64_t)gridDim.x * (NT / 32), lane, t_begin, t_end, j_begin);
  Msgs ms = msgs;
  ms.prepare(nmsg);
  WalkState& walk = walks[warp];  // used by lane 0
  if (lane == 0 && t_begin < t_end) {  // the first tiles' copies go out first
    walk.j = j_begin;
    walk_load(walk, ms, tile_off);
    for (uint32_t s = 0; s < S && t_begin + s < t_end; ++s) {
      meta[warp][s] = walk_view(walk, ms, tile_off, t_begin + s, tile, out_tile);
      issue_tile(meta[warp][s], wbase + s * in_b, &full[warp][s]);
    }
  }
  // short messages (no tiles) while those copies are in flight
  if (small_max > 0)
    code_short_messages<DECODE>(ms, nmsg, small_max, table, first_bad, outlen, flags);
  if (t_begin >= t_end) return;

  bool timed_out = false;
  uint32_t s = 0, phase = 0;
  int64_t t = t_begin;
  for (; t < t_end; ++t) {
    uint8_t* in = wbase + s * in_b;
    const bool ok = mbar_wait_backoff(&full[warp][s], phase);
    if (__any_sync(0xFFFFFFFFu, !ok)) {
      timed_out = true;
      break;
    }
    const TileView v = meta[warp][s];
    if (DECODE) {
      // the previous tile's bulk store has finished reading the output buffer
      if (lane == 0 && t > t_begin) bulk_wait_read(0);
      __syncwarp();
      decode_tile<false>(v, in, obase, table,
                  reinterpret_cast<unsigned long long*>(first_bad + v.j), outlen + v.j, lane, flags);
    } else {
      encode_tile<false>(v, in, table, lane, flags);
      fence_proxy_async_smem();  // the stage's reads come before its next copy
      __syncwarp();
    }
    if (lane == 0 && t + S < t_end) {
      meta[warp][s] = walk_view(walk, ms, tile_off, t + S, tile, out_tile);
      issue_tile(meta[warp][s], in, &full[warp][s]);
    }
    if (++s == S) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (timed_out && lane == 0) {
    atomicOr(&g_batch_fault, 1u);
    // wait (bounded) for the copies still in flight into this warp's stages
    for (uint32_t i = 0; i < S && t + i < t_end; ++i) {
      mbar_wait_bounded(&full[warp][s], phase, 500000000ull);
      if (++s == S) {
        s = 0;
        phase ^= 1u;
      }
    }
  }
  if (DECODE && lane == 0) bulk_wait_all();
}

// The same persistent walk without staging: every lane keeps the walk in
// registers (one warp-instruction each, as on one lane), and the tiles'
// units move straight between global memory and registers, so a warp needs
// no shared memory, barrier or copy engine, and a tile may be longer than a
// stage could hold.
template <int NT, int DECODE, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_direct(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ tile_off,
                   const int64_t* __restrict__ weight_off, int64_t tile,
                   int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen, uint32_t flags,
                   int64_t small_max) {
  __shared__ uint8_t table[DECODE ? 256 : 64];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (DECODE) {
    init_tables(nullptr, table, flags & kFlagUrl);
  } else {
    init_tables(table, nullptr, flags & kFlagUrl);
  }
  const int64_t out_tile = out_tile_bytes(DECODE, tile);
  int64_t t_begin, t_end, j_begin;
  warp_tile_range(tile_off, weight_off, nmsg, tile, (int64_t)blockIdx.x * (NT / 32) + warp,
                  (int64_t)gridDim.x * (NT / 32), lane, t_begin, t_end, j_begin);
  Msgs ms = msgs;
  ms.prepare(nmsg);
  if (small_max > 0)
    code_short_messages<DECODE>(ms, nmsg, small_max, table, first_bad, outlen, flags);
  if (t_begin >= t_end) return;
  WalkState walk;
  walk.j = j_begin;
  walk_load(walk, ms, tile_off);
  for (int64_t t = t_begin; t < t_end; ++t) {
    TileView v = walk_view(walk, ms, tile_off, t, tile, out_tile);
    v.o = v.ia = v.ib = 0u;  // nothing staged
    if (DECODE) {
      decode_tile<true>(v, nullptr, nullptr, table,
                        reinterpret_cast<unsigned long long*>(first_bad + v.j), outlen + v.j, lane,
                        flags);
    } else {
      encode_tile<true>(v, nullptr, table, lane, flags);
    }
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
size_t batch_smem_bytes(int decode, const BatchConfig& c) {
  if (c.kernel == 2) return 0;  // unstaged tiles
  return (size_t)(c.threads / 32) * warp_smem_bytes(decode, c.tile, (uint32_t)c.stages);
}

size_t batch_scratch_bytes(int64_t nmsg) {
  const int64_t nparts = (nmsg + kScanPerBlock - 1) / kScanPerBlock;
  return (size_t)(nmsg + 1) * 16 + (size_t)std::max<int64_t>(nparts, 1) * 24;
}

cudaError_t batch_offsets(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                          int64_t* tile_off, int64_t* weight_off, int64_t tile, void* scratch_parts,
                          int64_t* first_bad, int64_t* outlen, cudaStream_t stream,
                          uint32_t flags, int64_t small_max) {
  const int64_t nparts = (nmsg + kScanPerBlock - 1) / kScanPerBlock;
  int64_t* parts = static_cast<int64_t*>(scratch_parts);
  if (nparts > 0) {
    k_scan_local<<<(unsigned)nparts, kScanThreads, 0, stream>>>(in_off, nmsg, decode, tile, flags,
                                                                small_max, out_off, tile_off,
                                                                weight_off, parts, nparts);
    k_scan_parts<<<1, kScanThreads, 0, stream>>>(parts, nparts);
  }
  const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
  k_scan_add<<<(unsigned)blocks, 256, 0, stream>>>(nmsg, out_off, tile_off, weight_off, parts,
                                                   nparts, first_bad, outlen);
  return cudaGetLastError();
}

namespace {
template <int NT, class Msgs>
cudaError_t launch_work(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* tile_off,
                        const int64_t* weight_off, int32_t* status, int64_t* first_bad,
                        int64_t* outlen, const BatchConfig& cfg, const DeviceInfo* di,
                        uint32_t flags, cudaStream_t stream, int64_t small_max) {
  const bool direct = cfg.kernel == 2;
  const size_t smem = batch_smem_bytes(decode, cfg);
  const void* kernel;
  if (direct) {
    kernel = decode ? reinterpret_cast<const void*>(k_batch_direct<NT, 1, Msgs>)
                    : reinterpret_cast<const void*>(k_batch_direct<NT, 0, Msgs>);
  } else {
    kernel = decode ? reinterpret_cast<const void*>(k_batch_code<NT, 1, Msgs>)
                    : reinterpret_cast<const void*>(k_batch_code<NT, 0, Msgs>);
  }
  int fit = 0;
  cudaError_t e = kernel_prepare(kernel, smem, NT, &fit);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  const int bps = cfg.blocks_per_sm > 0 ? std::min(fit, cfg.blocks_per_sm) : fit;
  const int grid = di->sm_count * bps;
  const uint32_t stages = (uint32_t)cfg.stages;
  if (direct) {
    if (decode) {
      k_batch_direct<NT, 1, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, tile_off, weight_off,
                                                           cfg.tile, first_bad, outlen, flags,
                                                           small_max);
    } else {
      k_batch_direct<NT, 0, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, tile_off, weight_off,
                                                           cfg.tile, nullptr, nullptr, flags,
                                                           small_max);
    }
  } else if (decode) {
    k_batch_code<NT, 1, Msgs><<<grid, NT, smem, stream>>>(msgs, nmsg, tile_off, weight_off,
                                                          cfg.tile, stages, first_bad, outlen,
                                                          flags, small_max);
  } else {
    k_batch_code<NT, 0, Msgs><<<grid, NT, smem, stream>>>(msgs, nmsg, tile_off, weight_off,
                                                          cfg.tile, stages, nullptr, nullptr,
                                                          flags, small_max);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !decode) return e;
  const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
  k_batch_decode_finish<Msgs><<<(unsigned)blocks, 256, 0, stream>>>(msgs, nmsg, status, first_bad,
                                                                   outlen, flags);
  return cudaGetLastError();
}

template <class Msgs>
cudaError_t launch_work_any(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* tile_off,
                            const int64_t* weight_off, int32_t* status, int64_t* first_bad,
                            int64_t* outlen, const BatchConfig& cfg, uint32_t flags,
                            cudaStream_t stream, int64_t small_max = 0) {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  switch (cfg.threads) {
    case 128:
      return launch_work<128>(decode, msgs, nmsg, tile_off, weight_off, status, first_bad, outlen,
                              cfg, di, flags, stream, small_max);
    case 512:
      return launch_work<512>(decode, msgs, nmsg, tile_off, weight_off, status, first_bad, outlen,
                              cfg, di, flags, stream, small_max);
    default:
      return launch_work<256>(decode, msgs, nmsg, tile_off, weight_off, status, first_bad, outlen,
                              cfg, di, flags, stream, small_max);
  }
}
}  // namespace

cudaError_t batch_launch_desc(int decode, const MsgDesc* desc, int64_t nmsg, uint8_t* dst,
                              const int64_t* tile_off, const int64_t* weight_off,
                              int32_t* status, int64_t* first_bad, int64_t* outlen,
                              const BatchConfig& cfg, bool init_results, cudaStream_t stream,
                              uint32_t flags) {
  if (decode && init_results) {
    const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
    k_batch_decode_init<<<(unsigned)blocks, 256, 0, stream>>>(nmsg, first_bad, outlen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_work_any(decode, DescMsgs{desc, dst}, nmsg, tile_off, weight_off, status,
                         first_bad, outlen, cfg, flags, stream);
}

cudaError_t batch_launch(const BatchArgs& a, const BatchConfig& cfg) {
  const int64_t small_max = cfg.kernel != 1 ? batch_small_max(a.decode) : 0;
  cudaError_t e = batch_offsets(a.decode, a.in_off, a.nmsg, a.out_off, a.tile_off, a.weight_off,
                                cfg.tile, a.parts, a.decode ? a.first_bad : nullptr,
                                a.decode ? a.outlen : nullptr, a.stream, a.flags, small_max);
  if (e != cudaSuccess) return e;
  // src_hi (the end of the packed input, in_off[nmsg]) is read on the device
  PackedMsgs msgs{a.src, a.in_off, a.dst, a.out_off, nullptr};
  // short messages go one thread each at the start of the tile kernel
  return launch_work_any(a.decode, msgs, a.nmsg, a.tile_off, a.weight_off, a.status, a.first_bad,
                         a.outlen, cfg, a.flags, a.stream, small_max);
}

// Longest messages (input bytes / characters) coded one thread each by
// default: below these lengths that is faster on GB300 than a tile per
// message, and a thread's chain of units stays short next to its tiles.
int64_t batch_small_max(int decode) { return decode ? 344 : 256; }

int batch_read_and_clear_fault(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_batch_fault, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_batch_fault, &zero, sizeof(zero));
  *out = v;
  return e == cudaSuccess ? 0 : cuda_status(e, "reading the fault word");
}

}  // namespace gb64
