// Batched encode and decode of many packed messages in one kernel per
// direction.
//
//   1. k_scan_onepass: a device prefix sum (one pass, decoupled look-back) over the
//      messages of (output length, weight). Output length is
//      4 * ceil(n / 3) (encode) or 3 * floor(m / 4) (decode capacity); a
//      message longer than the short-message limit is cut into
//      ceil(length / tile) tiles and weighs its length plus a fixed cost per
//      tile, a shorter one weighs 0. The exclusive sums become out_off
//      (returned to the caller) and weight_off (scratch).
//   2. k_batch_flat / k_batch_flat_enc (kernel choice 3): a batch with
//      padded encodings of at least 1 Ki characters per message on average
//      is coded as one buffer (see the flat sections below); the kernels of
//      step 3 then return at once.
//   3. k_batch_code / k_batch_direct (encode or decode): a persistent grid.
//      Its threads first code the short messages one each; then every warp
//      takes the tiles that start in its equal share of the total weight,
//      finds the message of its first one by a search in weight_off and
//      walks forward message by message. k_batch_code stages each tile in
//      shared memory by a bulk copy (TMA) several tiles ahead; k_batch_direct
//      reads and writes the tiles' units straight from and to global
//      memory. Both code units with the codecs of common.cuh; per-message
//      padding (encode) and final quad, error index and length rule
//      (decode) are handled in the tile that holds the message end.
//   4. k_batch_decode_finish: per-message status, first_bad and outlen
//      (after the flat decode, also each message's final group).
// All launches have fixed shapes, so a call can be captured in a CUDA graph.
#include <algorithm>
#include <atomic>

#include "batch.h"
#include "common.cuh"
#include "internal.h"
#include "search.cuh"

namespace gb64 {

static __device__ unsigned int g_batch_fault;

constexpr int kMaxBatchStages = 6;

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int64_t kScanPerBlock = (int64_t)kScanThreads * kScanItems;
static_assert(kScanPerBlock == kBatchScanPerBlock, "batch_scratch_bytes sizes the scan blocks");
constexpr int64_t kNoBad = INT64_MAX;
constexpr int64_t kTileCost = kBatchTileCost;

// ----------------------------------------------------------------- scan
// floor(n / d) for 0 <= n < 2^48 and 2 <= d < 2^16 by one multiply-high:
// with m = ceil(2^64 / d) = d^-1 * (2^64 + e), 0 <= e < d, n * m / 2^64 =
// n / d + n * e / (d * 2^64) exceeds n / d by less than 1 / d, too little
// to reach the next integer. Saves the 64-bit division routine (and its
// registers) in the tile walk; device buffers are far below 2^48 bytes.
struct DivBy {
  uint64_t m;
  __host__ __device__ static DivBy of(int64_t d) { return DivBy{~0ull / (uint64_t)d + 1}; }
  __device__ __forceinline__ int64_t operator()(int64_t n) const {
    return (int64_t)__umul64hi((uint64_t)n, m);
  }
};

// Tiles of a message of len bytes / characters: none at most small_max
// (threads code it one each), else ceil(len / tile). The scan and the tile
// walk both count them this way.
__device__ __forceinline__ int64_t msg_tiles(int64_t len, int64_t tile, DivBy by_tile,
                                             int64_t small_max) {
  return len > small_max ? by_tile(len + tile - 1) : 0;
}

// Weight of a message with `tiles` tiles: what the tile kernels divide
// evenly among their warps.
__device__ __forceinline__ int64_t msg_weight(int64_t len, int64_t tiles) {
  return tiles ? len + tiles * kTileCost : 0;
}

// Output length and weight of one message (by_tile = DivBy::of(tile)).
__device__ __forceinline__ void msg_values(int decode, int64_t len, int64_t tile, DivBy by_tile,
                                           uint32_t flags, int64_t small_max, int64_t& outv,
                                           int64_t& weight) {
  if (len < 0) len = 0;
  outv = decode ? (int64_t)decoded_cap_flags((uint64_t)len, flags)
                : (int64_t)encoded_len_flags((uint64_t)len, flags);
  weight = msg_weight(len, msg_tiles(len, tile, by_tile, small_max));
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

// One scan block's totals as the blocks after it see them: flag = the
// call's number * 4 + kPartAgg (its own totals are published) or kPartInc
// (its inclusive prefix is published too).
struct ScanPart {
  unsigned long long flag;
  int64_t agg_o, agg_w, inc_o, inc_w;
};
constexpr unsigned long long kPartAgg = 1, kPartInc = 2;

// The prefix sum of (output length, weight) in one pass (a decoupled
// look-back): each CTA scans its 2,048 messages, publishes their totals, and
// its first warp adds up the totals of the blocks before its own, 32 at a
// time, walking back until it meets a published inclusive prefix; then
// every message's offsets are written (and, decoding, first_bad and outlen
// cleared). The flags carry the call's number (epoch), so the scratch needs
// no clearing. A block waits only on lower-numbered blocks, which the
// hardware starts first (and batches of up to about a million messages fit
// the GPU at once); the waits are bounded by wait_ns all the same, and one
// that runs out sets the fault word (the calls then report
// B64_ERR_TIMEOUT) and leaves the offsets unwritten.
__global__ void __launch_bounds__(kScanThreads)
    k_scan_onepass(const int64_t* __restrict__ in_off, int64_t nmsg, int decode, int64_t tile,
                   uint32_t flags, int64_t small_max, int64_t* __restrict__ out_off,
                   int64_t* __restrict__ weight_off, volatile ScanPart* parts,
                   unsigned long long epoch, int64_t* __restrict__ first_bad,
                   int64_t* __restrict__ outlen, uint64_t wait_ns) {
  __shared__ int64_t s_base_o, s_base_w;
  __shared__ uint32_t s_ok;
  const int64_t blk = blockIdx.x;
  const int64_t base = blk * kScanPerBlock + (int64_t)threadIdx.x * kScanItems;
  const DivBy by_tile = DivBy::of(tile);
  int64_t vo[kScanItems], vw[kScanItems];
  int64_t so = 0, sw = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    vo[i] = vw[i] = 0;
    if (j < nmsg)
      msg_values(decode, in_off[j + 1] - in_off[j], tile, by_tile, flags, small_max, vo[i],
                 vw[i]);
    so += vo[i];
    sw += vw[i];
  }
  int64_t eo = so, ew = sw, to, tw;
  block_exclusive_scan2(eo, ew, to, tw);
  if (threadIdx.x < 32) {  // warp 0: publish, then look back 32 blocks at a time
    const uint32_t lane = threadIdx.x;
    const unsigned long long tagged = epoch << 2;
    volatile ScanPart* me = parts + blk;
    if (lane == 0 && blk > 0) {
      me->agg_o = to;
      me->agg_w = tw;
      __threadfence();
      me->flag = tagged | kPartAgg;
    }
    int64_t ex_o = 0, ex_w = 0;
    bool ok = true;
    const uint64_t t0 = global_timer_ns();
    for (int64_t q = blk - 1; q >= 0; q -= 32) {
      const int64_t mine = q - (int64_t)lane;  // lanes see blocks q, q - 1, .., q - 31
      const bool valid = mine >= 0;
      unsigned long long f = 0;
      for (;;) {  // until every block of the window has published
        if (valid) f = parts[mine].flag;
        if (__all_sync(0xFFFFFFFFu, !valid || (f & ~3ull) == tagged)) break;
        if (__any_sync(0xFFFFFFFFu, global_timer_ns() - t0 > wait_ns)) {
          ok = false;
          break;
        }
      }
      if (!ok) break;
      __threadfence();
      // the nearest block with its inclusive prefix published ends the walk
      const uint32_t inc = __ballot_sync(0xFFFFFFFFu, valid && (f & 3ull) == kPartInc);
      const uint32_t stop = inc ? (uint32_t)(__ffs(inc) - 1) : 32u;
      int64_t vo = 0, vw = 0;
      if (valid && lane < stop) {
        vo = parts[mine].agg_o;
        vw = parts[mine].agg_w;
      } else if (valid && lane == stop) {
        vo = parts[mine].inc_o;
        vw = parts[mine].inc_w;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        vo += __shfl_down_sync(0xFFFFFFFFu, vo, d);
        vw += __shfl_down_sync(0xFFFFFFFFu, vw, d);
      }
      ex_o += __shfl_sync(0xFFFFFFFFu, vo, 0);
      ex_w += __shfl_sync(0xFFFFFFFFu, vw, 0);
      if (inc) break;
    }
    if (lane == 0) {
      me->inc_o = ex_o + to;
      me->inc_w = ex_w + tw;
      __threadfence();
      me->flag = tagged | kPartInc;
      s_base_o = ex_o;
      s_base_w = ex_w;
      s_ok = ok ? 1u : 0u;
      if (!ok) atomicOr(&g_batch_fault, 1u);
    }
  }
  __syncthreads();
  if (!s_ok) return;
  eo += s_base_o;
  ew += s_base_w;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = base + i;
    eo += vo[i];
    ew += vw[i];
    if (j < nmsg) {
      out_off[j + 1] = eo;
      weight_off[j + 1] = ew;
      if (first_bad) first_bad[j] = kNoBad;
      if (outlen) outlen[j] = 0;
    }
  }
  if (blk == 0 && threadIdx.x == 0) {
    out_off[0] = 0;
    weight_off[0] = 0;
  }
}

// ------------------------------------------------------------ tile walk
// One message as a tile sees it: its bytes and its output. Aligned-word
// reads near its ends stay within the bounds its batch gives (lo, hi).
struct Msg {
  const uint8_t* src;
  int64_t len;
  uint8_t* out;
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
    return Msg{src + m0, __ldg(in_off + j + 1) - m0, dst + __ldg(out_off + j)};
  }
  // the packed input buffer
  __device__ __forceinline__ const uint8_t* lo(const Msg&) const { return src; }
  __device__ __forceinline__ const uint8_t* hi(const Msg&) const { return src_hi; }
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
    return Msg{d.src, d.len, dst + d.out_off};
  }
  // the message itself
  __device__ __forceinline__ const uint8_t* lo(const Msg& m) const { return m.src; }
  __device__ __forceinline__ const uint8_t* hi(const Msg& m) const { return m.src + m.len; }
  __device__ __forceinline__ int64_t len(int64_t j) const { return desc[j].len; }
  __device__ __forceinline__ void prepare(int64_t) {}
};

// Whether a packed decode batch takes the flat decode (k_batch_flat: every
// length a multiple of 4 and a mean length of at least kFlatMinMean
// characters); the flat kernel, the tile walk and the finish kernel decide
// alike.
constexpr int64_t kFlatMinMean = 1024;
template <class Msgs>
__device__ __forceinline__ bool flat_batch(const Msgs&, int64_t) {
  return false;
}
template <>
__device__ __forceinline__ bool flat_batch<PackedMsgs>(const PackedMsgs& ms, int64_t nmsg) {
  if (nmsg <= 0) return false;
  const int64_t M = __ldg(ms.in_off + nmsg), Mo = __ldg(ms.out_off + nmsg);
  return 4 * Mo == 3 * M && M >= kFlatMinMean * nmsg;
}

// ------------------------------------------------------ warp pipeline
// Every warp walks its own share of the tiles (see WalkState below). Tile k
// of message j holds input bytes [t0, t0 + len) of j, t0 = k * tile,
// len <= tile. Staged, the tile's 16-byte-aligned interior is copied into
// the warp's input stage by one bulk copy, issued `stages` tiles ahead;
// stage position o + i holds input byte t0 + i, o being the tile start's
// address mod 16, so positions [ia, ib) are the copied ones. Units whose
// bytes reach outside [ia, ib) read global memory instead. A staged decode
// puts output byte i of the tile at position o2 + i of the warp's output
// buffer (o2 = the output start's address mod 16); the aligned interior
// leaves by one bulk store, the two ragged ends (at most 15 bytes each) by
// byte stores. Encoding, and unstaged, outputs go straight to global memory.
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

// The tile geometry of a launch.
struct TileShape {
  int64_t tile;       // input bytes / characters of a whole tile
  int64_t out_tile;   // its output bytes
  int64_t small_max;  // longest message coded one thread each (0: none)
  DivBy by_tile;      // division by tile
  DivBy by_step;      // division by tile + kTileCost
};

// A warp's walk over its tiles. Warp w of the grid's nw warps owns the
// weight [W*w/nw, W*(w+1)/nw) of the batch's total W and takes the tiles
// that start in it, tile k of message j starting at weight weight_off[j] +
// k * (tile + kTileCost): equal shares of bytes and tiles, whatever the mix
// of lengths (equal tile counts would not be equal work, the last tile of
// a message being short). The walk finds the message of its first tile by
// a search, then moves forward one message at a time, counting each one's
// tiles from its length as the scan did; the offsets arrays are read only
// when it enters the next message.
struct WalkState {
  Msg m;
  int64_t j;       // current message
  int64_t ntiles;  // its tiles
  int64_t k;       // its next tile
  int64_t wk;      // weight offset of tile k
  int64_t w_end;   // end of the warp's share
};

// Starts a walk at message j (found by owner_of_warp for w_begin), at its
// first tile starting at or after w_begin.
template <class Msgs>
__device__ __forceinline__ void walk_begin(WalkState& w, const Msgs& ms, const int64_t* weight_off,
                                           int64_t j, int64_t w_begin, int64_t w_end,
                                           const TileShape& ts) {
  w.j = j;
  w.m = ms.get(j);
  w.ntiles = msg_tiles(w.m.len, ts.tile, ts.by_tile, ts.small_max);
  const int64_t w0 = __ldg(weight_off + j);
  w.k = ts.by_step(w_begin - w0 + ts.tile + kTileCost - 1);
  w.wk = w0 + w.k * (ts.tile + kTileCost);
  w.w_end = w_end;
}

// The view of the walk's next tile; false when the warp's share is done.
template <class Msgs>
__device__ __forceinline__ bool walk_next(WalkState& w, const Msgs& ms, int64_t nmsg,
                                          const TileShape& ts, TileView& v) {
  const int64_t tile = ts.tile;
  while (w.k >= w.ntiles) {  // on to the next message with tiles
    // tile k (= ntiles) would start where the message's weight ends, less
    // the last tile's shortfall from a whole tile
    w.wk -= w.ntiles ? w.ntiles * tile - w.m.len : 0;
    if (++w.j >= nmsg) return false;
    w.m = ms.get(w.j);
    w.ntiles = msg_tiles(w.m.len, tile, ts.by_tile, ts.small_max);
    w.k = 0;
  }
  if (w.wk >= w.w_end) return false;
  const Msg m = w.m;
  const int64_t k = w.k++;
  w.wk += tile + kTileCost;
  v.msrc = m.src;
  v.mout = m.out;
  v.lo = ms.lo(m);
  v.hi = ms.hi(m);
  v.dst = m.out + k * ts.out_tile;
  v.t0 = k * tile;
  v.mlen = m.len;
  v.j = w.j;
  v.len = (uint32_t)tmin<int64_t>(tile, m.len - v.t0);
  const uintptr_t s = reinterpret_cast<uintptr_t>(m.src + v.t0);
  const uintptr_t a = (s + 15u) & ~(uintptr_t)15u, b = (s + v.len) & ~(uintptr_t)15u;
  v.o = (uint32_t)(s & 15u);
  v.ia = v.o ? 16u : 0u;
  v.ib = b > a ? v.ia + (uint32_t)(b - a) : v.ia;
  return true;
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

// The batched encoders code each 12-bit half of a group with one lookup in
// a table of character pairs: entry v holds the characters of the 6-bit
// values v >> 6 (low byte) and v & 63 (high byte). The pairs follow the
// 64-character alphabet in each encoding kernel's table (kEncTableBytes in
// all), so a coder handed the alphabet T finds them at T + 64. Two 16-bit
// lookups and two field extractions per group take the place of four byte
// lookups and four extractions: Algorithm 1's map B applied to two values
// at once, the trade of a larger table for fewer shifts and masks that
// Section 2.2 describes for scalar encoders.
constexpr uint32_t kEncTableBytes = 64u + 2u * 4096u;

__device__ __forceinline__ void init_enc_pairs(uint8_t* T, bool url) {
  uint16_t* P = reinterpret_cast<uint16_t*>(T + 64);
  for (uint32_t v = threadIdx.x; v < 4096u; v += blockDim.x)
    P[v] = (uint16_t)(alphabet_char(v >> 6, url) | (alphabet_char(v & 63u, url) << 8));
  for (uint32_t v = threadIdx.x; v < 64u; v += blockDim.x) T[v] = (uint8_t)alphabet_char(v, url);
  __syncthreads();
}

// One group (three bytes big-endian in bits 23..0; bits above 23 are
// ignored) -> four characters, first in the low byte.
__device__ __forceinline__ uint32_t enc_group_pairs(uint32_t g, const uint8_t* T) {
  const uint8_t* P = T + 64;
  const uint32_t a = *reinterpret_cast<const uint16_t*>(P + ((g >> 11) & 0x1FFEu));
  const uint32_t b = *reinterpret_cast<const uint16_t*>(P + ((g << 1) & 0x1FFEu));
  return __byte_perm(a, b, 0x5410);
}

// Stream bytes x0..x11 in little-endian words w0, w1, w2 -> 16 characters.
__device__ __forceinline__ uint4 enc_unit_pairs(uint32_t w0, uint32_t w1, uint32_t w2,
                                                const uint8_t* T) {
  uint4 o;
  o.x = enc_group_pairs(__byte_perm(w0, 0u, 0x4012), T);  // x0 x1 x2
  o.y = enc_group_pairs(__byte_perm(w0, w1, 0x3345), T);  // x3 x4 x5
  o.z = enc_group_pairs(__byte_perm(w1, w2, 0x2234), T);  // x6 x7 x8
  o.w = enc_group_pairs(__byte_perm(w2, 0u, 0x4123), T);  // x9 x10 x11
  return o;
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
    st_global_v4_cs(db + 16 * i, enc_unit_pairs(x, y, z, T));
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
        st_global_v4_cs(db + 16 * i, enc_unit_pairs(x, y, z, T));
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
      const uint4 e = enc_unit_pairs(w.x, w.y, w.z, T);
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
        c = enc_unit_pairs(w.x, w.y, w.z, T);
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
      if (u0 + k < nu) store16_any(d + 16 * (u0 + k), enc_unit_pairs(w[k].x, w[k].y, w[k].z, T));
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
                     reinterpret_cast<unsigned long long*>(first_bad + j), outlen + j, flags,
                     ms.lo(m), ms.hi(m));
    } else {
      encode_message(m.src, m.len, m.out, table, flags, ms.lo(m), ms.hi(m));
    }
  }
}

// Shared memory of a warp (staged tiles): `stages` input stages and, for
// decode, one output buffer.
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

// The share [w_begin, w_end) of the batch's weight that warp w of the
// grid's nw warps codes.
__device__ __forceinline__ void warp_share(const int64_t* weight_off, int64_t nmsg, int64_t w,
                                           int64_t nw, int64_t& w_begin, int64_t& w_end) {
  const int64_t total = __ldg(weight_off + nmsg);
  w_begin = total * w / nw;
  w_end = total * (w + 1) / nw;
}

// The persistent kernel of both directions with staged tiles. Lane 0 of a
// warp walks its tiles, issuing each one's bulk copy `stages` tiles ahead
// and leaving its view beside the stage; the warp codes the staged tiles
// in order.
template <int NT, int DECODE, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_code(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ weight_off, TileShape ts,
                 uint32_t stages, int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen,
                 uint32_t flags, WaitTest wt) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(16) uint8_t table[DECODE ? 256 : kEncTableBytes];
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
    init_enc_pairs(table, flags & kFlagUrl);
  }
  const uint32_t in_b = stage_in_bytes(ts.tile);
  uint8_t* wbase = smem + (size_t)warp * warp_smem_bytes(DECODE, ts.tile, S);
  uint8_t* obase = wbase + S * in_b;  // decode: the output buffer

  int64_t w_begin, w_end;
  warp_share(weight_off, nmsg, (int64_t)blockIdx.x * (NT / 32) + warp,
             (int64_t)gridDim.x * (NT / 32), w_begin, w_end);
  Msgs ms = msgs;
  ms.prepare(nmsg);
  WalkState& walk = walks[warp];  // used by lane 0
  uint32_t primed = 0;            // tiles issued before the loop (lane 0)
  bool more = false;              // the walk may have further tiles (lane 0)
  if (w_begin < w_end) {          // the first tiles' copies go out first
    const int64_t j0 = owner_of_warp(weight_off, nmsg, w_begin, lane);
    if (lane == 0) {
      walk_begin(walk, ms, weight_off, j0, w_begin, w_end, ts);
      TileView v;
      // (test stall: the grid's first warp leaves out its first copy)
      const bool stall = wt.stall && blockIdx.x == 0 && warp == 0;
      while (primed < S && walk_next(walk, ms, nmsg, ts, v)) {
        meta[warp][primed] = v;
        if (!(stall && primed == 0)) issue_tile(v, wbase + primed * in_b, &full[warp][primed]);
        ++primed;
      }
      more = primed == S;
    }
  }
  // short messages (no tiles) while those copies are in flight
  if (ts.small_max > 0)
    code_short_messages<DECODE>(ms, nmsg, ts.small_max, table, first_bad, outlen, flags);
  uint32_t pending = __shfl_sync(0xFFFFFFFFu, primed, 0);  // tiles issued, not yet coded
  if (pending == 0) return;

  bool timed_out = false, first = true;
  uint32_t s = 0, phase = 0;
  while (pending > 0) {
    uint8_t* in = wbase + s * in_b;
    const bool ok = mbar_wait_backoff(&full[warp][s], phase, wt.limit_ns);
    if (__any_sync(0xFFFFFFFFu, !ok)) {
      timed_out = true;
      break;
    }
    const TileView v = meta[warp][s];
    if (DECODE) {
      // the previous tile's bulk store has finished reading the output buffer
      if (lane == 0 && !first) bulk_wait_read(0);
      __syncwarp();
      decode_tile<false>(v, in, obase, table,
                         reinterpret_cast<unsigned long long*>(first_bad + v.j), outlen + v.j,
                         lane, flags);
    } else {
      encode_tile<false>(v, in, table, lane, flags);
      fence_proxy_async_smem();  // the stage's reads come before its next copy
      __syncwarp();
    }
    uint32_t issued = 0;
    if (lane == 0 && more) {
      TileView nv;
      more = walk_next(walk, ms, nmsg, ts, nv);
      if (more) {
        meta[warp][s] = nv;
        issue_tile(nv, in, &full[warp][s]);
        issued = 1;
      }
    }
    pending = pending - 1 + __shfl_sync(0xFFFFFFFFu, issued, 0);
    first = false;
    if (++s == S) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (timed_out && lane == 0) {
    atomicOr(&g_batch_fault, 1u);
    // wait (bounded) for the copies still in flight into this warp's stages
    for (uint32_t i = 0; i < pending; ++i) {
      mbar_wait_bounded(&full[warp][s], phase, 500000000ull);
      if (++s == S) {
        s = 0;
        phase ^= 1u;
      }
    }
  }
  if (DECODE && lane == 0) bulk_wait_all();
}

// The same walk without staging: every lane keeps the walk in registers
// (one warp-instruction each, as on one lane), and the tiles' units move
// straight between global memory and registers, so a warp needs no shared
// memory, barrier or copy engine, and a tile may be longer than a stage
// could hold. after_flat: k_batch_flat ran before; a batch it decoded is
// left alone.
template <int NT, int DECODE, class Msgs>
__global__ void __launch_bounds__(NT)
    k_batch_direct(Msgs msgs, int64_t nmsg, const int64_t* __restrict__ weight_off, TileShape ts,
                   int64_t* __restrict__ first_bad, int64_t* __restrict__ outlen, uint32_t flags,
                   uint32_t after_flat) {
  __shared__ __align__(16) uint8_t table[DECODE ? 256 : kEncTableBytes];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (after_flat && (DECODE ? flat_batch(msgs, nmsg) : flat_enc_batch(msgs, nmsg))) return;
  if (DECODE) {
    init_tables(nullptr, table, flags & kFlagUrl);
  } else {
    init_enc_pairs(table, flags & kFlagUrl);
  }
  int64_t w_begin, w_end;
  warp_share(weight_off, nmsg, (int64_t)blockIdx.x * (NT / 32) + warp,
             (int64_t)gridDim.x * (NT / 32), w_begin, w_end);
  Msgs ms = msgs;
  ms.prepare(nmsg);
  if (ts.small_max > 0)
    code_short_messages<DECODE>(ms, nmsg, ts.small_max, table, first_bad, outlen, flags);
  if (w_begin >= w_end) return;
  WalkState walk;
  walk_begin(walk, ms, weight_off, owner_of_warp(weight_off, nmsg, w_begin, lane), w_begin, w_end,
             ts);
  for (;;) {
    TileView v;
    if (!walk_next(walk, ms, nmsg, ts, v)) break;
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

// ------------------------------------------------------------ flat decode
// A packed decode batch whose lengths are all multiples of 4 (every padded
// encoding) has message j's output at exactly 3/4 of its input offset (the
// capacities 3 floor(m / 4) sum to 3/4 of the characters then, and only
// then), so the whole batch decodes as one buffer: Algorithm 2 on every
// quad, by the single-buffer pipeline (one CTA of 512 threads per SM, each
// CTA a contiguous run of 60 Ki-character tiles staged by TMA two ahead,
// decoded units staged and stored by TMA). Only the last quad of a message,
// its final group (where '=' may stand), depends on the message: the finish
// kernel writes its bytes and checks its rules. Warp 0 issues the copies
// and marks, in a bitmask beside each stage, the final quads of the
// messages that end in that tile; a unit that flags a character in a
// marked quad is no error, any other flagged character is reported at its
// offset in its message. Batches of shorter messages (mean below
// kFlatMinMean characters: many ends per tile) and all others are left to
// the tile walk (k_batch_direct), which checks the same condition.
constexpr int kFlatThreads = 512;
constexpr uint32_t kFlatUnits = 8;  // 16-character units per decoding thread per tile
// warps 1.. decode (warp 0 issues), each of their threads kFlatUnits units
constexpr uint32_t kFlatTile = (uint32_t)(kFlatThreads - 32) * kFlatUnits * 16u;  // 61,440
constexpr uint32_t kFlatOut = kFlatTile / 4u * 3u;
constexpr uint32_t kFlatStages = 2;
constexpr uint32_t kFlatMaskWords = kFlatTile / 4u / 32u;  // one bit per quad

__host__ __device__ constexpr size_t flat_smem_bytes() {
  return (size_t)kFlatStages * kFlatTile + 2 * (size_t)kFlatOut;
}

// Whether a packed encode batch takes the flat encode (k_batch_flat_enc:
// padded output, so every message's characters start on a quad, and a mean
// output length of at least kFlatMinMean characters; the host checks the
// flags and the alignments); k_batch_flat_enc and the tile walk decide
// alike.
template <class Msgs>
__device__ __forceinline__ bool flat_enc_batch(const Msgs&, int64_t) {
  return false;
}
template <>
__device__ __forceinline__ bool flat_enc_batch<PackedMsgs>(const PackedMsgs& ms, int64_t nmsg) {
  return nmsg > 0 && __ldg(ms.out_off + nmsg) >= kFlatMinMean * nmsg;
}

// The first message j whose end in_off[j + 1] exceeds x (x < in_off[nmsg]),
// by the whole warp: each round probes 32 evenly spaced ends of the span
// left and keeps the part between the last one at most x and the first one
// above it (about five rounds for a million messages).
__device__ __forceinline__ int64_t first_end_after(const int64_t* in_off, int64_t nmsg, int64_t x,
                                                   uint32_t lane) {
  int64_t lo = 0, hi = nmsg - 1;
  while (hi > lo) {
    const int64_t span = hi - lo;
    const bool above = __ldg(in_off + lo + span * lane / 32 + 1) > x;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, above);
    if (b == 0) {
      lo = lo + span * 31 / 32 + 1;
    } else {
      const int64_t f = __ffs(b) - 1;
      const int64_t nlo = f ? lo + span * (f - 1) / 32 + 1 : lo;
      hi = lo + span * f / 32;
      lo = nlo;
    }
  }
  return lo;
}

// A unit of a flat tile that flagged a character (quads q0 .. q0 + 3 of the
// tile): each flagged quad that is not a marked final quad holds an invalid
// character; its first one goes to its message's first_bad.
__device__ __noinline__ void flat_flagged(uint4 v, uint32_t q0, const uint32_t* mask, int64_t T0,
                                          int64_t j_lo, const int64_t* in_off, int64_t nmsg,
                                          int64_t* first_bad, const uint8_t* D) {
  for (uint32_t q = 0; q < 4; ++q) {
    const uint32_t qi = q0 + q;
    if ((mask[qi >> 5] >> (qi & 31u)) & 1u) continue;
    const uint32_t x = word_of(v, q);
    for (uint32_t i = 0; i < 4; ++i) {
      if (D[(x >> (8u * i)) & 0xFFu] & kBadFlag) {
        const int64_t p = T0 + 4 * (int64_t)qi + i;
        int64_t lo = j_lo, hi = nmsg - 1;  // the first message ending after p
        while (lo < hi) {
          const int64_t mid = lo + (hi - lo) / 2;
          if (__ldg(in_off + mid + 1) > p) hi = mid; else lo = mid + 1;
        }
        atomicMin(reinterpret_cast<unsigned long long*>(first_bad + lo),
                  (unsigned long long)(p - __ldg(in_off + lo)));
        break;
      }
    }
  }
}

// One tile's place beside its stage (written by warp 0 before the arrive
// that publishes it).
struct FlatTile {
  int64_t T0;    // first character
  int64_t j_lo;  // first message ending after T0
  uint32_t len;  // characters
};

__global__ void __launch_bounds__(kFlatThreads, 1)
    k_batch_flat(PackedMsgs ms, int64_t nmsg, int64_t* __restrict__ first_bad, uint32_t flags,
                 WaitTest wt) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t D[256];
  __shared__ __align__(8) uint64_t full[kFlatStages];
  __shared__ FlatTile meta[kFlatStages];
  __shared__ uint32_t fmask[kFlatStages][kFlatMaskWords];
  constexpr int NT = kFlatThreads;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (!flat_batch(ms, nmsg)) return;  // the tile walk decodes the batch
  if (tid == 0) {  // two arrivals per phase: the copy's (with its bytes), then the mask's
    for (uint32_t s = 0; s < kFlatStages; ++s) mbar_init(&full[s], 2);
    fence_mbar_init();
  }
  init_tables(nullptr, D, flags & kFlagUrl);
  __syncthreads();
  const int64_t M = __ldg(ms.in_off + nmsg);
  const int64_t ntiles = (M + kFlatTile - 1) / kFlatTile;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t tb = tmin<int64_t>(ntiles, (int64_t)blockIdx.x * per);
  const int64_t te = tmin<int64_t>(ntiles, tb + per);
  if (tb >= te) return;
  uint8_t* outbuf0 = smem + (size_t)kFlatStages * kFlatTile;

  // warp 0: the first message ending after the next tile to issue, and the
  // lane's two offsets pairs of the walk's next round, loaded ahead (their
  // latency then passes while warp 0 waits for the tile in between)
  int64_t jw = 0;
  int64_t pe[2], pb[2];
  auto prefetch = [&]() {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t jj = jw + 32 * h + lane;
      pe[h] = INT64_MAX;
      pb[h] = 0;
      if (jj < nmsg) {
        pb[h] = __ldg(ms.in_off + jj);
        pe[h] = __ldg(ms.in_off + jj + 1);
      }
    }
  };
  if (warp == 0) {
    jw = first_end_after(ms.in_off, nmsg, tb * (int64_t)kFlatTile, lane);
    prefetch();
  }
  // by all of warp 0: lane 0 issues tile t's copy, then the warp marks the
  // final quads of the messages that end in the tile (two rounds of 32
  // messages per step) while the copy is in flight, and lane 0 arrives a
  // second time, which publishes the mask and the tile's place
  auto issue = [&](int64_t t, uint32_t s) {
    const int64_t T0 = t * (int64_t)kFlatTile;
    const uint32_t len = (uint32_t)tmin<int64_t>(kFlatTile, M - T0);
    const int64_t T1 = T0 + len;
    const bool stall = wt.stall && blockIdx.x == 0 && t == tb;  // test: no copy, no arrivals
    if (lane == 0 && !stall) {
      const uint32_t bytes = len & ~15u;
      if (bytes) {
        fence_proxy_async_smem();  // earlier generic reads of this stage come first
        mbar_arrive_expect_tx(&full[s], bytes);
        tma_load_1d(smem + (size_t)s * kFlatTile, ms.src + T0, bytes, &full[s]);
      } else {
        mbar_arrive(&full[s]);
      }
    }
    for (uint32_t i = lane; i < kFlatMaskWords; i += 32) fmask[s][i] = 0u;
    __syncwarp();
    const int64_t j_lo = jw;
    for (;;) {  // pe, pb hold the round's offsets (for messages jw ..)
      int n = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool inside = pe[h] <= T1;
        if (inside && pe[h] > pb[h]) {
          const uint32_t qi = (uint32_t)(pe[h] - 4 - T0) >> 2;
          atomicOr(&fmask[s][qi >> 5], 1u << (qi & 31u));
        }
        n += __popc(__ballot_sync(0xFFFFFFFFu, inside));
      }
      jw += n;
      prefetch();  // the next round's, or the next tile's first round
      if (n < 64) break;
    }
    __syncwarp();
    if (lane == 0) {
      meta[s] = FlatTile{T0, j_lo, len};
      if (!stall) mbar_arrive(&full[s]);
    }
  };
  if (warp == 0) {
    fence_proxy_async_smem();
    for (uint32_t s = 0; s < kFlatStages && tb + s < te; ++s) issue(tb + s, s);
  }

  bool timed_out = false;
  uint32_t k = 0;
  for (int64_t t = tb; t < te; ++t, ++k) {
    const uint32_t s = k % kFlatStages;
    const bool ok = mbar_wait_bounded(&full[s], (k / kFlatStages) & 1u, wt.limit_ns);
    uint32_t* ob = reinterpret_cast<uint32_t*>(outbuf0 + (size_t)(k & 1u) * kFlatOut);
    const FlatTile fm = meta[s];
    const uint32_t nu = fm.len / 16u;
    if (ok && warp != 0) {
      const uint4* in = reinterpret_cast<const uint4*>(smem + (size_t)s * kFlatTile);
      // flagged units (mostly padded final quads) are looked at after the
      // loop, which then has no call in it
      uint32_t flagged = 0;
#pragma unroll
      for (uint32_t i = 0; i < kFlatUnits; ++i) {
        const uint32_t u = tid - 32u + (NT - 32) * i;
        if (u < nu) {
          uint32_t err = 0;
          const uint3 o = dec_unit(in[u], D, err);
          ob[3 * u] = o.x;
          ob[3 * u + 1] = o.y;
          ob[3 * u + 2] = o.z;
          if (err & kBadFlag) flagged |= 1u << i;
        }
      }
      while (flagged) {
        const uint32_t i = __ffs(flagged) - 1;
        flagged &= flagged - 1;
        const uint32_t u = tid - 32u + (NT - 32) * i;
        flat_flagged(in[u], 4u * u, fmask[s], fm.T0, fm.j_lo, ms.in_off, nmsg, first_bad, D);
      }
      // whole quads after the last unit (the last tile of the batch only)
      const uint32_t nq = (fm.len - 16u * nu) / 4u;
      if (tid - 32u < nq) {
        const uint32_t qi = 4u * nu + (tid - 32u);
        const int64_t p = fm.T0 + 4 * (int64_t)qi;
        const uint32_t x = *reinterpret_cast<const uint32_t*>(ms.src + p);
        uint32_t err = 0;
        const uint32_t val = dec_quad(x, D, err);
        if (!(err & kBadFlag)) {
          uint8_t* w = ms.dst + p / 4 * 3;
          w[0] = (uint8_t)(val >> 16);
          w[1] = (uint8_t)(val >> 8);
          w[2] = (uint8_t)val;
        } else {
          flat_flagged(make_uint4(x, 0x41414141u, 0x41414141u, 0x41414141u), qi, fmask[s],
                       fm.T0, fm.j_lo, ms.in_off, nmsg, first_bad, D);
        }
      }
    }
    fence_proxy_async_smem();
    if (tid == 0) bulk_wait_read_all();  // the other output buffer is free again
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      if (tid == 0) {  // wait (bounded) for this CTA's copies in flight
        for (uint32_t jx = 0; jx < kFlatStages; ++jx) {
          const uint32_t kk = k + jx;
          const int64_t tt = t + jx;
          if (tt < te && !(wt.stall && blockIdx.x == 0 && tt == tb))
            mbar_wait_bounded(&full[kk % kFlatStages], (kk / kFlatStages) & 1u, 500000000ull);
        }
      }
      break;
    }
    if (warp == 0) {
      if (lane == 0) {
        const uint32_t ob_bytes = 12u * nu;
        const uint32_t sb = ob_bytes & ~15u;
        uint8_t* gout = ms.dst + fm.T0 / 4 * 3;
        if (sb) {
          tma_store_1d(gout, ob, sb);
          bulk_commit();
        }
        const uint8_t* obb = reinterpret_cast<const uint8_t*>(ob);
        for (uint32_t i = sb; i < ob_bytes; ++i) gout[i] = obb[i];
      }
      const int64_t t2 = t + kFlatStages;
      if (t2 < te) issue(t2, s);
    }
  }
  if (tid == 0) {
    bulk_wait_all();
    if (timed_out) atomicOr(&g_batch_fault, 1u);
  }
}

// ------------------------------------------------------------ flat encode
// The same idea for encoding. With padding, message j's characters start
// on a quad (out_off[j] = 4 qs_j) and quad q of it encodes input bytes
// 3 q + d_j (d_j = in_off[j] - 3 qs_j): so the batch's output is one flat
// sequence of quads, and the input of an output tile is one contiguous
// range. Each CTA takes a contiguous run of output tiles of 53,760
// characters; warp 0 stages each tile's input range by TMA and lists in a
// segment table beside it the messages that overlap the tile (first and
// end quad, shift, bytes of the last group); the other warps encode
// 16-character units, a unit inside one message, short of its last quad,
// from 12 staged bytes (Algorithm 1's main loop), any other unit quad by
// quad with the message's last group padded (Algorithm 1's tail). The
// characters go straight to global memory in aligned 16-byte stores (the
// tile's output starts on 16 bytes), four tiles' input staged ahead.
constexpr uint32_t kFlatEncUnits = 7;
constexpr uint32_t kFlatEncTile = (uint32_t)(kFlatThreads - 32) * kFlatEncUnits * 16u;  // 53,760
constexpr uint32_t kFlatEncQuads = kFlatEncTile / 4u;
// a tile's input, at most 3 bytes per quad, after up to 15 bytes of alignment
// and before the 16 bytes a unit's word reads may pass its last byte
constexpr uint32_t kFlatEncStage = (kFlatEncQuads * 3u + 32u + 127u) & ~127u;
constexpr uint32_t kFlatMaxSegs = 512;
constexpr uint32_t kFlatEncStages = 4;

__host__ __device__ constexpr size_t flat_enc_smem_bytes() {
  return (size_t)kFlatEncStages * kFlatEncStage +
         (size_t)kFlatEncStages * kFlatMaxSegs * sizeof(int4);
}

// One message as a tile sees it: quads [qs, qe) relative to the tile's
// first quad, stage position 3 q + sd of quad q's first byte, and the
// bytes of its last group (1..3).
__device__ __forceinline__ int4 flat_seg(int32_t qs, int32_t qe, int32_t sd, int32_t last) {
  return make_int4(qs, qe, sd, last);
}

// A tile's place beside its stage (written by warp 0 before the arrive that
// publishes it).
struct FlatEncTile {
  int64_t Q0;      // first quad
  int64_t G;       // input offset of stage byte 0 (16-byte aligned)
  int64_t j_cut;   // first message not in the segment table (nmsg: none)
  uint32_t nq;     // quads
  uint32_t nseg;   // segments listed
  uint32_t ia, ib; // staged bytes
};

// The message of quad q (absolute) among [lo, nmsg): quads of message j are
// [out_off[j] / 4, out_off[j + 1] / 4).
__device__ __forceinline__ int64_t flat_msg_of_quad(const int64_t* out_off, int64_t nmsg,
                                                    int64_t lo, int64_t q) {
  int64_t hi = nmsg - 1;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (__ldg(out_off + mid + 1) > 4 * q) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Quads [q0, q1) of a tile (relative), one at a time: the message's shift
// from the segment table (or, past the table's cut, from the offsets), its
// bytes from the stage when staged, else from global memory, encoded with
// the tail rule of its last group; the characters to ob (the tile's output).
__device__ __noinline__ void flat_enc_quads(const FlatEncTile fm, const int4* segs, uint32_t k,
                                            uint32_t q0, uint32_t q1, const uint8_t* st,
                                            const PackedMsgs ms, int64_t nmsg, uint32_t* ob,
                                            const uint8_t* T) {
  for (uint32_t q = q0; q < q1; ++q) {
    int64_t in;
    uint32_t cnt = 3;
    const int64_t qa = fm.Q0 + q;
    int4 sg = make_int4(0, 0, 0, 0);
    bool found = false;
    while (k < fm.nseg) {
      sg = segs[k];
      if ((uint32_t)sg.y > q) {
        found = (uint32_t)max(sg.x, 0) <= q;
        break;
      }
      ++k;
    }
    if (found) {
      in = fm.G + 3 * (int64_t)q + sg.z;
      if (q + 1 == (uint32_t)sg.y) cnt = (uint32_t)sg.w;
    } else {  // past the table's cut: the offsets
      const int64_t j = flat_msg_of_quad(ms.out_off, nmsg, fm.j_cut, qa);
      const int64_t qs = __ldg(ms.out_off + j) / 4, qe = __ldg(ms.out_off + j + 1) / 4;
      const int64_t i0 = __ldg(ms.in_off + j), n = __ldg(ms.in_off + j + 1) - i0;
      in = i0 + 3 * (qa - qs);
      if (qa + 1 == qe) cnt = (uint32_t)(n - 3 * (qe - 1 - qs));
    }
    uint32_t b[3] = {0, 0, 0};
    const int64_t sp = in - fm.G;
    for (uint32_t i = 0; i < cnt; ++i) {
      const int64_t x = sp + i;
      b[i] = (x >= fm.ia && x < fm.ib) ? st[x] : ms.src[in + i];
    }
    ob[q] = enc_tail_group(b[0], b[1], b[2], cnt, T);
  }
}

__global__ void __launch_bounds__(kFlatThreads, 1)
    k_batch_flat_enc(PackedMsgs ms, int64_t nmsg, uint32_t flags, WaitTest wt) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t T[64];
  __shared__ __align__(8) uint64_t full[kFlatEncStages];
  __shared__ FlatEncTile meta[kFlatEncStages];
  // per stage and row of 32 units: the segment of the row's first quad, and
  // the row's shift when the whole row is one message's, short of its last
  // quad, and staged (kNotSimple otherwise)
  __shared__ uint16_t rowseg[kFlatEncStages][kFlatEncQuads / 128u];
  __shared__ int32_t rowsd[kFlatEncStages][kFlatEncQuads / 128u];
  constexpr int32_t kNotSimple = INT32_MIN;
  constexpr int NT = kFlatThreads;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  if (!flat_enc_batch(ms, nmsg)) return;  // the tile walk encodes the batch
  if (tid == 0) {  // two arrivals per phase: the copy's (with its bytes), then the table's
    for (uint32_t s = 0; s < kFlatEncStages; ++s) mbar_init(&full[s], 2);
    fence_mbar_init();
  }
  init_tables(T, nullptr, flags & kFlagUrl);
  __syncthreads();
  const int64_t N = __ldg(ms.in_off + nmsg);   // input bytes
  const int64_t NQ = __ldg(ms.out_off + nmsg) / 4;  // output quads
  const int64_t ntiles = (NQ + kFlatEncQuads - 1) / kFlatEncQuads;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t tb = tmin<int64_t>(ntiles, (int64_t)blockIdx.x * per);
  const int64_t te = tmin<int64_t>(ntiles, tb + per);
  if (tb >= te) return;
  int4* segs0 = reinterpret_cast<int4*>(smem + (size_t)kFlatEncStages * kFlatEncStage);

  // warp 0: the first message whose quads reach past the next tile's start,
  // and the lane's two messages of the walk's next round, loaded ahead
  int64_t jw = 0;
  int64_t pqs[2], pqe[2], pin[2], pn[2];
  auto prefetch = [&]() {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t jj = jw + 32 * h + lane;
      pqs[h] = pqe[h] = INT64_MAX;
      pin[h] = pn[h] = 0;
      if (jj < nmsg) {
        pqs[h] = __ldg(ms.out_off + jj) / 4;
        pqe[h] = __ldg(ms.out_off + jj + 1) / 4;
        pin[h] = __ldg(ms.in_off + jj);
        pn[h] = __ldg(ms.in_off + jj + 1) - pin[h];
      }
    }
  };
  if (warp == 0) {
    jw = first_end_after(ms.out_off, nmsg, 4 * tb * (int64_t)kFlatEncQuads, lane);
    prefetch();
  }
  // by all of warp 0: the tile's input range (from its first quad's
  // message), lane 0's copy of it, then the segment table while the copy
  // is in flight, and lane 0's second arrival
  auto issue = [&](int64_t t, uint32_t s) {
    const int64_t Q0 = t * (int64_t)kFlatEncQuads;
    const uint32_t nq = (uint32_t)tmin<int64_t>(kFlatEncQuads, NQ - Q0);
    const int64_t Q1 = Q0 + nq;
    // message jw holds quad Q0 (lane 0's prefetched values)
    const int64_t qs0 = __shfl_sync(0xFFFFFFFFu, pqs[0], 0);
    const int64_t in0 = __shfl_sync(0xFFFFFFFFu, pin[0], 0);
    const int64_t inQ0 = in0 + 3 * (Q0 - qs0);
    const int64_t G = inQ0 & ~(int64_t)15;
    const int64_t hi = tmin<int64_t>((inQ0 + 3 * (int64_t)nq + 15) & ~(int64_t)15, N & ~(int64_t)15);
    const uint32_t ib = hi > G ? (uint32_t)(hi - G) : 0u;
    const bool stall = wt.stall && blockIdx.x == 0 && t == tb;  // test: no copy, no arrivals
    if (lane == 0 && !stall) {
      if (ib) {
        fence_proxy_async_smem();  // earlier generic reads of this stage come first
        mbar_arrive_expect_tx(&full[s], ib);
        tma_load_1d(smem + (size_t)s * kFlatEncStage, ms.src + G, ib, &full[s]);
      } else {
        mbar_arrive(&full[s]);
      }
    }
    int4* segs = segs0 + (size_t)s * kFlatMaxSegs;
    uint32_t nseg = 0;
    int64_t j_cut = nmsg;
    for (;;) {  // pqs .. hold the round's messages (jw ..)
      int n = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool take = pqs[h] < Q1 && pqe[h] > pqs[h];  // overlaps the tile, not empty
        const uint32_t bt = __ballot_sync(0xFFFFFFFFu, take);
        const uint32_t k = nseg + __popc(bt & ((1u << lane) - 1u));
        if (take && k < kFlatMaxSegs) {
          const int64_t qs = pqs[h] - Q0, qe = pqe[h] - Q0;
          const int64_t sd = pin[h] - 3 * pqs[h] + 3 * Q0 - G;
          const int32_t last = (int32_t)(pn[h] - 3 * (pqe[h] - 1 - pqs[h]));
          segs[k] = flat_seg((int32_t)tmax<int64_t>(qs, -1), (int32_t)tmin<int64_t>(qe, nq + 1),
                             (int32_t)sd, last);
        }
        const uint32_t cb = __ballot_sync(0xFFFFFFFFu, take && k == kFlatMaxSegs);
        if (cb && j_cut == nmsg) j_cut = jw + 32 * h + (__ffs(cb) - 1);  // (warp-uniform)
        nseg += __popc(bt);
        n += __popc(__ballot_sync(0xFFFFFFFFu, pqe[h] <= Q1));  // ends inside the tile
      }
      jw += n;
      prefetch();  // the next round's, or the next tile's first round
      if (n < 64) break;
    }
    __syncwarp();
    const uint32_t nsg = min(nseg, kFlatMaxSegs);
    // the row table, one row per lane at a time: the last segment starting
    // at or before the row's first quad (no search when the tile holds one
    // message), and the row's shift when it is simple
    const uint32_t nrows = (nq + 127u) / 128u;
    for (uint32_t r = lane; r < nrows; r += 32) {
      const uint32_t qa = 128u * r, qb = qa + 128u;  // the row's quads
      uint32_t lo = 0, hi = nsg;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (segs[mid].x <= (int32_t)qa) lo = mid; else hi = mid;
      }
      const int4 g = segs[lo];
      const bool simple = nsg > 0 && (int32_t)qb < g.y && qb <= nq &&
                          ((3u * (qb - 4u) + (uint32_t)g.z) & ~3u) + 16u <= ib &&
                          (int64_t)3 * qa + g.z >= 0;
      rowseg[s][r] = (uint16_t)lo;
      rowsd[s][r] = simple ? g.z : kNotSimple;
    }
    __syncwarp();
    if (lane == 0) {
      meta[s] = FlatEncTile{Q0, G, j_cut, nq, nsg, 0u, ib};
      if (!stall) mbar_arrive(&full[s]);
    }
  };
  if (warp == 0) {
    fence_proxy_async_smem();
    for (uint32_t s = 0; s < kFlatEncStages && tb + s < te; ++s) issue(tb + s, s);
  }

  bool timed_out = false;
  uint32_t k = 0;
  for (int64_t t = tb; t < te; ++t, ++k) {
    const uint32_t s = k % kFlatEncStages;
    const bool ok = mbar_wait_bounded(&full[s], (k / kFlatEncStages) & 1u, wt.limit_ns);
    const FlatEncTile fm = meta[s];
    uint32_t* ob = reinterpret_cast<uint32_t*>(ms.dst + 4 * fm.Q0);  // the tile's output
    if (ok && warp != 0) {
      const uint8_t* st = smem + (size_t)s * kFlatEncStage;
      const int4* segs = segs0 + (size_t)s * kFlatMaxSegs;
      const uint16_t* rows = rowseg[s];
      const uint32_t nu = (fm.nq + 3u) / 4u;
      // every unit by the main loop's rule (12 staged bytes of one message:
      // its segment from the row table, then at most a step or two), with
      // no branch on the outcome, so that the units' loads overlap; the few
      // units that rule does not fit (a message end or start inside, an
      // unstaged range) are marked and done again quad by quad
      uint32_t redo = 0;
#pragma unroll
      for (uint32_t i = 0; i < kFlatEncUnits; ++i) {
        const uint32_t u = tid - 32u + (NT - 32) * i;
        // a warp's 32 units of a step form one row (480 = 15 rows)
        const int32_t rsd = u < nu ? rowsd[s][u >> 5] : kNotSimple;
        if (rsd != kNotSimple) {  // one message's row: the main loop alone
          const uint32_t sp = 12u * u + (uint32_t)rsd;
          const uint32_t* w = reinterpret_cast<const uint32_t*>(st + (sp & ~3u));
          const uint32_t sh = 8u * (sp & 3u);
          const uint32_t x0 = w[0], x1 = w[1], x2 = w[2], x3 = w[3];
          st_global_v4_cs(reinterpret_cast<uint8_t*>(ob) + 16u * u,
                          enc_unit(__funnelshift_r(x0, x1, sh), __funnelshift_r(x1, x2, sh),
                                   __funnelshift_r(x2, x3, sh), T));
        } else if (u < nu) {
          const uint32_t q = 4u * u;
          uint32_t k = rows[u >> 5];
          while (k + 1 < fm.nseg && segs[k + 1].x <= (int32_t)q) ++k;
          const int4 sg = segs[k];
          const uint32_t sp = 3u * q + (uint32_t)sg.z;
          const uint32_t a = min(sp & ~3u, kFlatEncStage - 16u);  // (stays in the stage)
          const uint32_t* w = reinterpret_cast<const uint32_t*>(st + a);
          const uint32_t sh = 8u * (sp & 3u);
          const uint32_t x0 = w[0], x1 = w[1], x2 = w[2], x3 = w[3];
          const uint4 o = enc_unit(__funnelshift_r(x0, x1, sh), __funnelshift_r(x1, x2, sh),
                                   __funnelshift_r(x2, x3, sh), T);
          const bool fits = sg.x <= (int32_t)q && (int32_t)q + 4 < sg.y && q + 4u <= fm.nq &&
                            (sp & ~3u) + 16u <= fm.ib;
          if (fits) st_global_v4_cs(reinterpret_cast<uint8_t*>(ob) + 16u * u, o);
          else redo |= 1u << i;
        }
      }
      while (redo) {  // quad by quad: each in its message, the last group padded
        const uint32_t i = __ffs(redo) - 1;
        redo &= redo - 1;
        const uint32_t u = tid - 32u + (NT - 32) * i;
        const uint32_t q = 4u * u;
        uint32_t kq = rows[u >> 5];
        for (uint32_t e = 0; e < 4; ++e) {
          const uint32_t qq = q + e;
          if (qq >= fm.nq) break;
          while (kq + 1 < fm.nseg && segs[kq].y <= (int32_t)qq) ++kq;
          const int4 g = segs[kq];
          const uint32_t gp = 3u * qq + (uint32_t)g.z;
          const uint32_t ga = gp & ~3u;
          if (g.x > (int32_t)qq || g.y <= (int32_t)qq || ga + 8u > fm.ib) {
            flat_enc_quads(fm, segs, kq, qq, qq + 1, st, ms, nmsg, ob, T);  // rare
            continue;
          }
          const uint32_t cnt = qq + 1 == (uint32_t)g.y ? (uint32_t)g.w : 3u;
          const uint32_t* w = reinterpret_cast<const uint32_t*>(st + ga);
          uint32_t x = __funnelshift_r(w[0], w[1], 8u * (gp & 3u));
          x &= cnt == 1 ? 0xFFu : cnt == 2 ? 0xFFFFu : 0xFFFFFFu;
          uint32_t c4 = enc_group(__byte_perm(x, 0u, 0x4012), T);
          if (cnt == 1) c4 = (c4 & 0x0000FFFFu) | (kPadChar << 16) | (kPadChar << 24);
          if (cnt == 2) c4 = (c4 & 0x00FFFFFFu) | (kPadChar << 24);
          ob[qq] = c4;
        }
      }
    }
    fence_proxy_async_smem();  // this stage's reads come before its next copy
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      if (tid == 0) {  // wait (bounded) for this CTA's copies in flight
        for (uint32_t jx = 0; jx < kFlatEncStages; ++jx) {
          const uint32_t kk = k + jx;
          const int64_t tt = t + jx;
          if (tt < te && !(wt.stall && blockIdx.x == 0 && tt == tb))
            mbar_wait_bounded(&full[kk % kFlatEncStages], (kk / kFlatEncStages) & 1u,
                              500000000ull);
        }
      }
      break;
    }
    if (warp == 0) {
      const int64_t t2 = t + kFlatEncStages;
      if (t2 < te) issue(t2, s);
    }
  }
  if (tid == 0) {
    bulk_wait_all();
    if (timed_out) atomicOr(&g_batch_fault, 1u);
  }
}

// Per-message status: first bad character wins, then the length rule, then
// Appendix A's check (decoder of the final group returned a negative code).
// While the fault word is set (a tile kernel gave up on a bounded wait, and
// b64_device_fault has not cleared it since), every message reports
// B64_ERR_TIMEOUT: some of them were never decoded.
// after_flat: k_batch_flat ran before; for a batch it decoded, the final
// group of each message is decoded here (its bytes written, its rules
// checked).
template <class Msgs>
__global__ void k_batch_decode_finish(Msgs msgs, int64_t nmsg, int32_t* __restrict__ status,
                                      int64_t* __restrict__ first_bad,
                                      int64_t* __restrict__ outlen, uint32_t flags,
                                      uint32_t after_flat) {
  __shared__ uint8_t D[256];
  const bool flat = after_flat && flat_batch(msgs, nmsg);
  if (flat) {
    init_tables(nullptr, D, flags & kFlagUrl);
    __syncthreads();
  }
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nmsg) return;
  const uint64_t m = (uint64_t)max((long long)0, (long long)msgs.len(j));
  if (*(volatile unsigned int*)&g_batch_fault) {
    status[j] = B64_ERR_TIMEOUT;
    first_bad[j] = (int64_t)m;
    outlen[j] = 0;
    return;
  }
  const uint64_t body_end = decode_body_end(m);
  int64_t final = (body_end < m) ? outlen[j] : 0;
  if (flat && m > 0) {
    const Msg g = msgs.get(j);
    final = dec_final_group(g.src, m, body_end, g.out, D,
                            reinterpret_cast<unsigned long long*>(first_bad + j), flags);
  }
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
  if (c.kernel >= 2) return 0;  // unstaged tiles (and the flat decode's own kernel)
  return (size_t)(c.threads / 32) * warp_smem_bytes(decode, c.tile, (uint32_t)c.stages);
}

cudaError_t batch_offsets(int decode, const int64_t* in_off, int64_t nmsg, int64_t* out_off,
                          int64_t* weight_off, int64_t tile, void* scratch_parts,
                          int64_t* first_bad, int64_t* outlen, cudaStream_t stream,
                          uint32_t flags, int64_t small_max) {
  static std::atomic<unsigned long long> calls{0};
  const unsigned long long epoch = ++calls;  // this call's number (never 0)
  const int64_t nblocks = std::max<int64_t>(1, (nmsg + kScanPerBlock - 1) / kScanPerBlock);
  volatile ScanPart* parts = static_cast<volatile ScanPart*>(scratch_parts);
  k_scan_onepass<<<(unsigned)nblocks, kScanThreads, 0, stream>>>(
      in_off, nmsg, decode, tile, flags, small_max, out_off, weight_off, parts, epoch, first_bad,
      outlen, wait_test().limit_ns);
  return cudaGetLastError();
}

namespace {
// The flat decode needs 16-byte aligned packed input and output (its bulk
// copies); descriptor batches never take it.
bool flat_possible(const PackedMsgs& m) {
  return ((reinterpret_cast<uintptr_t>(m.src) | reinterpret_cast<uintptr_t>(m.dst)) & 15u) == 0;
}
bool flat_possible(const DescMsgs&) { return false; }

// Launches k_batch_flat (one CTA per SM); it returns at once unless the
// batch qualifies.
cudaError_t launch_flat(const PackedMsgs& msgs, int64_t nmsg, int64_t* first_bad,
                        const DeviceInfo* di, uint32_t flags, cudaStream_t stream) {
  int fit = 0;
  cudaError_t e = kernel_prepare(reinterpret_cast<const void*>(k_batch_flat), flat_smem_bytes(),
                                 kFlatThreads, &fit);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  k_batch_flat<<<di->sm_count, kFlatThreads, flat_smem_bytes(), stream>>>(msgs, nmsg, first_bad,
                                                                          flags, wait_test());
  return cudaGetLastError();
}
cudaError_t launch_flat(const DescMsgs&, int64_t, int64_t*, const DeviceInfo*, uint32_t,
                        cudaStream_t) {
  return cudaErrorInvalidValue;
}

// Launches k_batch_flat_enc (one CTA per SM); it returns at once unless the
// batch qualifies.
cudaError_t launch_flat_enc(const PackedMsgs& msgs, int64_t nmsg, const DeviceInfo* di,
                            uint32_t flags, cudaStream_t stream) {
  int fit = 0;
  cudaError_t e = kernel_prepare(reinterpret_cast<const void*>(k_batch_flat_enc),
                                 flat_enc_smem_bytes(), kFlatThreads, &fit);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  k_batch_flat_enc<<<di->sm_count, kFlatThreads, flat_enc_smem_bytes(), stream>>>(
      msgs, nmsg, flags, wait_test());
  return cudaGetLastError();
}
cudaError_t launch_flat_enc(const DescMsgs&, int64_t, const DeviceInfo*, uint32_t, cudaStream_t) {
  return cudaErrorInvalidValue;
}

template <int NT, class Msgs>
cudaError_t launch_work(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* weight_off,
                        int32_t* status, int64_t* first_bad,
                        int64_t* outlen, const BatchConfig& cfg, const DeviceInfo* di,
                        uint32_t flags, cudaStream_t stream, int64_t small_max) {
  // kernel 3: the flat decode or encode when the batch qualifies (padded
  // output, for encode), else the unstaged tiles
  const bool flat =
      cfg.kernel == 3 && flat_possible(msgs) && (decode || !(flags & kFlagNoPad));
  const bool direct = cfg.kernel >= 2;
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
  const TileShape ts{cfg.tile, out_tile_bytes(decode, cfg.tile), small_max, DivBy::of(cfg.tile),
                     DivBy::of(cfg.tile + kTileCost)};
  if (flat) {
    e = decode ? launch_flat(msgs, nmsg, first_bad, di, flags, stream)
               : launch_flat_enc(msgs, nmsg, di, flags, stream);
    if (e != cudaSuccess) return e;
  }
  if (direct) {
    if (decode) {
      k_batch_direct<NT, 1, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, weight_off, ts, first_bad,
                                                           outlen, flags, flat ? 1u : 0u);
    } else {
      k_batch_direct<NT, 0, Msgs><<<grid, NT, 0, stream>>>(msgs, nmsg, weight_off, ts, nullptr,
                                                           nullptr, flags, flat ? 1u : 0u);
    }
  } else if (decode) {
    k_batch_code<NT, 1, Msgs><<<grid, NT, smem, stream>>>(msgs, nmsg, weight_off, ts, stages,
                                                          first_bad, outlen, flags, wait_test());
  } else {
    k_batch_code<NT, 0, Msgs><<<grid, NT, smem, stream>>>(msgs, nmsg, weight_off, ts, stages,
                                                          nullptr, nullptr, flags, wait_test());
  }
  e = cudaGetLastError();
  if (e != cudaSuccess || !decode) return e;
  const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
  k_batch_decode_finish<Msgs><<<(unsigned)blocks, 256, 0, stream>>>(msgs, nmsg, status, first_bad,
                                                                   outlen, flags, flat ? 1u : 0u);
  return cudaGetLastError();
}

template <class Msgs>
cudaError_t launch_work_any(int decode, const Msgs& msgs, int64_t nmsg, const int64_t* weight_off,
                            int32_t* status, int64_t* first_bad,
                            int64_t* outlen, const BatchConfig& cfg, uint32_t flags,
                            cudaStream_t stream, int64_t small_max = 0) {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  switch (cfg.threads) {
    case 128:
      return launch_work<128>(decode, msgs, nmsg, weight_off, status, first_bad, outlen, cfg, di,
                              flags, stream, small_max);
    case 512:
      return launch_work<512>(decode, msgs, nmsg, weight_off, status, first_bad, outlen, cfg, di,
                              flags, stream, small_max);
    default:
      return launch_work<256>(decode, msgs, nmsg, weight_off, status, first_bad, outlen, cfg, di,
                              flags, stream, small_max);
  }
}
}  // namespace

cudaError_t batch_launch_desc(int decode, const MsgDesc* desc, int64_t nmsg, uint8_t* dst,
                              const int64_t* weight_off, int32_t* status, int64_t* first_bad,
                              int64_t* outlen,
                              const BatchConfig& cfg, bool init_results, cudaStream_t stream,
                              uint32_t flags) {
  if (decode && init_results) {
    const int64_t blocks = std::max<int64_t>(1, (nmsg + 255) / 256);
    k_batch_decode_init<<<(unsigned)blocks, 256, 0, stream>>>(nmsg, first_bad, outlen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_work_any(decode, DescMsgs{desc, dst}, nmsg, weight_off, status, first_bad, outlen,
                         cfg, flags, stream);
}

cudaError_t batch_launch(const BatchArgs& a, const BatchConfig& cfg) {
  const int64_t small_max = cfg.kernel != 1 ? batch_small_max(a.decode) : 0;
  cudaError_t e = batch_offsets(a.decode, a.in_off, a.nmsg, a.out_off, a.weight_off, cfg.tile,
                                a.parts, a.decode ? a.first_bad : nullptr,
                                a.decode ? a.outlen : nullptr, a.stream, a.flags, small_max);
  if (e != cudaSuccess) return e;
  // src_hi (the end of the packed input, in_off[nmsg]) is read on the device
  PackedMsgs msgs{a.src, a.in_off, a.dst, a.out_off, nullptr};
  // short messages go one thread each at the start of the tile kernel
  return launch_work_any(a.decode, msgs, a.nmsg, a.weight_off, a.status, a.first_bad, a.outlen,
                         cfg, a.flags, a.stream, small_max);
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
