// Decode with whitespace removal (Appendix B): space, line feed and carriage
// return are dropped before decoding, and the first bad index is reported in
// offsets of the original input.
//
// Fast path, one pass over the data (k_ws_lines): base64 text with
// whitespace is almost always cut into lines of one fixed length L by one
// fixed separator of w = 1 or 2 bytes (MIME: 76 + CR LF, PEM: 64 + LF), and
// may end in a little whitespace. Every CTA derives that line model from the
// first 4 KiB and the last 16 bytes of the input; the k-th kept character is
// then original character k + w * floor(k / L), so the kernel decodes the
// kept characters in place, without compacting them: each tile of kept
// characters has its original span staged in shared memory by one TMA bulk
// copy (issued, with the tile's geometry, by warp 0, which decodes no units
// itself), and each thread of the other warps cuts the separator out of its
// 16 + w byte window (whole-word selects when L is a multiple of 4, byte
// masks otherwise; with no line breaks and an aligned input the window is
// one 16-byte load). The model is checked on every byte of the input: a kept
// position must not hold whitespace (the decode table flags it), a
// separator position must (one short pass per tile over the separators of
// its lines). The kernel is one cooperative launch: after their tiles the
// CTAs meet at a grid barrier, and if any byte broke the model they clear
// the result and decode the input again by the general path below, in the
// same launch; so the result is always that of the general path.
//
// General path (any whitespace; also when the input has no usable line
// model or the output is not 16-byte aligned), over warp tiles of 2048
// characters (64 per lane) that each warp works on alone, its phases
// between grid barriers:
//   1. per warp tile, the number kept; whitespace is found four bytes at a
//      time;
//   2. the exclusive prefix of the counts (each CTA sums a range, then
//      scans it from the sum of the ranges before it); its last entry is the
//      compacted length m';
//   3. every warp tile's kept characters packed at its prefix (a warp scan
//      of the lane counts) in the warp's shared buffer and written to a
//      scratch buffer with one bulk store;
//   4. the packed characters decoded (Algorithm 2), the first bad index
//      reduced in compacted offsets;
//   5. the status, first_bad mapped back to an original offset (binary
//      search over the prefix, then a warp scan inside the warp tile); on
//      success first_bad = m.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tuner.h"

namespace gb64 {
namespace {

constexpr int kWsPerThread = 64;                    // characters per lane in a warp tile
constexpr int64_t kWarpTile = 32 * kWsPerThread;  // characters per warp tile of the general path
constexpr int kMaxWsCtas = 1024;                    // bound of the per-CTA totals in the scratch

// Flags shared by the CTAs of a launch; at the start of the scratch block
// (cleared by the host before each launch).
struct WsHeader {
  uint32_t violation;    // some byte broke the line model
  uint32_t bar_count;    // grid barrier of the general path: CTAs arrived,
  uint32_t bar_gen;      // and the barrier's generation
};
constexpr size_t kWsHeaderBytes = 256;

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
// past m read as space).
__device__ __forceinline__ void load_chars(const uint8_t* src, int64_t m, int64_t at,
                                           uint32_t (&w)[16]) {
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
}

// Keep-mask of 64 characters (bit k = character k kept).
__device__ __forceinline__ uint64_t keep_mask(const uint32_t (&w)[16]) {
  uint64_t mask = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) mask |= (uint64_t)keep4(w[i]) << (4 * i);
  return mask;
}

// The lane's 64 characters of a warp tile, loaded one step ahead: next
// holds those of warp tile t (loaded by the previous step); they move to cur
// and the warp's next tile (t + stride) is loaded into next, so that its
// loads are in flight while tile t is worked on.
__device__ __forceinline__ void step_chars(const uint8_t* src, int64_t m, int64_t t,
                                           int64_t stride, int64_t ntiles, uint32_t (&cur)[16],
                                           uint32_t (&next)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) cur[i] = next[i];
  const int64_t tn = t + stride;
  if (tn < ntiles) load_chars(src, m, tn * kWarpTile + (int64_t)kWsPerThread * (threadIdx.x & 31u), next);
}

// Block-wide exclusive scan of one int64 per thread (NT threads); *total
// gets the sum.
template <int NT>
__device__ __forceinline__ int64_t block_excl_scan64(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums64[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_sums64[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = lane < NT / 32 ? warp_sums64[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < NT / 32) warp_sums64[lane] = t;
  }
  __syncthreads();
  *total = warp_sums64[NT / 32 - 1];
  const int64_t r = (warp ? warp_sums64[warp - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

// Block-wide sum of one int64 per thread (NT threads).
template <int NT>
__device__ __forceinline__ int64_t block_sum64(int64_t v) {
  int64_t total;
  block_excl_scan64<NT>(v, &total);
  return total;
}

// Packs one warp tile's kept characters (the lane's 64 in w) at out +
// offset, by the warp alone: in its shared buffer wbuf (kWarpTile + 32
// bytes) at the output's phase (position o2 + i holds output byte i, o2 =
// the output address mod 16), then the aligned interior by one bulk store,
// the ragged ends (at most 15 bytes each) by byte stores of lanes 0..15 and
// 16..31. sel: the 16 byte_perm selectors that move the kept bytes of a word
// (keep bits k4) to its low end, in order. The bulk store of the previous
// tile has finished reading wbuf before it is written again.
__device__ __forceinline__ void compact_warp_tile(const uint32_t (&w)[16], int64_t offset,
                                                  uint8_t* out, uint8_t* wbuf,
                                                  const uint16_t* sel) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t mask = keep_mask(w);
  const uint32_t n = (uint32_t)__popcll(mask);
  uint32_t incl = n;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if ((int)lane >= d) incl += y;
  }
  const uint32_t olen = __shfl_sync(0xFFFFFFFFu, incl, 31);
  uint8_t* d = out + offset;
  const uintptr_t da = reinterpret_cast<uintptr_t>(d);
  const uint32_t o2 = (uint32_t)(da & 15u);
  if (lane == 0) bulk_wait_read_all();
  __syncwarp();
  uint32_t p = o2 + incl - n;
  // branch-free, so that the lanes never split over a word with whitespace:
  // the word's kept bytes moved down by one byte_perm, then stored under
  // predicates
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t k4 = (uint32_t)(mask >> (4 * i)) & 15u;
    const uint32_t v = __byte_perm(w[i], 0u, sel[k4]);
    const uint32_t c = __popc(k4);
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k)
      if (k < c) wbuf[p + k] = (uint8_t)(v >> (8 * k));
    p += c;
  }
  fence_proxy_async_smem();
  __syncwarp();
  const uintptr_t lo = (da + 15u) & ~(uintptr_t)15u, hi = (da + olen) & ~(uintptr_t)15u;
  if (lane == 0 && hi > lo) {
    tma_store_1d(reinterpret_cast<void*>(lo), wbuf + (o2 ? 16u : 0u), (uint32_t)(hi - lo));
    bulk_commit();
  }
  const uint32_t head = (uint32_t)(tmin<uintptr_t>(lo, da + olen) - da);
  const uint32_t ie = hi > lo ? (uint32_t)(hi - da) : head;
  if (lane < head) {
    d[lane] = wbuf[o2 + lane];
  } else if (lane >= 16u && lane - 16u < olen - ie) {
    d[ie + lane - 16u] = wbuf[o2 + ie + lane - 16u];
  }
  __syncwarp();
}

__device__ __forceinline__ bool is_ws(uint32_t x) { return x == 0x20 || x == 0x0A || x == 0x0D; }

// Original index of compacted character k (k < prefix[ntiles]), by one
// warp: the warp tile holding it (binary search of the prefix), then the
// kept characters of each lane's 64 of the tile counted and prefixed, then
// one lane's scan of its part.
__device__ int64_t original_index(const uint8_t* src, int64_t m, const int64_t* prefix,
                                  int64_t ntiles, int64_t k, uint32_t lane) {
  int64_t lo = 0, hi = ntiles;  // prefix[lo] <= k < prefix[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) / 2;
    if (prefix[mid] <= k) lo = mid; else hi = mid;
  }
  const int64_t part = kWsPerThread;
  const int64_t b = lo * kWarpTile + lane * part, e = tmin<int64_t>(m, b + part);
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

// Set by a kernel of this file that gave up on a bounded wait.
static __device__ unsigned int g_ws_fault;

// Barrier of all CTAs of a cooperative launch (all resident), on the
// header's counter and generation; waits at most limit_ns. False if it ran
// out (the fault word is then set).
__device__ bool grid_sync(WsHeader* h, uint64_t limit_ns) {
  __syncthreads();
  uint32_t ok = 1;
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = &h->bar_gen;
    const uint32_t g0 = *gen;
    __threadfence();
    if (atomicAdd(&h->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&h->bar_count, 0u);
      __threadfence();
      atomicAdd(&h->bar_gen, 1u);
    } else {
      const uint64_t t0 = global_timer_ns();
      while (*gen == g0) {
        if (global_timer_ns() - t0 > limit_ns) {
          ok = 0;
          atomicOr(&g_ws_fault, 1u);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// The status of a call whose grid barrier gave up (thread 0 of each CTA
// that saw it; the same values from each).
__device__ __forceinline__ void ws_timed_out(b64_result* res, uint64_t m) {
  if (threadIdx.x != 0) return;
  volatile b64_result* r = res;
  r->first_bad = (int64_t)m;
  r->outlen = 0;
  r->status = B64_ERR_TIMEOUT;
}

struct GeneralArgs {
  const uint8_t* src;
  uint64_t m;
  uint8_t* dst;
  b64_result* res;
  WsHeader* hdr;
  int64_t* prefix;  // ntiles + 1 entries: warp tile counts, then their exclusive prefix
  int64_t* blk;     // kMaxWsCtas entries: per-CTA totals of the counts
  uint8_t* packed;  // the kept characters (16-byte aligned)
  uint32_t flags;
  uint64_t wait_ns;
};

// The general path, run by every CTA of the (cooperative) launch over warp
// tiles of 2048 characters, each warp on its own (no block barriers in the
// passes over the data, which matters with one CTA per SM). Phases, between
// grid barriers: (1) each warp tile's kept characters counted; (2) their
// exclusive prefix (prefix[ntiles] = m', the compacted length): each CTA
// sums a contiguous range of the counts, then scans it from the sum of the
// ranges before it; (3) each warp tile packed at its prefix; (4) the packed
// characters decoded (Algorithm 2: units of 16 characters, then whole
// quads, then the final group), the first bad index reduced in compacted
// offsets; (5) CTA 0 writes the status with first_bad mapped to an original
// offset (m on success). smem: NT / 32 warp buffers of kWarpTile + 32
// bytes; sel and D as for compact_warp_tile and the decode. Out of line, so
// that the registers of the line-model loop do not depend on it.
template <int NT>
__device__ __noinline__ void general_path(const GeneralArgs a, uint8_t* smem, const uint16_t* sel,
                                          const uint8_t* D) {
  constexpr uint32_t kWarps = NT / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const int64_t m = (int64_t)a.m;
  const int64_t ntiles = tmax<int64_t>(1, (m + kWarpTile - 1) / kWarpTile);
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, nw = (int64_t)gridDim.x * kWarps;
  unsigned long long* first_bad = reinterpret_cast<unsigned long long*>(&a.res->first_bad);
  uint32_t cur[16], next[16];
  // (1) counts
  if (gw < ntiles) load_chars(a.src, m, gw * kWarpTile + (int64_t)kWsPerThread * lane, next);
  for (int64_t t = gw; t < ntiles; t += nw) {
    step_chars(a.src, m, t, nw, ntiles, cur, next);
    const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)__popcll(keep_mask(cur)));
    if (lane == 0) a.prefix[t] = c;
  }
  if (!grid_sync(a.hdr, a.wait_ns)) return ws_timed_out(a.res, a.m);
  // (2) exclusive prefix: per-CTA range totals, then each range scanned
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = tmin<int64_t>(ntiles, (int64_t)blockIdx.x * per);
  const int64_t r1 = tmin<int64_t>(ntiles, r0 + per);
  {
    int64_t sum = 0;
    for (int64_t i = r0 + tid; i < r1; i += NT) sum += a.prefix[i];
    const int64_t total = block_sum64<NT>(sum);
    if (tid == 0) a.blk[blockIdx.x] = total;
  }
  if (!grid_sync(a.hdr, a.wait_ns)) return ws_timed_out(a.res, a.m);
  {
    int64_t before = 0;
    for (uint32_t b = tid; b < blockIdx.x; b += NT) before += a.blk[b];
    int64_t run = block_sum64<NT>(before);
    for (int64_t i0 = r0; i0 < r1; i0 += NT) {
      const int64_t i = i0 + tid;
      const int64_t v = i < r1 ? a.prefix[i] : 0;
      int64_t total;
      const int64_t ex = block_excl_scan64<NT>(v, &total);
      if (i < r1) a.prefix[i] = run + ex;
      run += total;
    }
    if (blockIdx.x == gridDim.x - 1 && tid == 0) a.prefix[ntiles] = run;
  }
  if (!grid_sync(a.hdr, a.wait_ns)) return ws_timed_out(a.res, a.m);
  // (3) compaction, each warp into its own buffer
  uint8_t* wbuf = smem + (size_t)warp * (kWarpTile + 32);
  if (gw < ntiles) load_chars(a.src, m, gw * kWarpTile + (int64_t)kWsPerThread * lane, next);
  for (int64_t t = gw; t < ntiles; t += nw) {
    step_chars(a.src, m, t, nw, ntiles, cur, next);
    compact_warp_tile(cur, a.prefix[t], a.packed, wbuf, sel);
  }
  if (lane == 0) {
    bulk_wait_all();
    // the bulk stores (async proxy) come before the generic reads of phase 4
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  if (!grid_sync(a.hdr, a.wait_ns)) return ws_timed_out(a.res, a.m);
  // (4) decode of the packed characters
  const uint64_t mc = (uint64_t)a.prefix[ntiles];
  const uint64_t be = decode_body_end(mc);
  const uint64_t nunits = be / 16;
  // kPer units per thread and step, all loaded before any is decoded (one
  // CTA per SM: the loads in flight have to cover the memory latency)
  constexpr uint32_t kPer = 8;
  const uint64_t stride = (uint64_t)gridDim.x * NT * kPer;
  unsigned long long bad = ~0ull;
  for (uint64_t base = (uint64_t)blockIdx.x * NT * kPer; base < nunits; base += stride) {
    // consecutive lanes own consecutive units and store them together
    uint4 w[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint64_t u = base + k * NT + tid;
      w[k] = u < nunits ? *reinterpret_cast<const uint4*>(a.packed + 16 * u) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
      const uint64_t u = base + k * NT + tid;
      uint3 o = make_uint3(0, 0, 0);
      if (u < nunits) {
        uint32_t err = 0;
        o = dec_unit(w[k], D, err);
        if ((err & kBadFlag) && bad == ~0ull) bad = 16 * u + dec_unit_first_bad(w[k], D);
      }
      const uint64_t u0 = base + k * NT + (tid & ~31u);
      if (u0 < nunits)
        store12_warp(a.dst + 12 * u0, o, lane, (uint32_t)tmin<uint64_t>(32, nunits - u0));
    }
  }
  warp_min_to(first_bad, bad);
  if (blockIdx.x == 0) {
    const uint64_t q0 = 16 * nunits;
    const uint32_t nq = (uint32_t)((be - q0) / 4);
    if (tid < nq) {
      const uint64_t idx = q0 + 4 * tid;
      const uint8_t* p = a.packed + idx;
      const uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                         ((uint32_t)p[3] << 24);
      uint32_t err = 0;
      const uint32_t v = dec_quad(x, D, err);
      if (err & kBadFlag) {
        for (uint32_t k = 0; k < 4; ++k)
          if (D[(x >> (8 * k)) & 0xFFu] & kBadFlag) {
            atomicMin(first_bad, (unsigned long long)(idx + k));
            break;
          }
      } else {
        uint8_t* q = a.dst + idx / 4 * 3;
        q[0] = (uint8_t)(v >> 16);
        q[1] = (uint8_t)(v >> 8);
        q[2] = (uint8_t)v;
      }
    }
    if (tid == NT - 1 && be < mc)
      a.res->outlen = dec_final_group(a.packed, mc, be, a.dst, D, first_bad, a.flags);
  }
  if (!grid_sync(a.hdr, a.wait_ns)) return ws_timed_out(a.res, a.m);
  // (5) the status, first_bad in original offsets
  if (blockIdx.x == 0 && tid < 32) {
    volatile b64_result* r = a.res;
    const unsigned long long fb = *first_bad;
    const int64_t final_bytes = be < mc ? r->outlen : 0;
    const FinalStatus f = final_status(mc, be, fb, final_bytes, a.flags);
    int64_t out = m;
    if (f.status > 0 && f.first_bad < (int64_t)mc)
      out = original_index(a.src, m, a.prefix, ntiles, f.first_bad, lane);
    __syncwarp();
    if (lane == 0) {
      if (atomicAdd(&g_ws_fault, 0u)) {
        r->first_bad = m;
        r->outlen = 0;
        r->status = B64_ERR_TIMEOUT;
      } else {
        r->first_bad = out;
        r->outlen = f.outlen;
        r->status = f.status;
      }
    }
  }
}

// ------------------------------------------------------ line-model decode
constexpr uint32_t kProbe = 4096;        // characters searched for the first line break
constexpr uint32_t kMaxTrail = 16;       // trailing whitespace the model can drop
constexpr uint32_t kNoLines = 1u << 28;  // line length standing for "no line breaks"
constexpr uint32_t kMaxLineStages = 6;
constexpr uint32_t kWsClass = 0x40;      // decode-table bit of space, line feed, carriage return
// Left in b64_result.internal by a decode that the line-model kernel
// finished (the general path leaves its CTA counter there).
constexpr uint32_t kLinePathMark = 0x4C494E45u;


struct LinesArgs {
  const uint8_t* src;
  uint64_t m;
  uint8_t* dst;  // 16-byte aligned unless general is set
  b64_result* res;
  WsHeader* hdr;
  int64_t* prefix;   // scratch of the general path (see GeneralArgs)
  int64_t* blk;
  uint8_t* packed;
  uint32_t general;  // 1: the general path alone (an output the bulk stores cannot take)
  uint32_t upt;      // 16-character units per thread per tile
  uint32_t stages;   // input stages
  uint32_t flags;
  uint32_t stall;    // test: CTA 0 leaves out its first copy
  uint64_t wait_ns;  // limit of the stage waits and grid barriers
};

// Bytes of an input stage for a tile of tile_c kept characters: the kept
// characters, at most one 2-byte separator per 16 of them (lines are at
// least 16 long), the separator after the last unit, and the alignment of
// the copy, with room for the last window's word reads.
__host__ __device__ constexpr uint32_t line_stage_bytes(uint32_t tile_c) {
  return (tile_c + tile_c / 8 + 128 + 127) & ~127u;
}

// The layout the input is assumed to have: kept characters in lines of L,
// each line but the last followed by the same w separator bytes, then at
// most kMaxTrail bytes of whitespace.
struct LineModel {
  uint64_t m1;     // input length without its trailing whitespace
  uint64_t mc;     // characters kept
  uint64_t inv_L;  // ceil(2^64 / L): floor(k / L) = umulhi(k, inv_L) for k < 2^48
  uint32_t L;      // characters per line (kNoLines: no line breaks at all)
  uint32_t w;      // separator bytes (0: no line breaks)
  uint32_t magic;  // ceil(2^32 / L): floor(n / L) = umulhi(n, magic) for n < 2^18
  uint32_t ok;     // the input can be tried against this model
  // original index of kept character k
  __device__ __forceinline__ uint64_t orig(uint64_t k) const {
    return w ? k + w * __umul64hi(k, inv_L) : k;
  }
  // kept character k ends a line that a separator follows
  __device__ __forceinline__ bool ends_line(uint64_t k) const {
    if (!w || k + 1 >= mc) return false;
    return __umul64hi(k + 1, inv_L) * L == k + 1;
  }
};

__device__ __forceinline__ uint32_t word4(uint4 v, uint32_t k) {
  return k < 2 ? (k == 0 ? v.x : v.y) : (k == 2 ? v.z : v.w);
}

// Derives the line model (every CTA alike): the trailing whitespace from the
// last kMaxTrail bytes, the first line break from the first kProbe bytes.
// A first break at p0 of w = 1 or 2 whitespace bytes gives L = p0; then the
// input without its trailing whitespace must be whole lines of L + w plus a
// last line of 1..L characters. No break in the probe: no line breaks (any
// later whitespace will break the model). Models the kernel cannot use (L <
// 16, a break of 3 or more bytes, a trailing run that may be longer than
// kMaxTrail, lengths that do not fit) are marked not ok.
template <int NT>
__device__ void find_line_model(const uint8_t* src, uint64_t m, const uint8_t* D,
                                LineModel& out, uint32_t* s_first, uint32_t* s_trail) {
  const uint32_t tid = threadIdx.x;
  if (tid < 32) {
    const bool ws = tid < kMaxTrail && tid < m && (D[src[m - 1 - tid]] & kWsClass);
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, ws);
    if (tid == 0) *s_trail = (uint32_t)__ffs(~bal) - 1u;
  }
  const uint32_t P = (uint32_t)tmin<uint64_t>(m, kProbe);
  uint32_t mine = ~0u;
#pragma unroll 4
  for (uint32_t i = tid; i < P; i += NT)
    if (mine == ~0u && (D[src[i]] & kWsClass)) mine = i;
  mine = __reduce_min_sync(0xFFFFFFFFu, mine);
  if ((tid & 31u) == 0 && mine != ~0u) atomicMin(s_first, mine);
  __syncthreads();
  if (tid == 0) {
    LineModel r;
    const uint32_t t = *s_trail;
    r.m1 = m - t;
    r.mc = r.m1;
    r.ok = !(t == kMaxTrail && m > kMaxTrail);
    r.L = kNoLines;
    r.w = 0;
    r.inv_L = 0;
    const uint32_t p0 = *s_first;
    if (p0 < r.m1) {
      uint32_t w = 1;
      if (p0 + 1 < r.m1 && (D[src[p0 + 1]] & kWsClass)) {
        w = 2;
        if (p0 + 2 < r.m1 && (D[src[p0 + 2]] & kWsClass)) r.ok = 0;
      }
      if (p0 < 16) {
        r.ok = 0;
      } else {
        const uint64_t nl = p0 + w;
        const uint64_t q = r.m1 / nl, rest = r.m1 - q * nl;
        if (rest == 0 || rest > p0) r.ok = 0;
        r.L = p0;
        r.w = w;
        r.inv_L = ~0ull / p0 + 1;
        r.mc = q * p0 + rest;
      }
    }
    r.magic = 0xFFFFFFFFu / r.L + 1u;
    out = r;
  }
  __syncthreads();
}

// Bytes [o, o + 20) of the input as five little-endian words, read one by
// one from global memory (bytes at or past m read as 0): the windows of the
// few units whose bytes were not all staged.
__device__ __forceinline__ void window_global(const uint8_t* src, uint64_t m, uint64_t o,
                                              uint32_t (&A)[6]) {
#pragma unroll
  for (uint32_t k = 0; k < 5; ++k) {
    uint32_t x = 0;
#pragma unroll
    for (uint32_t b = 0; b < 4; ++b) {
      const uint64_t i = o + 4 * k + b;
      if (i < m) x |= (uint32_t)src[i] << (8 * b);
    }
    A[k] = x;
  }
}

// The separator after kept character k (original index o) is whitespace.
__device__ __forceinline__ bool sep_ok(const LineModel& md, const uint8_t* src, uint64_t k,
                                       uint64_t o, const uint8_t* D) {
  if (!md.ends_line(k)) return true;
  bool ok = (D[src[o + 1]] & kWsClass) != 0;
  if (md.w > 1) ok = ok && (D[src[o + 2]] & kWsClass) != 0;
  return ok;
}

// One tile's geometry, computed once by the issuing thread and left beside
// the stage: kept characters [off, off + len), body characters (before the
// final group) [off, off + body), whole units nu. Stage byte 0 holds the
// byte at the 16-byte aligned address G; the tile's first kept character
// sits at stage position s0; the bulk copy fills stage positions [ia, ib)
// (the 16-byte aligned part of the tile's original span that lies inside
// the input); units [u_lo, u_hi) have their whole window of 16 + w bytes
// there, the few others read theirs from global memory. The units end nsep
// lines that a kept character follows; their separators are checked once
// per tile (the r-th follows kept character off + (r + 1) L - c0 - 1).
struct LineTile {
  uint64_t off;
  uint64_t a0;  // original index of kept character off
  uintptr_t G;
  uint32_t len, body, nu, s0, ia, ib;
  uint32_t c0;  // position of kept character off in its line
  uint32_t u_lo, u_hi;
  uint32_t nsep;
};

// Window of unit u: p = kept characters from the unit start to its line
// end (huge with no line breaks), su = stage position of its first byte.
__device__ __forceinline__ void unit_geom(const LineModel& md, const LineTile& g, uint32_t w,
                                          uint32_t u, uint32_t& p, uint32_t& su) {
  p = 1u << 30;
  su = g.s0 + 16u * u;
  if (w) {
    const uint32_t n = g.c0 + 16u * u;
    const uint32_t jr = __umulhi(n, md.magic);  // line breaks before the unit
    p = md.L - (n - jr * md.L);
    su += w * jr;
  }
}

__device__ __forceinline__ void line_tile(const LineModel& md, const LinesArgs& a, uint64_t t,
                                          uint32_t tile_c, uint64_t body_end, LineTile& g) {
  g.off = t * tile_c;
  g.len = (uint32_t)tmin<uint64_t>(tile_c, md.mc - g.off);
  g.body = body_end > g.off ? (uint32_t)tmin<uint64_t>(g.len, body_end - g.off) : 0u;
  g.nu = g.body / 16u;
  g.a0 = md.orig(g.off);
  g.c0 = md.w ? (uint32_t)(g.off - __umul64hi(g.off, md.inv_L) * md.L) : 0u;
  g.nsep = 0;
  if (md.w && g.nu) {  // lines j with off <= (j + 1) L - 1 < off + 16 nu and (j + 1) L < mc
    const uint64_t ja = __umul64hi(g.off, md.inv_L);
    const uint64_t jb = tmin(__umul64hi(g.off + 16ull * g.nu, md.inv_L), __umul64hi(md.mc - 1, md.inv_L));
    g.nsep = jb > ja ? (uint32_t)(jb - ja) : 0u;
  }
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.src);
  const uintptr_t A = base + g.a0;
  g.G = A & ~(uintptr_t)15;
  g.s0 = (uint32_t)(A - g.G);
  g.ia = g.ib = 0;
  g.u_lo = g.u_hi = 0;
  if (g.nu) {
    const uint64_t b = tmin<uint64_t>(md.orig(g.off + 16ull * (g.nu - 1)) + 16u + md.w, a.m);
    const uintptr_t lo = (base + 15u) & ~(uintptr_t)15, hi = (base + a.m) & ~(uintptr_t)15;
    const uintptr_t ta = tmax<uintptr_t>(g.G, lo);
    const uintptr_t tb = tmin<uintptr_t>((base + b + 15u) & ~(uintptr_t)15, hi);
    if (tb > ta) {
      g.ia = (uint32_t)(ta - g.G);
      g.ib = (uint32_t)(tb - g.G);
      // ia is 0 or 16, so every unit after the first starts at or after it;
      // from the end, drop the units whose window passes ib
      g.u_lo = g.s0 >= g.ia ? 0u : 1u;
      uint32_t u = g.nu;
      while (u > g.u_lo) {
        uint32_t p, su;
        unit_geom(md, g, md.w, u - 1, p, su);
        if (su + 16u + md.w <= g.ib) break;
        --u;
      }
      g.u_hi = u;
      if (g.u_lo > g.u_hi) g.u_lo = g.u_hi;
    }
  }
}

// The unit's 16 kept characters from its window A (bytes [0, 20)): the W
// separator bytes at window position p are cut out when p < 16 (the
// separators themselves are checked by lines_separators).
template <uint32_t W, bool WORDCUT>
__device__ __forceinline__ uint4 cut_unit(const uint32_t (&A)[5], uint32_t p) {
  uint32_t V[4] = {A[0], A[1], A[2], A[3]};
  if (W) {
    const uint32_t pp = min(p, 16u);
    if (WORDCUT) {  // p is a multiple of 4
#pragma unroll
      for (int i = 1; i < 4; ++i)
        if (pp <= 4u * i) V[i] = __funnelshift_r(A[i], A[i + 1], 8u * W);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t shifted = __funnelshift_r(A[i], A[i + 1], 8u * W);
        const int bits = max(0, (int)(8u * pp) - 32 * i);
        const uint32_t keep = __funnelshift_lc(0xFFFFFFFFu, 0u, (uint32_t)bits);
        V[i] = (A[i] & keep) | (shifted & ~keep);
      }
    }
  }
  return make_uint4(V[0], V[1], V[2], V[3]);
}

// The window of a unit from the stage: (W ? 6 : 5) aligned words and funnel
// shifts.
template <uint32_t W>
__device__ __forceinline__ void stage_window(const uint8_t* st, uint32_t su, uint32_t (&A)[5]) {
  const uint32_t* q = reinterpret_cast<const uint32_t*>(st + (su & ~3u));
  const uint32_t sh = 8u * (su & 3u);
  uint32_t Q[6];
#pragma unroll
  for (int i = 0; i < 5; ++i) Q[i] = q[i];
  Q[5] = W ? q[5] : 0u;
#pragma unroll
  for (int i = 0; i < 5; ++i) A[i] = __funnelshift_r(Q[i], Q[i + 1], sh);
}

// The unit's 16 kept characters, from the stage or (outside [u_lo, u_hi))
// from global memory.
template <uint32_t W, bool WORDCUT>
__device__ __forceinline__ uint4 unit_chars(const LineModel& md, const LineTile& g,
                                            const uint8_t* st, const uint8_t* src, uint64_t m,
                                            uint32_t u, uint32_t& p, uint32_t& su) {
  unit_geom(md, g, W, u, p, su);
  uint32_t A[5];
  if (u >= g.u_lo && u < g.u_hi) {
    stage_window<W>(st, su, A);
  } else {
    uint32_t G6[6];
    window_global(src, m, g.a0 + (su - g.s0), G6);
#pragma unroll
    for (int i = 0; i < 5; ++i) A[i] = G6[i];
  }
  return cut_unit<W, WORDCUT>(A, p);
}

// What a classification found: a byte that breaks the model, and the least
// original index of an invalid character (~0: none).
struct Found {
  bool viol;
  unsigned long long bad;
};

// Classifies the 16 characters v of a unit that flagged one: whitespace at a
// kept position breaks the model; any other flagged character is invalid
// (ou: original index of window byte 0, pp: window bytes before the cut).
template <uint32_t W>
__device__ __forceinline__ void classify_unit(uint4 v, uint64_t ou, uint32_t pp, const uint8_t* D,
                                              Found& f) {
  for (uint32_t i = 0; i < 16; ++i) {
    const uint32_t d = D[(word4(v, i >> 2) >> (8u * (i & 3u))) & 0xFFu];
    if (d & kWsClass) {
      f.viol = true;
    } else if (d & kBadFlag) {
      f.bad = tmin<unsigned long long>(f.bad, ou + i + (i >= pp ? W : 0u));
    }
  }
}

// A tile's units that are not all staged (at most a few per tile), each
// classified at once if it flagged a character. The rare paths take the
// model and the tile by value, so that the caller's copies stay in
// registers.
template <int NT, uint32_t W, bool WORDCUT>
__device__ __noinline__ Found lines_edge_units(const LineModel md, const LineTile g,
                                               const uint8_t* src, uint64_t m, uint32_t* ob,
                                               const uint8_t* D) {
  Found f{false, ~0ull};
  const uint32_t n_lo = g.u_lo, n_hi = g.nu - g.u_hi;
  for (uint32_t i = threadIdx.x; i < n_lo + n_hi; i += NT) {
    const uint32_t u = i < n_lo ? i : g.u_hi + (i - n_lo);
    uint32_t p, su, err = 0;
    const uint4 v = unit_chars<W, WORDCUT>(md, g, nullptr, src, m, u, p, su);
    const uint3 o = dec_unit(v, D, err);
    ob[3 * u] = o.x;
    ob[3 * u + 1] = o.y;
    ob[3 * u + 2] = o.z;
    if (err & kBadFlag) classify_unit<W>(v, g.a0 + (su - g.s0), min(p, 16u), D, f);
  }
  return f;
}

// After one of the thread's staged units [u_lo, u_hi) flagged a character:
// those units (the main loop's: u_lo + threadIdx.x - 32 + k * (NT - 32)) are
// read and classified again.
template <int NT, uint32_t W, bool WORDCUT>
__device__ __noinline__ Found lines_rescan(const LineModel md, const LineTile g,
                                           const uint8_t* st, const uint8_t* src, uint64_t m,
                                           const uint8_t* D) {
  Found f{false, ~0ull};
  for (uint32_t u = g.u_lo + threadIdx.x - 32u; threadIdx.x >= 32u && u < g.u_hi; u += NT - 32) {
    uint32_t p, su;
    const uint4 v = unit_chars<W, WORDCUT>(md, g, st, src, m, u, p, su);
    classify_unit<W>(v, g.a0 + (su - g.s0), min(p, 16u), D, f);
  }
  return f;
}

// The separators of the lines that the tile's units end (when a kept
// character follows) are whitespace: nsep of them, one per thread at a time,
// the r-th at stage position s0 + (r + 1) L - c0 + W r (read from global
// memory when it lies outside the staged bytes). One pass per tile costs
// far less than a check in every unit, since a line holds several units.
template <int NT, uint32_t W>
__device__ __forceinline__ bool lines_separators(const LineModel& md, const LineTile& g,
                                                 const uint8_t* st, const uint8_t* src,
                                                 const uint8_t* D) {
  if (W == 0) return false;
  bool bad = false;
  const uint32_t step = md.L + W;
  for (uint32_t r = threadIdx.x; r < g.nsep; r += NT) {
    const uint32_t sp = g.s0 + md.L - g.c0 + r * step;
    uint32_t c0, c1;
    if (sp >= g.ia && sp + W <= g.ib) {
      c0 = st[sp];
      c1 = st[sp + W - 1];
    } else {
      const uint8_t* q = src + (g.a0 + (sp - g.s0));
      c0 = q[0];
      c1 = q[W - 1];
    }
    bad |= (D[c0] & D[c1] & kWsClass) == 0;
  }
  return bad;
}

// Decodes the whole units [0, nu) of a staged tile into ob (12 bytes per
// unit), one 16-character unit per thread of warps 1.. at a time (warp 0
// issues the copies and stores, so its extra work per tile holds nobody up
// at the tile's barrier): its window of 16 + W
// bytes from the stage (a 16-byte load with no line breaks and an aligned
// input, else aligned words and funnel shifts), the separator that ends a
// line inside it cut out (and checked in a pass of its own). W: separator
// bytes (0: no line breaks); WORDCUT: L is a multiple of 4, so a line ends on
// a word of the window (whole-word selects), else the cut takes byte masks.
template <int NT, uint32_t W, bool WORDCUT>
__device__ __forceinline__ void lines_tile_units(const LineModel& md, const LineTile& g,
                                                 const uint8_t* st, const uint8_t* src,
                                                 uint64_t m, uint32_t* ob, const uint8_t* D,
                                                 bool& viol, unsigned long long& bad) {
  uint32_t err = 0;
  if (W == 0 && g.s0 == 0) {
    const uint4* in = reinterpret_cast<const uint4*>(st);
#pragma unroll 4
    for (uint32_t u = g.u_lo + threadIdx.x - 32u; threadIdx.x >= 32u && u < g.u_hi; u += NT - 32) {
      const uint3 o = dec_unit(in[u], D, err);
      ob[3 * u] = o.x;
      ob[3 * u + 1] = o.y;
      ob[3 * u + 2] = o.z;
    }
  } else {
#pragma unroll 2
    for (uint32_t u = g.u_lo + threadIdx.x - 32u; threadIdx.x >= 32u && u < g.u_hi; u += NT - 32) {
      uint32_t p, su;
      unit_geom(md, g, W, u, p, su);
      uint32_t A[5];
      stage_window<W>(st, su, A);
      const uint4 v = cut_unit<W, WORDCUT>(A, p);
      const uint3 o = dec_unit(v, D, err);
      ob[3 * u] = o.x;
      ob[3 * u + 1] = o.y;
      ob[3 * u + 2] = o.z;
    }
    if (lines_separators<NT, W>(md, g, st, src, D)) viol = true;
  }
  if (err & kBadFlag) {
    const Found f = lines_rescan<NT, W, WORDCUT>(md, g, st, src, m, D);
    viol |= f.viol;
    bad = tmin(bad, f.bad);
  }
  if (g.u_lo > 0 || g.u_hi < g.nu) {
    const Found f = lines_edge_units<NT, W, WORDCUT>(md, g, src, m, ob, D);
    viol |= f.viol;
    bad = tmin(bad, f.bad);
  }
}

// Runs in every CTA after its tiles: a CTA that saw a byte break the model
// raises the violation flag (one whose wait ran out, the fault word), then
// all CTAs meet at a grid barrier. True if some CTA raised the flag: the
// result is back to its cleared state and the general path decodes the
// input instead. Else CTA 0 has written the status, first_bad mapped to
// original offsets.
__device__ bool lines_finish(const LinesArgs& a, const LineModel& md, bool timed_out, bool viol) {
  if (__syncthreads_or(viol) && threadIdx.x == 0) atomicOr(&a.hdr->violation, 1u);
  if (timed_out && threadIdx.x == 0) atomicOr(&g_ws_fault, 1u);
  if (!grid_sync(a.hdr, a.wait_ns)) {
    ws_timed_out(a.res, a.m);
    return false;
  }
  const bool broke = *reinterpret_cast<volatile uint32_t*>(&a.hdr->violation) != 0;
  if (blockIdx.x != 0 || threadIdx.x != 0) return broke;
  volatile b64_result* r = a.res;
  const bool fault = atomicAdd(&g_ws_fault, 0u) != 0;
  if (broke) {
    r->first_bad = -1;
    r->outlen = -1;
    r->status = -1;
  } else if (fault) {
    r->first_bad = (int64_t)a.m;
    r->outlen = 0;
    r->status = B64_ERR_TIMEOUT;
  } else {
    const uint64_t be = decode_body_end(md.mc);
    const unsigned long long fb =
        atomicAdd(reinterpret_cast<unsigned long long*>(&a.res->first_bad), 0ull);
    const int64_t final_bytes = (be < md.mc) ? r->outlen : 0;
    const FinalStatus f = final_status(md.mc, be, fb, final_bytes, a.flags);
    r->first_bad = f.status == B64_OK                 ? (int64_t)a.m
                   : f.status == B64_ERR_INVALID_CHAR ? f.first_bad
                                                      : (int64_t)md.orig((uint64_t)f.first_bad);
    r->outlen = f.outlen;
    r->status = f.status;
    r->internal = kLinePathMark;
  }
  __threadfence();
  return broke;
}

// The one-pass decode under the line model md (see the top of this file),
// by every CTA; true if a byte broke the model in some CTA (lines_finish).
template <int NT>
__device__ __forceinline__ bool lines_decode(const LinesArgs& a, const LineModel md,
                                             const uint8_t* D, uint64_t* full, LineTile* tiles,
                                             uint8_t* smem) {
  const uint32_t tid = threadIdx.x;
  const uint32_t S = a.stages;
  const uint32_t tile_c = NT * a.upt * 16u;
  const uint32_t tile_o = NT * a.upt * 12u;
  const uint32_t stage_b = line_stage_bytes(tile_c);
  const uint64_t mc = md.mc;
  const uint64_t body_end = decode_body_end(mc);
  const uint64_t ntiles = (mc + tile_c - 1) / tile_c;
  const uint32_t w = md.w;
  // the unit loop this model takes (the same in every CTA)
  const uint32_t path = w == 0 ? 0u : (md.L % 4 == 0 ? w : 2u + w);
  uint8_t* outbuf0 = smem + (size_t)S * stage_b;

  // (the geometry is written before the arrive that publishes it)
  auto issue = [&](uint64_t t, uint32_t s) {
    if (a.stall && t == 0) return;
    LineTile g;
    line_tile(md, a, t, tile_c, body_end, g);
    tiles[s] = g;
    if (g.ib > g.ia) {
      fence_proxy_async_smem();  // earlier generic reads of this stage come first
      mbar_arrive_expect_tx(&full[s], g.ib - g.ia);
      tma_load_1d(smem + (size_t)s * stage_b + g.ia, reinterpret_cast<const void*>(g.G + g.ia),
                  g.ib - g.ia, &full[s]);
    } else {
      mbar_arrive(&full[s]);
    }
  };
  if (tid == 0) {
    fence_proxy_async_smem();
    for (uint32_t s = 0; s < S; ++s) {
      const uint64_t t = blockIdx.x + (uint64_t)s * gridDim.x;
      if (t < ntiles) issue(t, s);
    }
  }

  bool timed_out = false, viol = false;
  unsigned long long bad = ~0ull;  // least original index of an invalid character
  uint32_t k = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const uint32_t s = k % S;
    // another CTA's violation, read now and used after the tile, so that the
    // load's latency hides behind the tile's work
    const uint32_t others =
        tid == 0 ? *reinterpret_cast<volatile uint32_t*>(&a.hdr->violation) : 0u;
    const bool ok = mbar_wait_bounded(&full[s], (k / S) & 1u, a.wait_ns);
    const uint8_t* st = smem + (size_t)s * stage_b;
    uint32_t* ob = reinterpret_cast<uint32_t*>(outbuf0 + (size_t)(k & 1u) * tile_o);
    LineTile g;
    if (ok) {
      g = tiles[s];
      switch (path) {
        case 0: lines_tile_units<NT, 0, true>(md, g, st, a.src, a.m, ob, D, viol, bad); break;
        case 1: lines_tile_units<NT, 1, true>(md, g, st, a.src, a.m, ob, D, viol, bad); break;
        case 2: lines_tile_units<NT, 2, true>(md, g, st, a.src, a.m, ob, D, viol, bad); break;
        case 3: lines_tile_units<NT, 1, false>(md, g, st, a.src, a.m, ob, D, viol, bad); break;
        default: lines_tile_units<NT, 2, false>(md, g, st, a.src, a.m, ob, D, viol, bad); break;
      }
      // whole quads of the body after the last whole unit, gathered by index
      const uint32_t q0 = 16u * g.nu;
      const uint32_t nq = (g.body - q0) / 4u;
      if (tid < nq) {
        const uint64_t kq = g.off + q0 + 4u * tid;
        uint32_t x = 0;
        uint64_t oi[4];
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) {
          oi[i] = md.orig(kq + i);
          x |= (uint32_t)a.src[oi[i]] << (8u * i);
          if (!sep_ok(md, a.src, kq + i, oi[i], D)) viol = true;
        }
        uint32_t err = 0;
        const uint32_t val = dec_quad(x, D, err);
        if (err & kBadFlag) {
#pragma unroll
          for (uint32_t i = 0; i < 4; ++i) {
            const uint32_t d = D[(x >> (8u * i)) & 0xFFu];
            if (d & kWsClass) {
              viol = true;
            } else if (d & kBadFlag) {
              bad = tmin<unsigned long long>(bad, oi[i]);
            }
          }
        } else {
          uint8_t* wq = a.dst + kq / 4 * 3;
          wq[0] = (uint8_t)(val >> 16);
          wq[1] = (uint8_t)(val >> 8);
          wq[2] = (uint8_t)val;
        }
      }
      // final characters of the input
      if (tid == NT - 1 && body_end >= g.off && body_end < g.off + g.len) {
        const uint32_t cnt = (uint32_t)(mc - body_end);
        uint8_t fin[4] = {0, 0, 0, 0};
        uint64_t fo[4] = {0, 0, 0, 0};
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) {  // the loads of all four go out together
          if (i < cnt) {
            fo[i] = md.orig(body_end + i);
            fin[i] = a.src[fo[i]];
          }
        }
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) {
          if (i < cnt) {
            if (D[fin[i]] & kWsClass) viol = true;
            if (!sep_ok(md, a.src, body_end + i, fo[i], D)) viol = true;
          }
        }
        uint32_t bk = ~0u;
        const int r = dec_final_chars(fin, cnt, cnt == 4 && mc % 4 == 0, a.dst + body_end / 4 * 3,
                                      D, &bk, a.flags);
        if (bk != ~0u) bad = tmin<unsigned long long>(bad, fo[bk]);
        a.res->outlen = bk != ~0u ? 0 : r;
      }
    }
    fence_proxy_async_smem();
    if (tid == 0) bulk_wait_read_all();  // the other output buffer is free again
    const bool stop = __syncthreads_or(!ok || viol || others != 0);
    if (stop) {
      timed_out = __syncthreads_or(!ok);
      if (tid == 0) {  // wait (bounded) for this CTA's copies in flight
        for (uint32_t j = 0; j < S; ++j) {
          const uint32_t kk = k + j;
          const uint64_t tt = blockIdx.x + (uint64_t)kk * gridDim.x;
          if (tt < ntiles && !(a.stall && tt == 0))
            mbar_wait_bounded(&full[kk % S], (kk / S) & 1u, 500000000ull);
        }
      }
      break;
    }
    if (tid == 0) {
      const uint32_t ob_bytes = 12u * g.nu;
      const uint32_t sb = ob_bytes & ~15u;
      uint8_t* gout = a.dst + g.off / 4 * 3;
      if (sb) {
        tma_store_1d(gout, ob, sb);
        bulk_commit();
      }
      const uint8_t* obb = reinterpret_cast<const uint8_t*>(ob);
      for (uint32_t i = sb; i < ob_bytes; ++i) gout[i] = obb[i];
      const uint64_t t2 = t + (uint64_t)S * gridDim.x;
      if (t2 < ntiles) issue(t2, s);
    }
  }
  if (tid == 0) bulk_wait_all();
  warp_min_to(reinterpret_cast<unsigned long long*>(&a.res->first_bad), bad);
  return lines_finish(a, md, timed_out, viol);
}

// The whitespace-removing decode, one cooperative launch: the line-model
// decode, unless the host asked for the general path (an output the bulk
// stores cannot take) or the input has no line model the kernel can use;
// the general path when either holds or a byte broke the model.
template <int NT>
__global__ void __launch_bounds__(NT, 1) k_ws_lines(LinesArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t D[256];
  __shared__ uint16_t sel[16];
  __shared__ __align__(8) uint64_t full[kMaxLineStages];
  __shared__ LineTile tiles[kMaxLineStages];
  __shared__ LineModel md_s;
  __shared__ uint32_t s_first, s_trail;

  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    for (uint32_t s = 0; s < a.stages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    s_first = ~0u;
  }
  if (tid < 16) {  // byte_perm selectors of the general path's compaction
    uint32_t v = 0, r = 0;
    for (uint32_t k = 0; k < 4; ++k)
      if (tid & (1u << k)) v |= k << (4 * r++);
    sel[tid] = (uint16_t)v;
  }
  init_tables(nullptr, D, a.flags & kFlagUrl);
  if (tid == 0) {  // whitespace keeps the invalid flag and gets its class bit
    D[0x20] |= kWsClass;
    D[0x0A] |= kWsClass;
    D[0x0D] |= kWsClass;
  }
  __syncthreads();
  // the same decisions in every CTA
  bool general = a.general != 0;
  if (!general) {
    find_line_model<NT>(a.src, a.m, D, md_s, &s_first, &s_trail);
    general = !md_s.ok;
  }
  if (!general) general = lines_decode<NT>(a, md_s, D, full, tiles, smem);
  if (general) {
    const GeneralArgs ga{a.src, a.m, a.dst,   a.res,   a.hdr,
                         a.prefix, a.blk, a.packed, a.flags, a.wait_ns};
    general_path<NT>(ga, smem, sel, D);
  }
}

}  // namespace

namespace {

// One cooperative launch (the CTAs meet at grid barriers), one CTA per SM at
// most and at most one per tile of kept characters.
template <int NT>
cudaError_t launch_lines_nt(const LinesArgs& a0, const TileConfig& c, cudaStream_t stream) {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  LinesArgs a = a0;
  a.upt = (uint32_t)c.upt;
  a.stages = (uint32_t)c.stages;
  const uint32_t tile_c = NT * a.upt * 16u;
  const size_t smem = ws_lines_smem_bytes(c);
  int bps = 0;
  e = kernel_prepare(reinterpret_cast<const void*>(k_ws_lines<NT>), smem, NT, &bps);
  if (e != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  const uint64_t ntiles = std::max<uint64_t>(1, (a.m + tile_c - 1) / tile_c);
  const int grid = (int)std::min<uint64_t>(
      {ntiles, (uint64_t)di->sm_count * bps, (uint64_t)kMaxWsCtas});
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_ws_lines<NT>), grid, NT, args,
                                     smem, stream);
}

cudaError_t launch_lines(const LinesArgs& a, const TileConfig& c, cudaStream_t stream) {
  if (!ws_lines_config_valid(c)) return cudaErrorInvalidValue;
  return c.threads == 256 ? launch_lines_nt<256>(a, c, stream) : launch_lines_nt<512>(a, c, stream);
}

// Scratch of the whitespace decode, kept per device between calls (a
// stream-ordered allocation of about m bytes in every call cost about 20 us
// of host and device time on a 367 MB input). A call on another stream is
// ordered after the last user by an event; while the stream captures a
// graph, the call allocates from the stream-ordered allocator instead.
struct WsScratch {
  void* p = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
};
constexpr int kMaxDevices = 128;
std::mutex g_ws_mu;
WsScratch g_ws_scratch[kMaxDevices];

}  // namespace

// Shape of the line-model kernel, one CTA of 512 threads per SM: 56 KiB
// tiles of kept characters in 2 stages for large inputs (the fastest
// measured on GB300), smaller tiles below 64 MiB and 4 MiB so that every SM
// still gets tiles.
TileConfig default_ws_lines_config(uint64_t m) {
  return m >= (64ull << 20) ? TileConfig{512, 7, 2, 0}
         : m >= (4ull << 20) ? TileConfig{512, 2, 4, 0}
                             : TileConfig{512, 1, 4, 0};
}

bool ws_lines_config_valid(const TileConfig& c) {
  return (c.threads == 256 || c.threads == 512) && c.upt >= 1 &&
         c.upt <= 8 && (int64_t)c.threads * c.upt * 16 <= 65536 && c.stages >= 2 &&
         c.stages <= (int)kMaxLineStages;
}

// The input stages and two output buffers of the line-model decode, and at
// least the general path's packing buffer (which reuses them).
size_t ws_lines_smem_bytes(const TileConfig& c) {
  const uint32_t tile_c = (uint32_t)c.threads * c.upt * 16u;
  const size_t lines =
      (size_t)c.stages * line_stage_bytes(tile_c) + 2 * (size_t)c.threads * c.upt * 12u;
  return std::max(lines, (size_t)c.threads / 32 * (kWarpTile + 32));
}

// Header, packed characters, warp tile prefix and per-CTA totals.
size_t ws_scratch_bytes(uint64_t m) {
  const int64_t ntiles = std::max<int64_t>(1, ((int64_t)m + kWarpTile - 1) / kWarpTile);
  return kWsHeaderBytes + ((m + 255) & ~255ull) + (size_t)(ntiles + 1 + kMaxWsCtas) * 8;
}

// Enqueues the whitespace-removing decode into the given scratch;
// *d_result has been cleared. One launch: the line-model decode when dst is
// 16-byte aligned, with the general path in the same kernel when the model
// does not hold; the general path alone otherwise.
cudaError_t decode_ws_launch(const uint8_t* src, uint64_t m, uint8_t* dst, b64_result* d_result,
                             void* scratch, uint32_t flags, cudaStream_t stream) {
  WsHeader* hdr = static_cast<WsHeader*>(scratch);
  uint8_t* packed = static_cast<uint8_t*>(scratch) + kWsHeaderBytes;
  int64_t* prefix = reinterpret_cast<int64_t*>(packed + ((m + 255) & ~255ull));
  const int64_t ntiles = std::max<int64_t>(1, ((int64_t)m + kWarpTile - 1) / kWarpTile);
  int64_t* blk = prefix + ntiles + 1;
  const uint32_t dflags = flags & ~(uint32_t)B64_FLAG_SKIP_WS;
  const uint32_t general = (reinterpret_cast<uintptr_t>(dst) & 15u) != 0;
  const cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), stream);
  if (e != cudaSuccess) return e;
  const WaitTest wt = wait_test();
  const LinesArgs a{src, m, dst, d_result, hdr, prefix, blk, packed, general,
                    0, 0, dflags, wt.stall, wt.limit_ns};
  return launch_lines(a, ws_lines_config(m), stream);
}

// Enqueues the whitespace-removing decode with the device's kept scratch
// (or, under graph capture, a stream-ordered allocation).
cudaError_t decode_ws_enqueue(const uint8_t* src, uint64_t m, uint8_t* dst, b64_result* d_result,
                              uint32_t flags, cudaStream_t stream) {
  const size_t need = ws_scratch_bytes(m);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusNone) {
    void* scratch = nullptr;
    e = cudaMallocAsync(&scratch, need, stream);
    if (e != cudaSuccess) return e;
    e = decode_ws_launch(src, m, dst, d_result, scratch, flags, stream);
    const cudaError_t ef = cudaFreeAsync(scratch, stream);
    return e != cudaSuccess ? e : ef;
  }
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  if (di->device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_ws_mu);
  WsScratch& w = g_ws_scratch[di->device];
  if (!w.done) {
    e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      w.done = nullptr;
      return e;
    }
  }
  if (w.cap < need) {
    if (w.p) {
      e = cudaEventSynchronize(w.done);
      if (e == cudaSuccess) e = cudaFree(w.p);
      if (e != cudaSuccess) return e;
      w.p = nullptr;
      w.cap = 0;
    }
    const size_t cap = (need + (16u << 20) - 1) & ~(size_t)((16u << 20) - 1);
    e = cudaMalloc(&w.p, cap);
    if (e != cudaSuccess) {
      w.p = nullptr;
      return e;
    }
    w.cap = cap;
  }
  e = cudaStreamWaitEvent(stream, w.done, 0);
  if (e == cudaSuccess) e = decode_ws_launch(src, m, dst, d_result, w.p, flags, stream);
  const cudaError_t er = cudaEventRecord(w.done, stream);
  return e != cudaSuccess ? e : er;
}

// Frees the current device's kept scratch once its last user is done.
cudaError_t ws_release_scratch() {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  if (di->device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_ws_mu);
  WsScratch& w = g_ws_scratch[di->device];
  if (!w.p) return cudaSuccess;
  e = cudaEventSynchronize(w.done);
  if (e == cudaSuccess) e = cudaFree(w.p);
  if (e != cudaSuccess) return e;
  w.p = nullptr;
  w.cap = 0;
  return cudaSuccess;
}

int ws_read_and_clear_fault(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_ws_fault, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ws_fault, &zero, sizeof(zero));
  *out = v;
  return e == cudaSuccess ? 0 : cuda_status(e, "reading the fault word");
}

}  // namespace gb64
