// Device building blocks of the gb64 codec (sm_103a).
//
// - PTX wrappers for mbarrier and the 1-D TMA bulk copies
//   (cp.async.bulk global<->shared) with bounded waits.
// - The alphabet maps: encode maps a 6-bit value to its character by the
//   five ranges of Table 3 (offsets +65, +71, -4, -19, -16); decode inverts
//   that map into a 256-entry byte table whose entries outside the alphabet
//   carry bit 7 (the "invalid" flag, like the zero offset of Section 4.2).
//   Both live in shared memory; 64 or 256 bytes span at most 32 banks for
//   every ASCII input, so lookups by a warp never conflict on valid text.
// - Unit codecs: 12 bytes -> 16 characters (four groups of Algorithm 1's
//   main loop) and 16 characters -> 12 bytes (four quads of Algorithm 2's
//   main loop), with bytes regrouped by prmt (__byte_perm) and shifts.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gb64.h"
#include "rules.h"

namespace gb64 {

template <typename T>
__host__ __device__ __forceinline__ T tmin(T a, T b) {
  return a < b ? a : b;
}
template <typename T>
__host__ __device__ __forceinline__ T tmax(T a, T b) {
  return a > b ? a : b;
}

constexpr uint32_t kPadChar = 0x3D;  // '='
constexpr uint32_t kBadFlag = 0x80;  // decode-table flag for bytes outside the alphabet

// Table 3: 6-bit value -> ASCII code, by range; base64url (Section 2) maps
// 62 and 63 to '-' and '_'.
__host__ __device__ constexpr uint32_t alphabet_char(uint32_t v, bool url = false) {
  return v < 26 ? v + 65
       : v < 52 ? v + 71
       : v < 62 ? v - 4
       : v == 62 ? (url ? 0x2Du : v - 19)
                 : (url ? 0x5Fu : v - 16);
}

// Fills the shared tables. enc: 64 bytes; dec: 256 bytes (either may be null).
__device__ __forceinline__ void init_tables(uint8_t* enc, uint8_t* dec, bool url = false) {
  if (dec) {
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) dec[i] = (uint8_t)kBadFlag;
    __syncthreads();
  }
  for (uint32_t v = threadIdx.x; v < 64; v += blockDim.x) {
    const uint32_t c = alphabet_char(v, url);
    if (enc) enc[v] = (uint8_t)c;
    if (dec) dec[c] = (uint8_t)v;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase with the given parity to complete, for at most about
// limit_ns of wall time. Returns false on timeout (the caller reports it).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u && global_timer_ns() - t0 > limit_ns) return false;
  }
}

// try_wait with a suspend-time hint: the thread may sleep until the phase
// completes or about `ns` nanoseconds pass, instead of polling.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// As mbar_wait_bounded, but letting the hardware suspend the waiting warp
// until the phase completes, so that warps waiting for their next tile
// leave the issue slots to the warps computing.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (;;) {
    if (mbar_try_wait_suspend(bar, parity, 100000u)) return true;
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
}

// 1-D bulk copy global -> shared, completing `bytes` transactions on bar.
// Both addresses and bytes must be multiples of 16.
__device__ __forceinline__ void tma_load_1d(void* smem_dst, const void* gsrc, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 1-D bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void tma_store_1d(void* gdst, const void* smem_src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
               "r"(smem_addr(smem_src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// All committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// All committed bulk stores are complete (written to global memory).
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// At most n (0..3) of the committed bulk-store groups still read shared
// memory.
__device__ __forceinline__ void bulk_wait_read(uint32_t n) {
  switch (n) {
    case 0: asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory"); break;
    default: asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); break;
  }
}

// Orders this thread's generic-proxy shared-memory accesses with later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_global_v4_cs(void* p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// --------------------------------------------------------------- encode
// One group of Algorithm 1's main loop. g holds the three bytes big-endian
// in bits 23..0 (bits above 23 are ignored); returns the four characters as
// a little-endian word (first character in the low byte).
__device__ __forceinline__ uint32_t enc_group(uint32_t g, const uint8_t* T) {
  const uint32_t c0 = T[(g >> 18) & 63u];
  const uint32_t c1 = T[(g >> 12) & 63u];
  const uint32_t c2 = T[(g >> 6) & 63u];
  const uint32_t c3 = T[g & 63u];
  return __byte_perm(__byte_perm(c0, c1, 0x0040), __byte_perm(c2, c3, 0x0040), 0x5410);
}

// Four groups: stream bytes x0..x11 in little-endian words w0, w1, w2
// (x0 = low byte of w0) -> 16 characters.
__device__ __forceinline__ uint4 enc_unit(uint32_t w0, uint32_t w1, uint32_t w2,
                                          const uint8_t* T) {
  uint4 o;
  o.x = enc_group(__byte_perm(w0, 0u, 0x4012), T);  // x0 x1 x2
  o.y = enc_group(__byte_perm(w0, w1, 0x3345), T);  // x3 x4 x5
  o.z = enc_group(__byte_perm(w1, w2, 0x2234), T);  // x6 x7 x8
  o.w = enc_group(__byte_perm(w2, 0u, 0x4123), T);  // x9 x10 x11
  return o;
}

// The last, possibly partial, group: cnt (1..3) bytes b0..b2 -> four
// characters with "==" (cnt 1) or "=" (cnt 2) padding (Algorithm 1's tail).
__device__ __forceinline__ uint32_t enc_tail_group(uint32_t b0, uint32_t b1, uint32_t b2,
                                                   uint32_t cnt, const uint8_t* T) {
  if (cnt < 2) b1 = 0;
  if (cnt < 3) b2 = 0;
  uint32_t w = enc_group((b0 << 16) | (b1 << 8) | b2, T);
  if (cnt == 1) w = (w & 0x0000FFFFu) | (kPadChar << 16) | (kPadChar << 24);
  if (cnt == 2) w = (w & 0x00FFFFFFu) | (kPadChar << 24);
  return w;
}

// --------------------------------------------------------------- decode
// One quad of Algorithm 2's main loop: four characters (little-endian word)
// -> 24-bit value a*2^18 + b*2^12 + c*2^6 + d; err collects the table flags.
// Each character is picked out by one byte_perm, and the value is built by
// multiply-adds (the same value as shifts and ors for entries below 64; any
// other entry is flagged), which leaves the integer ALU pipe, the busiest in
// the decoders, fewer instructions.
__device__ __forceinline__ uint32_t dec_quad(uint32_t x, const uint8_t* D, uint32_t& err) {
  const uint32_t a = D[__byte_perm(x, 0u, 0x4440)];
  const uint32_t b = D[__byte_perm(x, 0u, 0x4441)];
  const uint32_t c = D[__byte_perm(x, 0u, 0x4442)];
  const uint32_t d = D[x >> 24];
  err |= a | b | c | d;
  return ((a * 64u + b) * 64u + c) * 64u + d;
}

// Four quads (16 characters) -> 12 output bytes (three little-endian words).
__device__ __forceinline__ uint3 dec_unit(uint4 w, const uint8_t* D, uint32_t& err) {
  const uint32_t v0 = dec_quad(w.x, D, err);
  const uint32_t v1 = dec_quad(w.y, D, err);
  const uint32_t v2 = dec_quad(w.z, D, err);
  const uint32_t v3 = dec_quad(w.w, D, err);
  uint3 o;
  o.x = __byte_perm(v0, v1, 0x6012);
  o.y = __byte_perm(v1, v2, 0x5601);
  o.z = __byte_perm(v2, v3, 0x4560);
  return o;
}

// Index (0..15) of the first character of a unit whose table entry is
// flagged, or 16 if none.
__device__ __forceinline__ uint32_t dec_unit_first_bad(uint4 w, const uint8_t* D) {
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (uint32_t k = 0; k < 16; ++k) {
    const uint32_t ch = (ws[k >> 2] >> (8 * (k & 3))) & 0xFFu;
    if (D[ch] & kBadFlag) return k;
  }
  return 16;
}

// ---------------------------------------------------- unaligned access
// Four little-endian words holding bytes p[0..15], for any alignment of p.
// Aligned words are read only when they lie inside [lo, hi); near the ends
// of the buffer single bytes are read instead.
__device__ __forceinline__ uint4 load16_any(const uint8_t* p, const uint8_t* lo,
                                            const uint8_t* hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t r = a & 3u;
  uint4 v;
  if (r == 0) {
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
    if ((a & 15u) == 0) return __ldg(reinterpret_cast<const uint4*>(p));
    v.x = __ldg(q);
    v.y = __ldg(q + 1);
    v.z = __ldg(q + 2);
    v.w = __ldg(q + 3);
    return v;
  }
  const uint8_t* base = p - r;
  if (base >= lo && base + 20 <= hi) {
    const uint32_t* q = reinterpret_cast<const uint32_t*>(base);
    const uint32_t q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3),
                   q4 = __ldg(q + 4);
    const uint32_t sh = 8 * r;
    v.x = __funnelshift_r(q0, q1, sh);
    v.y = __funnelshift_r(q1, q2, sh);
    v.z = __funnelshift_r(q2, q3, sh);
    v.w = __funnelshift_r(q3, q4, sh);
    return v;
  }
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[k] = (uint32_t)__ldg(p + 4 * k) | ((uint32_t)__ldg(p + 4 * k + 1) << 8) |
           ((uint32_t)__ldg(p + 4 * k + 2) << 16) | ((uint32_t)__ldg(p + 4 * k + 3) << 24);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Three little-endian words holding bytes p[0..11] (same rules).
__device__ __forceinline__ uint3 load12_any(const uint8_t* p, const uint8_t* lo,
                                            const uint8_t* hi) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t r = a & 3u;
  uint3 v;
  if (r == 0) {
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
    v.x = __ldg(q);
    v.y = __ldg(q + 1);
    v.z = __ldg(q + 2);
    return v;
  }
  const uint8_t* base = p - r;
  if (base >= lo && base + 16 <= hi) {
    const uint32_t* q = reinterpret_cast<const uint32_t*>(base);
    const uint32_t q0 = __ldg(q), q1 = __ldg(q + 1), q2 = __ldg(q + 2), q3 = __ldg(q + 3);
    const uint32_t sh = 8 * r;
    v.x = __funnelshift_r(q0, q1, sh);
    v.y = __funnelshift_r(q1, q2, sh);
    v.z = __funnelshift_r(q2, q3, sh);
    return v;
  }
  uint32_t w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    w[k] = (uint32_t)__ldg(p + 4 * k) | ((uint32_t)__ldg(p + 4 * k + 1) << 8) |
           ((uint32_t)__ldg(p + 4 * k + 2) << 16) | ((uint32_t)__ldg(p + 4 * k + 3) << 24);
  }
  return make_uint3(w[0], w[1], w[2]);
}

// Stores of 16 / 12 / 4 bytes at any alignment.
__device__ __forceinline__ void store16_any(uint8_t* p, uint4 v) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if ((a & 15u) == 0) {
    *reinterpret_cast<uint4*>(p) = v;
  } else if ((a & 3u) == 0) {
    uint32_t* q = reinterpret_cast<uint32_t*>(p);
    q[0] = v.x;
    q[1] = v.y;
    q[2] = v.z;
    q[3] = v.w;
  } else {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 16; ++k) p[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
  }
}

__device__ __forceinline__ void store4_any(uint8_t* p, uint32_t w) {
  if ((reinterpret_cast<uintptr_t>(p) & 3u) == 0) {
    *reinterpret_cast<uint32_t*>(p) = w;
  } else {
    p[0] = (uint8_t)w;
    p[1] = (uint8_t)(w >> 8);
    p[2] = (uint8_t)(w >> 16);
    p[3] = (uint8_t)(w >> 24);
  }
}

// Bytes [sft, sft + 16) of the 32 bytes lo || hi (lo first, little-endian
// words), for sft in 0..15; sft is the same in every lane of a warp.
__device__ __forceinline__ uint4 realign16(uint4 lo, uint4 hi, uint32_t sft) {
  const uint32_t sh = 8u * (sft & 3u);
  uint32_t a, b, c, d, e;
  switch (sft >> 2) {
    case 0: a = lo.x; b = lo.y; c = lo.z; d = lo.w; e = hi.x; break;
    case 1: a = lo.y; b = lo.z; c = lo.w; d = hi.x; e = hi.y; break;
    case 2: a = lo.z; b = lo.w; c = hi.x; d = hi.y; e = hi.z; break;
    default: a = lo.w; b = hi.x; c = hi.y; d = hi.z; e = hi.w; break;
  }
  return make_uint4(__funnelshift_r(a, b, sh), __funnelshift_r(b, c, sh), __funnelshift_r(c, d, sh),
                    __funnelshift_r(d, e, sh));
}

// Bytes p[0..11] of shared memory as three little-endian words, read as
// aligned words (one more when p is not word-aligned).
__device__ __forceinline__ uint3 lds12(const uint8_t* p) {
  const uint32_t r = (uint32_t)(reinterpret_cast<uintptr_t>(p) & 3u);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(p - r);
  if (r == 0) return make_uint3(q[0], q[1], q[2]);
  const uint32_t sh = 8u * r;
  const uint32_t q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
  return make_uint3(__funnelshift_r(q0, q1, sh), __funnelshift_r(q1, q2, sh),
                    __funnelshift_r(q2, q3, sh));
}

// Writes the final group's characters: 4 with padding, or cnt + 1 (2 or 3)
// when padding is omitted (a full group, cnt = 3, always writes 4).
__device__ __forceinline__ void store_tail_group(uint8_t* p, uint32_t w, uint32_t cnt,
                                                 uint32_t flags) {
  if (cnt == 3 || !(flags & kFlagNoPad)) {
    store4_any(p, w);
  } else {
    for (uint32_t k = 0; k <= cnt; ++k) p[k] = (uint8_t)(w >> (8 * k));
  }
}

// Warp-cooperative store: lane l writes its 12 bytes v at p + 12 * l, for
// lanes l < nv (all 32 lanes must call it). At any alignment of p the lanes
// write whole aligned 32-bit words, each built with a funnel shift from the
// lane's own words and the previous lane's last word (shuffled up); only
// the first and last few bytes of the warp's span use byte stores.
__device__ __forceinline__ void store12_warp(uint8_t* p, uint3 v, uint32_t lane, uint32_t nv) {
  const uint32_t r = reinterpret_cast<uintptr_t>(p) & 3u;
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, v.z, 1);
  if (lane >= nv) return;
  uint8_t* q = p + 12 * lane;
  if (r == 0) {
    uint32_t* w = reinterpret_cast<uint32_t*>(q);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    return;
  }
  const uint32_t sh = 8 * (4 - r);
  uint32_t* w = reinterpret_cast<uint32_t*>(q - r);  // aligned word holding q[0]
  if (lane == 0) {
    for (uint32_t k = 0; k < 4 - r; ++k) q[k] = (uint8_t)(v.x >> (8 * k));
  } else {
    w[0] = __funnelshift_r(prev, v.x, sh);
  }
  w[1] = __funnelshift_r(v.x, v.y, sh);
  w[2] = __funnelshift_r(v.y, v.z, sh);
  if (lane == nv - 1)
    for (uint32_t k = 0; k < r; ++k) q[12 - r + k] = (uint8_t)(v.z >> (sh + 8 * k));
}

// ------------------------------------------------------- final group
// The final characters p[0..cnt) of a message, cnt = 1..4: a last quad that
// may end in "=" or "==" (quad: cnt == 4 and the message length is a
// multiple of 4), or 1-3 characters of an incomplete group (an unpadded
// final group under kFlagNoPad, else only validated). Writes the decoded
// bytes at o. On an invalid character sets *bad to its index k (0..3) and
// returns 0. Returns the bytes written (0..3), or -(1 + k) when Appendix A's
// check (kFlagStrictTail) fails at character k: with "==" (or 2 unpadded
// characters) the second character must have (value * 16) mod 256 = 0,
// with "=" (or 3) the third must have (value * 64) mod 256 = 0.
static __device__ __noinline__ int dec_final_chars(const uint8_t* p, uint32_t cnt, bool quad,
                                                   uint8_t* o, const uint8_t* D, uint32_t* bad,
                                                   uint32_t flags) {
  const bool strict = (flags & kFlagStrictTail) != 0;
  if (quad) {
    const uint32_t c[4] = {p[0], p[1], p[2], p[3]};
    uint32_t npad = 0;
    if (c[3] == kPadChar) npad = (c[2] == kPadChar) ? 2 : 1;
    uint32_t v[4];
    for (uint32_t k = 0; k < 4; ++k) {
      const bool is_pad = k >= 4 - npad;
      const uint32_t d = D[c[k]];
      if (!is_pad && (d & kBadFlag)) {
        *bad = k;
        return 0;
      }
      v[k] = is_pad ? 0u : d;
    }
    if (strict && npad == 2 && (v[1] & 15u)) return -2;
    if (strict && npad == 1 && (v[2] & 3u)) return -3;
    const uint32_t val = (v[0] << 18) | (v[1] << 12) | (v[2] << 6) | v[3];
    o[0] = (uint8_t)(val >> 16);
    if (npad < 2) o[1] = (uint8_t)(val >> 8);
    if (npad < 1) o[2] = (uint8_t)val;
    return 3 - (int)npad;
  }
  uint32_t v[3] = {0, 0, 0};
  for (uint32_t k = 0; k < cnt; ++k) {
    const uint32_t d = D[p[k]];
    if (d & kBadFlag) {
      *bad = k;
      return 0;
    }
    if (k < 3) v[k] = d;
  }
  if (!(flags & kFlagNoPad) || cnt < 2) return 0;  // the length rule decides
  if (strict && cnt == 2 && (v[1] & 15u)) return -2;
  if (strict && cnt == 3 && (v[2] & 3u)) return -3;
  o[0] = (uint8_t)((v[0] << 2) | (v[1] >> 4));
  if (cnt == 3) o[1] = (uint8_t)(((v[1] & 15u) << 4) | (v[2] >> 2));
  return (int)cnt - 1;
}

// Final characters [body_end, m) of a message read from src (see
// dec_final_chars); lowers *first_bad on an invalid character. Returns the
// bytes written (0..3), or -(1 + k) when Appendix A's check fails at
// character body_end + k.
static __device__ __noinline__ int dec_final_group(const uint8_t* src, uint64_t m, uint64_t body_end,
                                            uint8_t* dst, const uint8_t* D,
                                            unsigned long long* first_bad, uint32_t flags) {
  const uint32_t cnt = (uint32_t)(m - body_end);
  uint32_t bad = ~0u;
  const int r = dec_final_chars(src + body_end, cnt, cnt == 4 && m % 4 == 0,
                                dst + body_end / 4 * 3, D, &bad, flags);
  if (bad != ~0u) {
    atomicMin(first_bad, (unsigned long long)(body_end + bad));
    return 0;
  }
  return r;
}

// ------------------------------------------------------ error reduction
// Lowers *target to min over the warp's lanes of idx (lanes pass
// UINT64_MAX for "none"). One atomic per warp that saw an error.
// Every lane of the warp must call it (it is a warp-wide convergence point).
__device__ __forceinline__ void warp_min_to(unsigned long long* target, unsigned long long idx) {
  const unsigned mask = 0xFFFFFFFFu;
  const bool any = __ballot_sync(mask, idx != ~0ull) != 0;
  if (!any) return;
  // 64-bit min in two 32-bit reduction steps
  const uint32_t hi = (uint32_t)(idx >> 32);
  const uint32_t min_hi = __reduce_min_sync(mask, hi);
  const uint32_t lo = (hi == min_hi) ? (uint32_t)idx : 0xFFFFFFFFu;
  const uint32_t min_lo = __reduce_min_sync(mask, lo);
  const unsigned long long m = ((unsigned long long)min_hi << 32) | min_lo;
  if ((threadIdx.x & 31u) == 0) atomicMin(target, m);
}

}  // namespace gb64
