// Batched encode and decode of packed messages as one stream ("flat"
// kernels): the output (encode) or the input (decode) of the whole batch is
// cut into fixed tiles that ignore message boundaries, so the work per tile
// does not depend on how the bytes are split into messages.
//
// Each CTA is one producer warp and kFlatConsumerWarps consumer warps
// (warp specialisation). The producer walks the CTA's contiguous range of
// tiles: it finds the message that owns each tile boundary (a 32-way search
// by the whole warp over the offsets array), publishes the tile's view in
// shared memory and issues the bulk copy (TMA) of the tile's input into a
// stage, up to `stages` tiles ahead; consumers wait on the stage's full
// barrier, code the tile and release the stage on its empty barrier.
//
//  - Encode (padded output): every message's output is a whole number of
//    4-character groups, so a 16-byte output chunk is 4 groups. The lane of
//    chunk c codes those groups: 12 contiguous input bytes of one message
//    (Algorithm 1 on a unit) or, at message ends, group by group (partial
//    final group with '=' padding). Chunks go to global memory in aligned
//    16-byte stores.
//  - Decode: the lane of the 16-character unit u of the packed input codes
//    its 4 quads when they are body quads of one message that starts at a
//    multiple of 4 (Algorithm 2 on a unit), else every quad that starts in
//    the unit, per message, and the message's final characters (padding,
//    unpadded final group, Appendix A's check). Output bytes go to an image
//    of the tile's output in shared memory, which leaves by one bulk store
//    (plus byte stores at its ragged ends); bytes of a message's output
//    capacity that no group writes are set to zero.
// Error positions are folded into first_bad[j] by atomicMin; outlen[j]
// receives the final group's result; k_batch_decode_finish (batch.cu)
// turns them into per-message status afterwards.
#include <algorithm>

#include "batch.h"
#include "common.cuh"
#include "internal.h"

namespace gb64 {

static __device__ unsigned int g_flat_fault;

namespace {

constexpr int kFlatConsumerWarps = 8;
constexpr int kFlatThreads = 32 * (1 + kFlatConsumerWarps);
constexpr int kFlatConsumers = 32 * kFlatConsumerWarps;
constexpr int kFlatMaxStages = 6;

// Largest j in [lo, hi) with off[j] <= x, given off[lo] <= x < off[hi]
// (off non-decreasing). All 32 lanes call it; every round probes 31 evenly
// spaced entries and keeps the sub-range that holds x.
__device__ __forceinline__ int64_t warp_owner(const int64_t* off, int64_t lo, int64_t hi, int64_t x,
                                              uint32_t lane) {
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + (int64_t)(lane + 1) * step;
    const bool le = p < hi && __ldg(off + p) <= x;
    const int k = __popc(__ballot_sync(0xFFFFFFFFu, le));
    const int64_t nlo = lo + (int64_t)k * step;
    hi = tmin<int64_t>(hi, nlo + step);
    lo = nlo;
  }
  return lo;
}

// The same search by one thread (binary).
__device__ __forceinline__ int64_t owner_in(const int64_t* off, int64_t lo, int64_t hi, int64_t x) {
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

struct FlatTile {
  int64_t a0, a1;  // encode: output bytes [a0, a1); decode: characters [a0, a1)
  int64_t b0, b1;  // encode: input bytes [b0, b1); decode: output bytes [b0, b1)
  int64_t j0, jn;  // owners of the tile's first position and of a1 (or the last message)
  uint32_t o, ia, ib;  // input byte X is staged at o + X - (encode: b0, decode: a0);
                       // positions [ia, ib) were copied
};

struct FlatArgs {
  const uint8_t* src;
  const int64_t* in_off;
  uint8_t* dst;
  const int64_t* out_off;
  int64_t nmsg;
  int64_t tile;  // encode: output bytes, decode: characters (multiple of 16 * consumers)
  uint32_t stages;
  uint32_t flags;
  int64_t* first_bad;
  int64_t* outlen;
  int64_t max_mean_len;  // > 0: code only batches of shorter messages on average
};

// The batch is left to the per-warp tile kernel (its mean message length is
// max_mean_len or more).
__device__ __forceinline__ bool flat_declines(const FlatArgs& a) {
  return a.max_mean_len > 0 && a.nmsg > 0 && __ldg(a.in_off + a.nmsg) / a.nmsg >= a.max_mean_len;
}

__device__ __forceinline__ void stage_layout(FlatTile& v, const uint8_t* src, int64_t x0, int64_t x1) {
  const uintptr_t s = reinterpret_cast<uintptr_t>(src + x0);
  const uintptr_t a = (s + 15u) & ~(uintptr_t)15u, b = reinterpret_cast<uintptr_t>(src + x1) & ~(uintptr_t)15u;
  v.o = (uint32_t)(s & 15u);
  v.ia = v.o ? 16u : 0u;
  v.ib = b > a ? v.ia + (uint32_t)(b - a) : v.ia;
}

// Producer: copy the tile's interior (one lane; the arrive publishes the view).
__device__ __forceinline__ void flat_issue(const FlatTile& v, const uint8_t* src, int64_t x0,
                                           uint8_t* stage, uint64_t* bar) {
  fence_proxy_async_smem();
  if (v.ib > v.ia) {
    mbar_arrive_expect_tx(bar, v.ib - v.ia);
    tma_load_1d(stage + v.ia, src + x0 + (v.ia - v.o), v.ib - v.ia, bar);
  } else {
    mbar_arrive(bar);
  }
}

// Stage-or-global byte reads of the input at absolute offset X (the stage
// holds offsets from x0 on).
struct StageReader {
  const uint8_t* stage;
  const uint8_t* src;
  int64_t x0, total;
  uint32_t o, ia, ib;
  __device__ __forceinline__ bool inside(int64_t X, uint32_t n) const {
    const int64_t p = (int64_t)o + (X - x0);
    return p >= (int64_t)ia && p + n <= (int64_t)ib;
  }
  __device__ __forceinline__ uint32_t byte(int64_t X) const {
    return inside(X, 1) ? (uint32_t)stage[o + (uint32_t)(X - x0)] : (uint32_t)src[X];
  }
};

// Producer warp of both kernels: views and copies of the CTA's tiles
// [t_begin, t_end). DECODE selects the tile geometry.
template <int DECODE>
__device__ void flat_producer(const FlatArgs& a, int64_t t_begin, int64_t t_end, int64_t in_total,
                              int64_t out_total, uint8_t* stages, uint32_t stage_b, uint64_t* full,
                              uint64_t* empty, FlatTile* meta, uint32_t lane) {
  const uint32_t S = a.stages;
  const int64_t* key = DECODE ? a.in_off : a.out_off;  // offsets the tiles cut
  const int64_t key_total = DECODE ? in_total : out_total;
  int64_t jcur = warp_owner(key, 0, a.nmsg, t_begin * a.tile, lane);
  uint32_t s = 0, phase = 0;
  int64_t t = t_begin;
  for (; t < t_end; ++t) {
    if (t - t_begin >= (int64_t)S) {
      bool ok = true;
      if (lane == 0) ok = mbar_wait_backoff(&empty[s], phase ^ 1u);
      if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) {
        if (lane == 0) atomicOr(&g_flat_fault, 1u);
        break;
      }
    }
    FlatTile v;
    v.a0 = t * a.tile;
    v.a1 = tmin<int64_t>(v.a0 + a.tile, key_total);
    v.j0 = jcur;
    const int64_t jn = v.a1 < key_total ? warp_owner(key, jcur, a.nmsg, v.a1, lane) : a.nmsg - 1;
    v.jn = jn;
    if (!DECODE) {
      // input bytes of output bytes [a0, a1): whole groups, 3 bytes per 4
      const int64_t o0 = __ldg(a.out_off + v.j0), i0 = __ldg(a.in_off + v.j0);
      v.b0 = i0 + 3 * ((v.a0 - o0) / 4);
      if (v.a1 < key_total) {
        v.b1 = __ldg(a.in_off + jn) + 3 * ((v.a1 - __ldg(a.out_off + jn)) / 4);
      } else {
        v.b1 = in_total;
      }
      stage_layout(v, a.src, v.b0, v.b1);
    } else {
      // output bytes of characters [a0, a1): capacity position of a quad
      // boundary, 3 bytes per 4 characters, capped at the message's end
      auto out_at = [&](int64_t c, int64_t j) -> int64_t {
        if (c >= in_total) return out_total;
        const int64_t i0 = __ldg(a.in_off + j);
        return tmin<int64_t>(__ldg(a.out_off + j) + 3 * ((c - i0 + 3) / 4), __ldg(a.out_off + j + 1));
      };
      v.b0 = out_at(v.a0, v.j0);
      v.b1 = out_at(v.a1, jn);
      // the copy reaches 16 characters past the tile: quads that start in
      // the tile may end in the next one
      stage_layout(v, a.src, v.a0, tmin<int64_t>(v.a1 + 16, in_total));
    }
    jcur = jn;
    if (lane == 0) {
      meta[s] = v;
      flat_issue(v, a.src, DECODE ? v.a0 : v.b0, stages + s * stage_b, &full[s]);
    }
    if (++s == S) {
      s = 0;
      phase ^= 1u;
    }
  }
  // the CTA must not end while copies into its stages are in flight: wait
  // (bounded) for the last S issued ones
  if (lane == 0) {
    for (uint32_t i = 0; i < S && t - 1 - (int64_t)i >= t_begin; ++i) {
      if (s == 0) {
        s = S - 1;
        phase ^= 1u;
      } else {
        --s;
      }
      mbar_wait_backoff(&full[s], phase, 500000000ull);
    }
  }
}

// ----------------------------------------------------------------- encode
constexpr int64_t kFar = 1 << 30;  // "beyond the tile" in tile-relative positions

// Bounds of one message (absolute), kept in registers across tiles.
struct MsgBounds {
  int64_t j = -1;
  int64_t o0 = 0, o1 = 0;  // output (encode) / input (decode) range
  int64_t i0 = 0, i1 = 0;  // input (encode) / output start and body end (decode)
};

// Message j as one tile's chunks see it, in 32-bit positions relative to the
// tile: its output [ob, oe) (relative to a0, clamped), the input of its group
// at ob (xb) and its input end (xe), both relative to b0.
struct EncCursor {
  int32_t ob, oe, xb, xe;
};

__device__ __forceinline__ MsgBounds enc_bounds(const FlatArgs& a, int64_t j) {
  MsgBounds m;
  m.j = j;
  m.o0 = __ldg(a.out_off + j);
  m.o1 = __ldg(a.out_off + j + 1);
  m.i0 = __ldg(a.in_off + j);
  m.i1 = __ldg(a.in_off + j + 1);
  return m;
}

__device__ __forceinline__ EncCursor enc_cursor(const MsgBounds& m, const FlatTile& v) {
  EncCursor c;
  if (m.o0 <= v.a0) {  // the message that holds the tile's first group
    c.ob = 0;
    c.xb = (int32_t)(m.i0 + 3 * ((v.a0 - m.o0) / 4) - v.b0);
  } else {
    c.ob = (int32_t)(m.o0 - v.a0);
    c.xb = (int32_t)(m.i0 - v.b0);
  }
  c.oe = (int32_t)tmin<int64_t>(m.o1 - v.a0, kFar);
  c.xe = (int32_t)tmin<int64_t>(m.i1 - v.b0, kFar);
  return c;
}

// A chunk at a message end, group by group (partial final groups padded
// with '='); returns the bounds of the message of its last group.
__device__ __forceinline__ MsgBounds enc_chunk_groups(const FlatArgs& a, const FlatTile& v,
                                                   MsgBounds mb, int32_t P, int32_t tile_len,
                                                   const uint8_t* st, const uint8_t* T) {
  const uint8_t* sb = a.src + v.b0;
  const int32_t so = (int32_t)v.o, sia = (int32_t)v.ia, sib = (int32_t)v.ib;
  auto in_byte = [&](int32_t X) -> uint32_t {
    const int32_t p = so + X;
    return (p >= sia && p < sib) ? (uint32_t)st[p] : (uint32_t)sb[X];
  };
  EncCursor cur = enc_cursor(mb, v);
  uint32_t wd[4];
  uint32_t n = 0;
  for (uint32_t k = 0; k < 4; ++k) {
    const int32_t Pk = P + 4 * (int32_t)k;
    if (Pk >= tile_len) break;
    if (Pk >= cur.oe) {
      mb = enc_bounds(a, owner_in(a.out_off, mb.j, v.jn + 1, v.a0 + Pk));
      cur = enc_cursor(mb, v);
    }
    const int32_t Xk = cur.xb + 3 * ((Pk - cur.ob) >> 2);
    const uint32_t cnt = (uint32_t)min(3, cur.xe - Xk);
    const uint32_t b0 = in_byte(Xk), b1 = cnt > 1 ? in_byte(Xk + 1) : 0u,
                   b2 = cnt > 2 ? in_byte(Xk + 2) : 0u;
    wd[k] = enc_tail_group(b0, b1, b2, cnt, T);
    n = k + 1;
  }
  uint8_t* d = a.dst + v.a0 + P;
  if (n == 4) {
    st_global_v4_cs(d, make_uint4(wd[0], wd[1], wd[2], wd[3]));
  } else {
    for (uint32_t k = 0; k < n; ++k) reinterpret_cast<uint32_t*>(d)[k] = wd[k];
  }
  return mb;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_flat_encode(FlatArgs a) {
  if (flat_declines(a)) return;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t T[64];
  __shared__ __align__(8) uint64_t full[kFlatMaxStages], empty[kFlatMaxStages];
  __shared__ FlatTile meta[kFlatMaxStages];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t S = a.stages;
  if (tid == 0) {
    for (uint32_t s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kFlatConsumerWarps);
    }
    fence_mbar_init();
  }
  init_tables(T, nullptr, a.flags & kFlagUrl);
  const int64_t in_total = __ldg(a.in_off + a.nmsg), out_total = __ldg(a.out_off + a.nmsg);
  const int64_t ntiles = (out_total + a.tile - 1) / a.tile;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_begin = (int64_t)blockIdx.x * per;
  const int64_t t_end = tmin<int64_t>(ntiles, t_begin + per);
  if (t_begin >= t_end) return;
  const uint32_t stage_b = (uint32_t)(a.tile / 4 * 3) + 32u;
  if (warp == 0) {
    flat_producer<0>(a, t_begin, t_end, in_total, out_total, smem, stage_b, full, empty, meta, lane);
    return;
  }
  const uint32_t ct = tid - 32u;  // consumer thread
  MsgBounds mb;                   // the message of this thread's last chunk
  uint32_t s = 0, phase = 0;
  for (int64_t t = t_begin; t < t_end; ++t) {
    const bool ok = mbar_wait_backoff(&full[s], phase);
    if (__any_sync(0xFFFFFFFFu, !ok)) {
      if (lane == 0) atomicOr(&g_flat_fault, 1u);
      return;
    }
    const FlatTile v = meta[s];
    const uint8_t* st = smem + s * stage_b;
    const uint8_t* sb = a.src + v.b0;  // input of the tile's first group
    uint8_t* dt = a.dst + v.a0;
    const int32_t tile_len = (int32_t)(v.a1 - v.a0);
    const int32_t so = (int32_t)v.o, sia = (int32_t)v.ia, sib = (int32_t)v.ib;
    int32_t P = 16 * (int32_t)ct;
    if (P < tile_len) {
      if (!(mb.o0 <= v.a0 + P && v.a0 + P < mb.o1))
        mb = enc_bounds(a, v.j0 == v.jn ? v.j0
                                        : owner_in(a.out_off, tmax<int64_t>(v.j0, mb.j), v.jn + 1,
                                                   v.a0 + P));
      EncCursor cur = enc_cursor(mb, v);
      for (; P < tile_len; P += 16 * kFlatConsumers) {
        if (P >= cur.oe) {
          mb = enc_bounds(a, owner_in(a.out_off, mb.j, v.jn + 1, v.a0 + P));
          cur = enc_cursor(mb, v);
        }
        const int32_t X = cur.xb + 3 * ((P - cur.ob) >> 2);
        if (P + 16 <= cur.oe && X + 12 <= cur.xe) {
          // four whole groups of one message: Algorithm 1 on a 12-byte unit
          const int32_t p = so + X;
          const uint3 w = (p >= sia && p + 12 <= sib) ? lds12(st + p)
                                                      : load12_any(sb + X, a.src, a.src + in_total);
          st_global_v4_cs(dt + P, enc_unit(w.x, w.y, w.z, T));
        } else {
          mb = enc_chunk_groups(a, v, mb, P, tile_len, st, T);
          cur = enc_cursor(mb, v);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (++s == S) {
      s = 0;
      phase ^= 1u;
    }
  }
}

// ----------------------------------------------------------------- decode

// 12 bytes (three little-endian words) to the image at any position.
__device__ __forceinline__ void img_put12(uint8_t* img, uint32_t p, uint3 o) {
  if ((p & 3u) == 0) {
    uint32_t* w = reinterpret_cast<uint32_t*>(img + p);
    w[0] = o.x;
    w[1] = o.y;
    w[2] = o.z;
    return;
  }
  const uint32_t r = p & 3u, sh = 8u * r;
  // bytes before the first aligned word, the two whole words, the rest
  uint8_t* q = img + p;
  for (uint32_t k = 0; k < 4 - r; ++k) q[k] = (uint8_t)(o.x >> (8 * k));
  uint32_t* w = reinterpret_cast<uint32_t*>(img + p + (4 - r));
  w[0] = __funnelshift_r(o.x, o.y, 32u - sh);
  w[1] = __funnelshift_r(o.y, o.z, 32u - sh);
  uint8_t* e = img + p + (12 - r);
  for (uint32_t k = 0; k < r; ++k) e[k] = (uint8_t)(o.z >> (8 * (4 - r + k)));
}

// Message j as one tile's units see it, in 32-bit positions relative to the
// tile's first character a0 (clamped to +-kFar): it covers [cs, ce), its
// body ends at cbody, its quads start at cb + 4k (aligned: cb is known, i.e.
// the message starts in the tile or a0 is a quad boundary of it), and the
// quad at cb writes output byte yb (relative to the tile's first output
// byte b0).
struct DecCursor {
  int32_t cs, ce, cbody, cb, yb;
  bool aligned;
};

// Decode bounds of message j: o0/o1 = its characters, i0 = its output
// offset, i1 = the end of its body (absolute character position).
__device__ __forceinline__ MsgBounds dec_bounds(const FlatArgs& a, int64_t j) {
  MsgBounds m;
  m.j = j;
  m.o0 = __ldg(a.in_off + j);
  m.o1 = __ldg(a.in_off + j + 1);
  m.i0 = __ldg(a.out_off + j);
  m.i1 = m.o0 + (int64_t)decode_body_end((uint64_t)(m.o1 - m.o0));
  return m;
}

__device__ __forceinline__ DecCursor dec_cursor(const MsgBounds& m, const FlatTile& v) {
  auto rel = [&](int64_t x) -> int32_t {
    return (int32_t)tmax<int64_t>(-kFar, tmin<int64_t>(x - v.a0, kFar));
  };
  DecCursor c;
  c.cs = rel(m.o0);
  c.ce = rel(m.o1);
  c.cbody = rel(m.i1);
  if (m.o0 > v.a0) {
    c.aligned = true;
    c.cb = (int32_t)(m.o0 - v.a0);
    c.yb = (int32_t)(m.i0 - v.b0);
  } else {
    c.aligned = ((v.a0 - m.o0) & 3) == 0;
    c.cb = 0;
    c.yb = (int32_t)(m.i0 + 3 * ((v.a0 - m.o0) / 4) - v.b0);
  }
  return c;
}

// Writes n (<= 3) bytes of v (high byte first) to the image at position p.
__device__ __forceinline__ void img_put3(uint8_t* img, uint32_t p, uint32_t val, uint32_t n) {
  img[p] = (uint8_t)(val >> 16);
  if (n > 1) img[p + 1] = (uint8_t)(val >> 8);
  if (n > 2) img[p + 2] = (uint8_t)val;
}

// Every group that starts in the unit [C, C + 16) of the tile, message by
// message from message j (which holds C): body quads one by one, and each
// message's final characters (decoded into the image, then the rest of its
// output capacity zeroed).
__device__ __forceinline__ void dec_unit_groups(const FlatArgs& a, const FlatTile& v,
                                             const StageReader& rd, const uint8_t* D,
                                             uint8_t* img, uint32_t o2, int64_t j, int32_t C) {
  auto img_pos = [&](int64_t Y) -> uint32_t { return o2 + (uint32_t)(Y - v.b0); };
  const int64_t Cabs = v.a0 + C;
  const int64_t cend = tmin<int64_t>(Cabs + 16, v.a1);
  int64_t i0 = __ldg(a.in_off + j);
  int64_t m = __ldg(a.in_off + j + 1) - i0;
  int64_t be = (int64_t)decode_body_end((uint64_t)m);
  while (true) {
    const int64_t q0 = tmax<int64_t>(Cabs, i0);
    int64_t q = i0 + ((q0 - i0 + 3) / 4) * 4;  // first group start of j at or after C
    const int64_t o0 = __ldg(a.out_off + j);
    for (; q < cend && q < i0 + be; q += 4) {
      uint32_t x = 0;
      for (uint32_t k = 0; k < 4; ++k) x |= rd.byte(q + k) << (8 * k);
      uint32_t err = 0;
      const uint32_t val = dec_quad(x, D, err);
      img_put3(img, img_pos(o0 + 3 * ((q - i0) / 4)), val, 3);
      if (err & kBadFlag) {
        for (uint32_t k = 0; k < 4; ++k)
          if (D[(x >> (8 * k)) & 0xFFu] & kBadFlag) {
            atomicMin(reinterpret_cast<unsigned long long*>(a.first_bad + j),
                      (unsigned long long)(q - i0 + k));
            break;
          }
      }
    }
    if (m > 0 && i0 + be >= Cabs && i0 + be < cend) {
      const int64_t ostart = o0 + 3 * (be / 4);
      uint8_t* base = img + img_pos(ostart) - 3 * (be / 4);
      const int r = dec_final_group(a.src + i0, (uint64_t)m, (uint64_t)be, base, D,
                                    reinterpret_cast<unsigned long long*>(a.first_bad + j),
                                    a.flags);
      a.outlen[j] = r;
      const int64_t cap_end = __ldg(a.out_off + j + 1);
      for (int64_t y = ostart + (r > 0 ? r : 0); y < cap_end; ++y) img[img_pos(y)] = 0;
    }
    // the next message, if it starts in this unit
    if (j + 1 >= a.nmsg) break;
    const int64_t nx = __ldg(a.in_off + j + 1);
    if (nx >= cend) break;
    ++j;
    i0 = nx;
    m = __ldg(a.in_off + j + 1) - i0;
    be = (int64_t)decode_body_end((uint64_t)m);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 3) k_flat_decode(FlatArgs a) {
  if (flat_declines(a)) return;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t D[256];
  __shared__ __align__(8) uint64_t full[kFlatMaxStages], empty[kFlatMaxStages];
  __shared__ __align__(8) uint64_t cbar;  // barrier of the consumer warps
  __shared__ FlatTile meta[kFlatMaxStages];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t S = a.stages;
  if (tid == 0) {
    for (uint32_t s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kFlatConsumerWarps);
    }
    mbar_init(&cbar, kFlatConsumerWarps);
    fence_mbar_init();
  }
  init_tables(nullptr, D, a.flags & kFlagUrl);
  const int64_t in_total = __ldg(a.in_off + a.nmsg), out_total = __ldg(a.out_off + a.nmsg);
  const int64_t ntiles = (in_total + a.tile - 1) / a.tile;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_begin = (int64_t)blockIdx.x * per;
  const int64_t t_end = tmin<int64_t>(ntiles, t_begin + per);
  if (t_begin >= t_end) return;
  const uint32_t stage_b = (uint32_t)a.tile + 48u;
  const uint32_t img_b = (uint32_t)(a.tile / 4 * 3) + 48u;
  uint8_t* imgs = smem + S * stage_b;
  if (warp == 0) {
    flat_producer<1>(a, t_begin, t_end, in_total, out_total, smem, stage_b, full, empty, meta, lane);
    return;
  }
  const uint32_t ct = tid - 32u;
  MsgBounds mb;  // the message of this thread's last unit
  // All consumer warps meet at cbar; the wait is bounded, so a warp that
  // gave up cannot leave the others blocked.
  uint32_t cphase = 0;
  auto consumers_meet = [&]() -> bool {
    __syncwarp();
    if (lane == 0) mbar_arrive(&cbar);
    const bool ok = mbar_wait_bounded(&cbar, cphase);
    cphase ^= 1u;
    return __all_sync(0xFFFFFFFFu, ok);
  };
  bool fault = false;
  uint32_t s = 0, phase = 0;
  for (int64_t t = t_begin; t < t_end; ++t) {
    const bool ok = mbar_wait_backoff(&full[s], phase);
    if (__any_sync(0xFFFFFFFFu, !ok)) {
      fault = true;
      break;
    }
    const FlatTile v = meta[s];
    const StageReader rd{smem + s * stage_b, a.src, v.a0, in_total, v.o, v.ia, v.ib};
    // the image buffer of this tile: the bulk store that last read it (two
    // tiles ago) has finished reading
    const uint32_t buf = (uint32_t)((t - t_begin) & 1);
    uint8_t* img = imgs + buf * img_b;
    if (ct == 0 && t - t_begin >= 2) bulk_wait_read(1);
    if (!consumers_meet()) {
      fault = true;
      break;
    }
    const uintptr_t dA = reinterpret_cast<uintptr_t>(a.dst + v.b0);
    const uint32_t o2 = (uint32_t)(dA & 15u);

    const int32_t tile_len = (int32_t)(v.a1 - v.a0);
    const uint8_t* st = rd.stage;
    int32_t C = 16 * (int32_t)ct;
    if (C < tile_len) {
      if (!(mb.o0 <= v.a0 + C && v.a0 + C < mb.o1))
        mb = dec_bounds(a, v.j0 == v.jn ? v.j0
                                        : owner_in(a.in_off, tmax<int64_t>(v.j0, mb.j), v.jn + 1,
                                                   v.a0 + C));
      DecCursor cur = dec_cursor(mb, v);
      for (; C < tile_len; C += 16 * kFlatConsumers) {
        if (C >= cur.ce) {
          mb = dec_bounds(a, owner_in(a.in_off, mb.j, v.jn + 1, v.a0 + C));
          cur = dec_cursor(mb, v);
        }
        if (cur.aligned && ((C - cur.cb) & 3) == 0 && C + 16 <= cur.cbody && C + 16 <= tile_len) {
          // four body quads of one message: Algorithm 2 on a 16-character unit
          const uint4 w = (v.o == 0 && C + 16 <= (int32_t)v.ib)
                              ? *reinterpret_cast<const uint4*>(st + C)
                              : load16_any(a.src + v.a0 + C, a.src, a.src + in_total);
          uint32_t err = 0;
          const uint3 o = dec_unit(w, D, err);
          img_put12(img, o2 + (uint32_t)(cur.yb + 3 * ((C - cur.cb) >> 2)), o);
          if (err & kBadFlag)
            atomicMin(reinterpret_cast<unsigned long long*>(a.first_bad + mb.j),
                      (unsigned long long)(v.a0 + C - mb.o0 + dec_unit_first_bad(w, D)));
        } else {
          dec_unit_groups(a, v, rd, D, img, o2, mb.j, C);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // the input stage is free
    // the image is complete: its aligned interior leaves by one bulk store
    fence_proxy_async_smem();
    if (!consumers_meet()) {
      fault = true;
      break;
    }
    {
      uint8_t* d = a.dst + v.b0;
      const uint32_t olen = (uint32_t)(v.b1 - v.b0);
      const uintptr_t da = reinterpret_cast<uintptr_t>(d);
      const uintptr_t lo = (da + 15u) & ~(uintptr_t)15u, hi = (da + olen) & ~(uintptr_t)15u;
      if (ct == 0) {
        if (hi > lo) tma_store_1d(reinterpret_cast<void*>(lo), img + (o2 ? 16u : 0u), (uint32_t)(hi - lo));
        bulk_commit();
      }
      const uint32_t head = (uint32_t)(tmin<uintptr_t>(lo, da + olen) - da);
      const uint32_t ie = hi > lo ? (uint32_t)(hi - da) : head;
      if (ct < head) {
        d[ct] = img[o2 + ct];
      } else if (ct >= 32u && ct - 32u < olen - ie) {
        d[ie + ct - 32u] = img[o2 + ie + ct - 32u];
      }
    }
    if (++s == S) {
      s = 0;
      phase ^= 1u;
    }
  }
  if (fault && lane == 0) atomicOr(&g_flat_fault, 1u);
  if (ct == 0) bulk_wait_all();
}

}  // namespace

size_t flat_smem_bytes(int decode, int64_t tile, int stages) {
  if (!decode) return (size_t)stages * (size_t)(tile / 4 * 3 + 32);
  return (size_t)stages * (size_t)(tile + 48) + 2 * (size_t)(tile / 4 * 3 + 48);
}

bool flat_eligible(int decode, const uint8_t* src, const uint8_t* dst, uint32_t flags) {
  if (decode) return (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
  return !(flags & kFlagNoPad) && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0;
}

cudaError_t flat_launch(int decode, const uint8_t* src, const int64_t* in_off, uint8_t* dst,
                        const int64_t* out_off, int64_t nmsg, int64_t* first_bad, int64_t* outlen,
                        const FlatConfig& cfg, uint32_t flags, cudaStream_t stream,
                        int64_t max_mean_len) {
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  const size_t smem = flat_smem_bytes(decode, cfg.tile, cfg.stages);
  const void* kernel = decode ? reinterpret_cast<const void*>(k_flat_decode<kFlatThreads>)
                              : reinterpret_cast<const void*>(k_flat_encode<kFlatThreads>);
  int fit = 0;
  e = kernel_prepare(kernel, smem, kFlatThreads, &fit);
  if (e != cudaSuccess) return e;
  if (fit < 1) return cudaErrorInvalidConfiguration;
  const int bps = cfg.blocks_per_sm > 0 ? std::min(fit, cfg.blocks_per_sm) : fit;
  FlatArgs a{src,   in_off,   dst,        out_off, nmsg, cfg.tile, (uint32_t)cfg.stages,
             flags, first_bad, outlen, max_mean_len};
  if (decode) {
    k_flat_decode<kFlatThreads><<<di->sm_count * bps, kFlatThreads, smem, stream>>>(a);
  } else {
    k_flat_encode<kFlatThreads><<<di->sm_count * bps, kFlatThreads, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

bool flat_config_valid(int decode, const FlatConfig& c) {
  const int64_t q = 16 * kFlatConsumers;
  if (c.tile < q || c.tile > 64 * q || c.tile % q) return false;
  if (c.stages < 2 || c.stages > kFlatMaxStages || c.blocks_per_sm < 0 || c.blocks_per_sm > 8)
    return false;
  return flat_smem_bytes(decode, c.tile, c.stages) <= kBatchSmemLimit;
}

// Mean message lengths below which the flat kernels code a packed batch
// faster than the per-warp tile kernels (measured on GB300 over lengths
// 16 B .. 1 MiB: the per-warp kernels win from about 256-byte payloads).
int64_t flat_mean_len_threshold(int decode) { return decode ? 256 : 384; }

FlatConfig default_flat_config(int decode) {
  return decode ? FlatConfig{16384, 3, 0} : FlatConfig{16384, 4, 0};
}

int flat_read_and_clear_fault(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_flat_fault, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_flat_fault, &zero, sizeof(zero));
  *out = v;
  return e == cudaSuccess ? 0 : cuda_status(e, "reading the fault word");
}

}  // namespace gb64
