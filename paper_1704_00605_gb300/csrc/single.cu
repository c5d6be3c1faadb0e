// Single-buffer encode and decode kernels.
//
// Fast path (src and dst 16-byte aligned): a persistent grid of CTAs, a few
// per SM, walks the buffer in tiles. One elected thread per CTA streams each
// tile into a ring of shared-memory stages with 1-D TMA bulk copies
// (cp.async.bulk + mbarrier transaction counts), so tens of kilobytes per SM
// are in flight while the CTA codes earlier tiles.
//   encode: tile = threads * upt * 12 bytes -> threads * upt * 16 characters;
//           each thread reads 12 bytes (three conflict-free 32-bit shared
//           loads), regroups them with prmt into four groups (Algorithm 1's
//           main loop), maps the 6-bit values through the shared alphabet
//           table, and writes 16 characters with one coalesced 16-byte store.
//   decode: tile = threads * upt * 16 characters -> threads * upt * 12 bytes;
//           each thread reads 16 characters (one 16-byte shared load), looks
//           each up in the shared 256-entry table (value or invalid flag),
//           packs four quads into 12 bytes (Algorithm 2's main loop), stages
//           them in shared memory, and one thread writes the tile back with a
//           TMA bulk store. A warp that saw a flagged character rescans its
//           units, reduces the first bad index with __reduce_min_sync and
//           lowers the global first_bad with one atomicMin.
// The last partial group (encode) and the final quad or partial quad (decode)
// are coded by one thread from global memory with the padding rules.
//
// Generic path (any alignment): grid-stride over 12-byte / 16-character
// units with aligned-word loads and funnel shifts, byte loads at the buffer
// ends, and stores split to the alignment of the destination.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gb64 {

constexpr int kMaxStages = 8;

// Set by a kernel that gave up on a bounded wait (read by b64_device_fault).
static __device__ unsigned int g_single_fault;

struct EncArgs {
  const uint8_t* src;
  uint64_t n;
  uint8_t* dst;
  uint32_t upt;
  uint32_t stages;
  uint32_t flags;
  uint32_t stall;    // test: CTA 0 leaves out its first copy
  uint64_t wait_ns;  // limit of the stage waits
};

struct DecArgs {
  const uint8_t* src;
  uint64_t m;
  uint64_t body_end;
  uint8_t* dst;
  b64_result* res;
  uint32_t upt;
  uint32_t stages;
  uint32_t flags;
  uint32_t stall;     // test: CTA 0 leaves out its first copy
  uint64_t wait_ns;  // limit of the stage waits
};

// ------------------------------------------------------------- encode/TMA
// FLAGS (kFlagUrl | kFlagNoPad) is a compile-time parameter: the default
// instantiation (0) carries no variant code at all.
template <int NT, uint32_t FLAGS>
__global__ void __launch_bounds__(NT) k_encode_tma(EncArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t T[64];
  __shared__ __align__(8) uint64_t full[kMaxStages];

  const uint32_t tid = threadIdx.x;
  const uint32_t S = a.stages;
  const uint32_t tile_in = NT * a.upt * 12u;
  const uint64_t ntiles = (a.n + tile_in - 1) / tile_in;

  if (tid == 0) {
    for (uint32_t s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  init_tables(T, nullptr, (FLAGS & kFlagUrl) != 0);

  auto issue = [&](uint64_t t, uint32_t s) {
    const uint64_t off = t * tile_in;
    const uint32_t len = (uint32_t)tmin<uint64_t>(tile_in, a.n - off);
    const uint32_t bytes = len & ~15u;
    if (bytes) {
      fence_proxy_async_smem();  // earlier generic reads of this stage come first
      mbar_arrive_expect_tx(&full[s], bytes);
      tma_load_1d(smem + (size_t)s * tile_in, a.src + off, bytes, &full[s]);
    } else {
      mbar_arrive(&full[s]);
    }
  };

  if (tid == 0) {
    fence_proxy_async_smem();
    for (uint32_t s = 0; s < S; ++s) {
      const uint64_t t = blockIdx.x + (uint64_t)s * gridDim.x;
      if (t < ntiles && !(a.stall && t == 0)) issue(t, s);
    }
  }

  uint32_t k = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const uint32_t s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], (k / S) & 1u, a.wait_ns);
    const uint64_t off = t * tile_in;
    const uint32_t len = (uint32_t)tmin<uint64_t>(tile_in, a.n - off);
    const uint32_t nu = (len & ~15u) / 12u;
    const uint32_t* buf = reinterpret_cast<const uint32_t*>(smem + (size_t)s * tile_in);
    uint8_t* out = a.dst + off / 3 * 4;
#pragma unroll 4
    for (uint32_t u = tid; u < nu; u += NT) {
      const uint4 o = enc_unit(buf[3 * u], buf[3 * u + 1], buf[3 * u + 2], T);
      st_global_v4_cs(out + 16 * (size_t)u, o);
    }
    if (len != tile_in) {
      // bytes past the last whole unit of the final tile: read from global
      const uint32_t done = 12u * nu;
      const uint32_t rest = len - done;
      const uint32_t ng = (rest + 2) / 3;
      for (uint32_t g = tid; g < ng; g += NT) {
        const uint8_t* p = a.src + off + done + 3 * g;
        const uint32_t cnt = min(3u, rest - 3 * g);
        const uint32_t b0 = p[0], b1 = cnt > 1 ? p[1] : 0u, b2 = cnt > 2 ? p[2] : 0u;
        if (FLAGS & kFlagNoPad)
          store_tail_group(out + 16 * (size_t)nu + 4 * g, enc_tail_group(b0, b1, b2, cnt, T), cnt,
                           kFlagNoPad);
        else
          store4_any(out + 16 * (size_t)nu + 4 * g, enc_tail_group(b0, b1, b2, cnt, T));
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&g_single_fault, 1u);
        for (uint32_t j = 0; j < S; ++j) {  // drain this CTA's copies in flight
          const uint32_t kk = k + j;
          const uint64_t tt = blockIdx.x + (uint64_t)kk * gridDim.x;
          if (tt < ntiles) mbar_wait_bounded(&full[kk % S], (kk / S) & 1u, 500000000ull);
        }
      }
      return;
    }
    if (tid == 0) {
      const uint64_t t2 = t + (uint64_t)S * gridDim.x;
      if (t2 < ntiles) issue(t2, s);
    }
  }
}

// ---------------------------------------------------------- encode/generic
template <int NT>
__global__ void __launch_bounds__(NT) k_encode_any(const uint8_t* __restrict__ src, uint64_t n,
                                                   uint8_t* __restrict__ dst, uint32_t flags) {
  __shared__ uint8_t T[64];
  init_tables(T, nullptr, flags & kFlagUrl);
  const uint64_t nunits = n / 12;
  const uint64_t stride = (uint64_t)gridDim.x * NT;
  for (uint64_t u = (uint64_t)blockIdx.x * NT + threadIdx.x; u < nunits; u += stride) {
    const uint3 w = load12_any(src + 12 * u, src, src + n);
    store16_any(dst + 16 * u, enc_unit(w.x, w.y, w.z, T));
  }
  if (blockIdx.x == 0) {
    const uint64_t done = 12 * nunits;
    const uint32_t rest = (uint32_t)(n - done);
    const uint32_t ng = (rest + 2) / 3;
    if (threadIdx.x < ng) {
      const uint32_t g = threadIdx.x;
      const uint8_t* p = src + done + 3 * g;
      const uint32_t cnt = min(3u, rest - 3 * g);
      const uint32_t b0 = p[0], b1 = cnt > 1 ? p[1] : 0u, b2 = cnt > 2 ? p[2] : 0u;
      store_tail_group(dst + 16 * nunits + 4 * g, enc_tail_group(b0, b1, b2, cnt, T), cnt, flags);
    }
  }
}

// ------------------------------------------------------- decode helpers
// Decodes one whole quad of the body read from global memory at p (index
// idx), writes its 3 bytes to out; returns the first bad index or ~0.
__device__ __forceinline__ unsigned long long dec_body_quad(const uint8_t* p, uint64_t idx,
                                                            uint8_t* out, const uint8_t* D) {
  const uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
                     ((uint32_t)p[3] << 24);
  uint32_t err = 0;
  const uint32_t v = dec_quad(x, D, err);
  if (err & kBadFlag) {
    for (uint32_t k = 0; k < 4; ++k)
      if (D[(x >> (8 * k)) & 0xFFu] & kBadFlag) return idx + k;
  }
  out[0] = (uint8_t)(v >> 16);
  out[1] = (uint8_t)(v >> 8);
  out[2] = (uint8_t)v;
  return ~0ull;
}

// Runs in every CTA after its work: the last CTA to arrive computes the
// status (first bad character wins, then the length rule).
__device__ void dec_finish(const DecArgs& a, bool timed_out) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (timed_out) atomicOr(&g_single_fault, 1u);
  const unsigned prev = atomicAdd(&a.res->internal, 1u);
  if (prev != gridDim.x - 2u) return;  // counter starts at 0xFFFFFFFF
  __threadfence();
  volatile b64_result* r = a.res;
  const unsigned long long fb =
      atomicAdd(reinterpret_cast<unsigned long long*>(&a.res->first_bad), 0ull);
  const bool fault = atomicAdd(&g_single_fault, 0u) != 0;
  const int64_t final_bytes = (a.body_end < a.m) ? r->outlen : 0;
  if (fault) {
    r->first_bad = (int64_t)a.m;
    r->outlen = 0;
    r->status = B64_ERR_TIMEOUT;
  } else {
    const FinalStatus f = final_status(a.m, a.body_end, fb, final_bytes, a.flags);
    r->first_bad = f.first_bad;
    r->outlen = f.outlen;
    r->status = f.status;
  }
  __threadfence();
}

// ------------------------------------------------------------- decode/TMA
template <int NT>
__global__ void __launch_bounds__(NT) k_decode_tma(DecArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint8_t D[256];
  __shared__ __align__(8) uint64_t full[kMaxStages];

  const uint32_t tid = threadIdx.x;
  const uint32_t S = a.stages;
  const uint32_t tile_c = NT * a.upt * 16u;
  const uint32_t tile_o = NT * a.upt * 12u;
  const uint64_t ntiles = (a.m + tile_c - 1) / tile_c;
  unsigned long long* first_bad = reinterpret_cast<unsigned long long*>(&a.res->first_bad);
  uint8_t* outbuf0 = smem + (size_t)S * tile_c;

  if (tid == 0) {
    for (uint32_t s = 0; s < S; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  init_tables(nullptr, D, a.flags & kFlagUrl);

  auto issue = [&](uint64_t t, uint32_t s) {
    const uint64_t off = t * tile_c;
    const uint32_t len = (uint32_t)tmin<uint64_t>(tile_c, a.m - off);
    const uint32_t bytes = len & ~15u;
    if (bytes) {
      fence_proxy_async_smem();  // earlier generic reads of this stage come first
      mbar_arrive_expect_tx(&full[s], bytes);
      tma_load_1d(smem + (size_t)s * tile_c, a.src + off, bytes, &full[s]);
    } else {
      mbar_arrive(&full[s]);
    }
  };

  if (tid == 0) {
    fence_proxy_async_smem();
    for (uint32_t s = 0; s < S; ++s) {
      const uint64_t t = blockIdx.x + (uint64_t)s * gridDim.x;
      if (t < ntiles && !(a.stall && t == 0)) issue(t, s);
    }
  }

  bool timed_out = false;
  uint32_t k = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const uint32_t s = k % S;
    const bool ok = mbar_wait_bounded(&full[s], (k / S) & 1u, a.wait_ns);
    const uint64_t off = t * tile_c;
    const uint32_t len = (uint32_t)tmin<uint64_t>(tile_c, a.m - off);
    const uint32_t body =
        a.body_end > off ? (uint32_t)tmin<uint64_t>(len, a.body_end - off) : 0u;
    const uint32_t nu = min(len & ~15u, body) / 16u;
    const uint4* in = reinterpret_cast<const uint4*>(smem + (size_t)s * tile_c);
    uint32_t* ob = reinterpret_cast<uint32_t*>(outbuf0 + (size_t)(k & 1u) * tile_o);

    uint32_t err = 0;
#pragma unroll 4
    for (uint32_t u = tid; u < nu; u += NT) {
      const uint3 o = dec_unit(in[u], D, err);
      ob[3 * u] = o.x;
      ob[3 * u + 1] = o.y;
      ob[3 * u + 2] = o.z;
    }
    unsigned long long bad = ~0ull;
    if (err & kBadFlag) {
      for (uint32_t u = tid; u < nu; u += NT) {
        const uint32_t j = dec_unit_first_bad(in[u], D);
        if (j < 16) {
          bad = off + 16ull * u + j;
          break;
        }
      }
    }
    warp_min_to(first_bad, bad);

    // whole quads of the body after the last whole unit of the tile
    const uint32_t q0 = 16u * nu;
    const uint32_t nq = (body - q0) / 4u;
    for (uint32_t q = tid; q < nq; q += NT) {
      const uint64_t idx = off + q0 + 4 * q;
      const unsigned long long b = dec_body_quad(a.src + idx, idx, a.dst + idx / 4 * 3, D);
      if (b != ~0ull) atomicMin(first_bad, b);
    }
    // final characters of the message
    if (tid == NT - 1 && a.body_end >= off && a.body_end < off + len) {
      a.res->outlen = dec_final_group(a.src, a.m, a.body_end, a.dst, D, first_bad, a.flags);
    }

    fence_proxy_async_smem();
    if (tid == 0) bulk_wait_read_all();  // the other output buffer is free again
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      if (tid == 0) {
        for (uint32_t j = 0; j < S; ++j) {
          const uint32_t kk = k + j;
          const uint64_t tt = blockIdx.x + (uint64_t)kk * gridDim.x;
          if (tt < ntiles) mbar_wait_bounded(&full[kk % S], (kk / S) & 1u, 500000000ull);
        }
      }
      break;
    }
    if (tid == 0) {
      const uint32_t ob_bytes = 12u * nu;
      const uint32_t sb = ob_bytes & ~15u;
      uint8_t* gout = a.dst + off / 4 * 3;
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
  dec_finish(a, timed_out);
}

// --------------------------------------------------------- decode/generic
template <int NT>
__global__ void __launch_bounds__(NT) k_decode_any(DecArgs a) {
  __shared__ uint8_t D[256];
  init_tables(nullptr, D, a.flags & kFlagUrl);
  unsigned long long* first_bad = reinterpret_cast<unsigned long long*>(&a.res->first_bad);
  const uint64_t nunits = a.body_end / 16;
  const uint64_t stride = (uint64_t)gridDim.x * NT;
  const uint32_t lane = threadIdx.x & 31u;
  unsigned long long bad = ~0ull;
  for (uint64_t base = (uint64_t)blockIdx.x * NT; base < nunits; base += stride) {
    // consecutive lanes own consecutive units and store them together
    const uint64_t u = base + threadIdx.x;
    uint3 o = make_uint3(0, 0, 0);
    if (u < nunits) {
      const uint4 w = load16_any(a.src + 16 * u, a.src, a.src + a.m);
      uint32_t err = 0;
      o = dec_unit(w, D, err);
      if ((err & kBadFlag) && bad == ~0ull) bad = 16 * u + dec_unit_first_bad(w, D);
    }
    const uint64_t u0 = base + (threadIdx.x & ~31u);
    if (u0 < nunits)
      store12_warp(a.dst + 12 * u0, o, lane, (uint32_t)tmin<uint64_t>(32, nunits - u0));
  }
  warp_min_to(first_bad, bad);
  if (blockIdx.x == 0) {
    const uint64_t q0 = 16 * nunits;
    const uint32_t nq = (uint32_t)((a.body_end - q0) / 4);
    if (threadIdx.x < nq) {
      const uint64_t idx = q0 + 4 * threadIdx.x;
      const unsigned long long b = dec_body_quad(a.src + idx, idx, a.dst + idx / 4 * 3, D);
      if (b != ~0ull) atomicMin(first_bad, b);
    }
    if (threadIdx.x == NT - 1 && a.body_end < a.m) {
      a.res->outlen = dec_final_group(a.src, a.m, a.body_end, a.dst, D, first_bad, a.flags);
    }
  }
  dec_finish(a, false);
}

// ------------------------------------------------------------------ host
// Shapes measured fastest on GB300 for buffers of 256 MiB and more (one CTA
// of 512 threads per SM, 48 KiB / 64 KiB TMA tiles), and a smaller tile for
// smaller buffers so that every SM still gets tiles.
TileConfig default_encode_config(uint64_t n) {
  return n >= (256ull << 20) ? TileConfig{512, 8, 4, 0} : TileConfig{256, 4, 4, 0};
}
TileConfig default_decode_config(uint64_t m) {
  return m >= (256ull << 20) ? TileConfig{512, 8, 2, 0} : TileConfig{256, 4, 3, 0};
}

size_t single_smem_bytes(int decode, const TileConfig& c) {
  const size_t tile = (size_t)c.threads * c.upt * (decode ? 16 : 12);
  return (size_t)c.stages * tile + (decode ? 2 * (size_t)c.threads * c.upt * 12 : 0);
}

// Raises the kernel's dynamic shared-memory limit to the device maximum
// (once per device and kernel: the limit belongs to the kernel, not to one
// launch) and returns how many CTAs of smem_bytes fit per SM (cached per
// device, kernel, size and block size, so small launches pay it once).
cudaError_t kernel_prepare(const void* kernel, size_t smem_bytes, int threads, int* blocks_per_sm) {
  struct Key {
    int device;
    const void* kernel;
    size_t smem;  // ~0 marks the entry recording the raised limit
    int threads;
    int bps;      // CTAs per SM, or the dynamic limit in the ~0 entry
  };
  static std::mutex mu;
  static std::vector<Key> cache;
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  const void* kp = kernel;
  std::lock_guard<std::mutex> g(mu);
  bool raised = false;
  for (const Key& k : cache) {
    if (k.device != di->device || k.kernel != kp) continue;
    if (k.smem == ~size_t(0)) raised = true;
    if (k.smem == smem_bytes && k.threads == threads) {
      *blocks_per_sm = k.bps;
      return cudaSuccess;
    }
  }
  if (!raised) {
    // dynamic + static shared memory of a CTA must stay within the opt-in limit
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    const int limit = di->max_smem_optin - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
    if (e != cudaSuccess) return e;
    cache.push_back(Key{di->device, kp, ~size_t(0), 0, limit});
  }
  for (const Key& k : cache)
    if (k.device == di->device && k.kernel == kp && k.smem == ~size_t(0) &&
        (int)smem_bytes > k.bps)
      return cudaErrorInvalidValue;  // the shape does not fit this device
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, threads, smem_bytes);
  if (e != cudaSuccess) return e;
  cache.push_back(Key{di->device, kp, smem_bytes, threads, *blocks_per_sm});
  return cudaSuccess;
}

namespace {

bool valid_config(const TileConfig& c) {
  return (c.threads == 128 || c.threads == 256 || c.threads == 512) && c.upt >= 1 &&
         c.upt <= 16 && c.stages >= 2 && c.stages <= kMaxStages && c.blocks_per_sm >= 0;
}

int resident_ctas(int fitting, const TileConfig& c) {
  return c.blocks_per_sm > 0 ? std::min(fitting, c.blocks_per_sm) : fitting;
}

template <int NT>
cudaError_t launch_encode_nt(const uint8_t* src, uint64_t n, uint8_t* dst, cudaStream_t stream,
                             const TileConfig& cfg, const DeviceInfo* di, uint32_t flags) {
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) &
                        15u) == 0;
  if (aligned) {
    const WaitTest wt = wait_test();
    EncArgs a{src, n, dst, (uint32_t)cfg.upt, (uint32_t)cfg.stages, flags, wt.stall, wt.limit_ns};
    const uint64_t tile_in = (uint64_t)NT * cfg.upt * 12u;
    const size_t smem = (size_t)cfg.stages * tile_in;
    const uint32_t f = flags & (kFlagUrl | kFlagNoPad);
    auto kernel = f == 0                          ? k_encode_tma<NT, 0>
                  : f == kFlagUrl                 ? k_encode_tma<NT, kFlagUrl>
                  : f == kFlagNoPad               ? k_encode_tma<NT, kFlagNoPad>
                                                  : k_encode_tma<NT, kFlagUrl | kFlagNoPad>;
    int bps = 0;
    cudaError_t e = kernel_prepare(reinterpret_cast<const void*>(kernel), smem, NT, &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const uint64_t ntiles = (n + tile_in - 1) / tile_in;
    const int grid =
        (int)std::min<uint64_t>(ntiles, (uint64_t)di->sm_count * resident_ctas(bps, cfg));
    kernel<<<grid, NT, smem, stream>>>(a);
    return cudaGetLastError();
  }
  const uint64_t units = n / 12 + 1;
  const int grid =
      (int)std::max<uint64_t>(1, std::min<uint64_t>((units + NT - 1) / NT, (uint64_t)di->sm_count * 8));
  k_encode_any<NT><<<grid, NT, 0, stream>>>(src, n, dst, flags);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_decode_nt(const DecArgs& a0, cudaStream_t stream, const TileConfig& cfg,
                             const DeviceInfo* di) {
  DecArgs a = a0;
  a.upt = (uint32_t)cfg.upt;
  a.stages = (uint32_t)cfg.stages;
  const WaitTest wt = wait_test();
  a.stall = wt.stall;
  a.wait_ns = wt.limit_ns;
  const bool aligned =
      ((reinterpret_cast<uintptr_t>(a.src) | reinterpret_cast<uintptr_t>(a.dst)) & 15u) == 0;
  if (aligned) {
    const uint64_t tile_c = (uint64_t)NT * cfg.upt * 16u;
    const uint64_t tile_o = (uint64_t)NT * cfg.upt * 12u;
    const size_t smem = (size_t)cfg.stages * tile_c + 2 * tile_o;
    int bps = 0;
    cudaError_t e =
        kernel_prepare(reinterpret_cast<const void*>(k_decode_tma<NT>), smem, NT, &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const uint64_t ntiles = std::max<uint64_t>(1, (a.m + tile_c - 1) / tile_c);
    const int grid =
        (int)std::min<uint64_t>(ntiles, (uint64_t)di->sm_count * resident_ctas(bps, cfg));
    k_decode_tma<NT><<<grid, NT, smem, stream>>>(a);
    return cudaGetLastError();
  }
  const uint64_t units = a.m / 16 + 1;
  const int grid =
      (int)std::max<uint64_t>(1, std::min<uint64_t>((units + NT - 1) / NT, (uint64_t)di->sm_count * 8));
  k_decode_any<NT><<<grid, NT, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_decode_any_nt(const DecArgs& a, cudaStream_t stream, const TileConfig& cfg) {
  if (!valid_config(cfg)) return cudaErrorInvalidValue;
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  switch (cfg.threads) {
    case 128: return launch_decode_nt<128>(a, stream, cfg, di);
    case 512: return launch_decode_nt<512>(a, stream, cfg, di);
    default: return launch_decode_nt<256>(a, stream, cfg, di);
  }
}

}  // namespace

cudaError_t launch_encode(const uint8_t* src, uint64_t n, uint8_t* dst, cudaStream_t stream,
                          const TileConfig& cfg, uint32_t flags) {
  if (!valid_config(cfg)) return cudaErrorInvalidValue;
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return e;
  switch (cfg.threads) {
    case 128: return launch_encode_nt<128>(src, n, dst, stream, cfg, di, flags);
    case 512: return launch_encode_nt<512>(src, n, dst, stream, cfg, di, flags);
    default: return launch_encode_nt<256>(src, n, dst, stream, cfg, di, flags);
  }
}

cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint64_t body_end, uint8_t* dst,
                          b64_result* res, cudaStream_t stream, const TileConfig& cfg,
                          uint32_t flags) {
  DecArgs a{src, m, body_end, dst, res, 0, 0, flags, 0, 0};
  return launch_decode_any_nt(a, stream, cfg);
}

int single_read_and_clear_fault(unsigned int* out) {
  unsigned int v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_single_fault, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_single_fault, &zero, sizeof(zero));
  *out = v;
  return e == cudaSuccess ? 0 : cuda_status(e, "reading the fault word");
}

}  // namespace gb64
