// Autotuner of launch shapes.
//
// Every kernel family has a table of shapes indexed by size bucket:
//   single encode/decode  bucket = input size class (<64 KiB, <1 MiB,
//                         <16 MiB, <256 MiB, larger); shape = threads per
//                         CTA, units per thread per tile (tile size), TMA
//                         stages, CTAs per SM;
//   batched encode/decode bucket = mean message length class (<256 B, <1 KiB,
//                         <4 KiB, <16 KiB, <64 KiB, <256 KiB, larger, unknown);
//                         shape = threads per CTA, tile size, CTAs per SM.
// b64_tune times every candidate shape of a family on device-generated data
// of the requested size (CUDA events, median of several runs), stores the
// fastest in the table and reports all trials. b64_tune_save/b64_tune_load
// persist the table; GB64_TUNE_FILE names a file loaded at first use.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "tuner.h"

namespace gb64 {
namespace {

struct Entry {
  bool set = false;
  b64_shape s{};
};

std::mutex g_mu;
Entry g_table[kKinds][kBuckets];
bool g_loaded = false;

int load_file_locked(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return B64_ERR_ARG;
  int kind, bucket, threads, upt, stages, bps;
  long long tile;
  float ms;
  while (fscanf(f, "%d %d %d %d %d %d %lld %f", &kind, &bucket, &threads, &upt, &stages, &bps,
                &tile, &ms) == 8) {
    if (kind < 0 || kind >= kKinds || bucket < 0 || bucket >= kBuckets) continue;
    Entry& e = g_table[kind][bucket];
    e.set = true;
    e.s = b64_shape{threads, upt, stages, bps, (int64_t)tile, ms};
  }
  fclose(f);
  return B64_OK;
}

void load_env_once_locked() {
  if (g_loaded) return;
  g_loaded = true;
  if (const char* p = getenv("GB64_TUNE_FILE")) load_file_locked(p);
}

BatchConfig batch_config_of(const b64_shape& s) {
  BatchConfig c{s.threads, s.tile, s.blocks_per_sm};
  c.stages = s.stages ? s.stages : 4;
  c.kernel = s.units_per_thread;  // batch kinds: the kernel choice
  return c;
}

bool shape_valid(int kind, const b64_shape& s) {
  if (kind == kDecodeWs)
    return ws_lines_config_valid(TileConfig{s.threads, s.units_per_thread, s.stages, 0});
  if (kind == kSingleEncode || kind == kSingleDecode) {
    TileConfig c{s.threads, s.units_per_thread, s.stages, s.blocks_per_sm};
    return (c.threads == 128 || c.threads == 256 || c.threads == 512) && c.upt >= 1 &&
           c.upt <= 16 && c.stages >= 2 && c.stages <= 8 && c.blocks_per_sm >= 0;
  }
  return batch_config_valid(kind == kBatchDecode, batch_config_of(s));
}

__global__ void k_fill_random(uint8_t* p, uint64_t n, uint64_t seed) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n + 7) / 8; i += stride) {
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    for (int k = 0; k < 8 && 8 * i + k < n; ++k) p[8 * i + k] = (uint8_t)(z >> (8 * k));
  }
}

struct DeviceBuffers {
  std::vector<void*> ptrs;
  ~DeviceBuffers() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
};

// Median of `reps` timed runs of fn (which enqueues on stream).
template <typename F>
cudaError_t time_median(F fn, cudaStream_t stream, int reps, float* ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return e;
  e = fn();  // warm-up
  std::vector<float> t;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, stream);
    if (e == cudaSuccess) e = fn();
    if (e == cudaSuccess) e = cudaEventRecord(b, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float x = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, a, b);
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return cudaSuccess;
}

std::vector<b64_shape> single_candidates(int decode, const DeviceInfo* di) {
  std::vector<b64_shape> out;
  const int unit = decode ? 16 : 12;
  for (int threads : {128, 256, 512})
    for (int upt : {1, 2, 4, 8})
      for (int stages : {2, 3, 4, 6})
        for (int bps : {0, 2}) {
          const int64_t tile = (int64_t)threads * upt * unit;
          const int64_t out_tile = decode ? 2 * (int64_t)threads * upt * 12 : 0;
          const int64_t smem = stages * tile + out_tile + 1024;
          if (tile < 4096 || tile > 65536 || smem > di->max_smem_optin) continue;
          out.push_back(b64_shape{threads, upt, stages, bps, tile, 0.f});
        }
  return out;
}

std::vector<b64_shape> batch_candidates(int decode) {
  std::vector<b64_shape> out;
  const int64_t row = decode ? 512 : 384;
  for (int threads : {128, 256})
    for (int rows : {2, 4, 8, 12, 16})
      for (int stages : {2, 3, 4, 6}) {  // staged tiles (kernel choice 0)
        const b64_shape s{threads, 0, stages, 0, row * rows, 0.f};
        if (batch_config_valid(decode, batch_config_of(s))) out.push_back(s);
      }
  for (int threads : {128, 256})
    for (int rows : {8, 16, 32, 64}) {  // unstaged tiles (kernel choice 2)
      const b64_shape s{threads, 2, 2, 0, row * rows, 0.f};
      if (batch_config_valid(decode, batch_config_of(s))) out.push_back(s);
    }
  for (int rows : {8, 32}) {  // the flat kernels, unstaged tiles otherwise (choice 3)
    const b64_shape s{decode ? 128 : 256, 3, 2, 0, row * rows, 0.f};
    if (batch_config_valid(decode, batch_config_of(s))) out.push_back(s);
  }
  return out;
}

}  // namespace

int bucket_of(int kind, int64_t total, int64_t nmsg) {
  if (kind == kSingleEncode || kind == kSingleDecode || kind == kDecodeWs) {
    const int64_t n = total < 0 ? 0 : total;
    if (n < (1ll << 16)) return 0;
    if (n < (1ll << 20)) return 1;
    if (n < (1ll << 24)) return 2;
    if (n < (1ll << 28)) return 3;
    return 4;
  }
  if (total < 0 || nmsg <= 0) return 7;
  const int64_t mean = total / nmsg;
  if (mean < 256) return 0;
  if (mean < 1024) return 1;
  if (mean < 4096) return 2;
  if (mean < 16384) return 3;
  if (mean < 65536) return 4;
  if (mean < 262144) return 5;
  return 6;
}

TileConfig single_config(int decode, uint64_t n) {
  std::lock_guard<std::mutex> g(g_mu);
  load_env_once_locked();
  const int kind = decode ? kSingleDecode : kSingleEncode;
  const Entry& e = g_table[kind][bucket_of(kind, (int64_t)n, 1)];
  if (e.set) return TileConfig{e.s.threads, e.s.units_per_thread, e.s.stages, e.s.blocks_per_sm};
  return decode ? default_decode_config(n) : default_encode_config(n);
}

TileConfig ws_lines_config(uint64_t m) {
  std::lock_guard<std::mutex> g(g_mu);
  load_env_once_locked();
  const Entry& e = g_table[kDecodeWs][bucket_of(kDecodeWs, (int64_t)m, 1)];
  if (e.set) return TileConfig{e.s.threads, e.s.units_per_thread, e.s.stages, 0};
  return default_ws_lines_config(m);
}

BatchConfig tuned_batch_config(int decode, int64_t nmsg, int64_t total_bytes) {
  std::lock_guard<std::mutex> g(g_mu);
  load_env_once_locked();
  const int kind = decode ? kBatchDecode : kBatchEncode;
  const Entry& e = g_table[kind][bucket_of(kind, total_bytes, nmsg)];
  if (e.set) return batch_config_of(e.s);
  return default_batch_config(decode, (total_bytes >= 0 && nmsg > 0) ? total_bytes / nmsg : -1);
}

}  // namespace gb64

using namespace gb64;

extern "C" {

int b64_shape_get(int kind, int64_t total, int64_t nmsg, b64_shape* out) {
  clear_error();
  if (kind < 0 || kind >= kKinds || !out) {
    set_error("bad kind or null output");
    return B64_ERR_ARG;
  }
  if (kind == kDecodeWs) {
    const TileConfig c = ws_lines_config((uint64_t)std::max<int64_t>(total, 0));
    *out = b64_shape{c.threads, c.upt, c.stages, 0, (int64_t)c.threads * c.upt * 16, 0.f};
  } else if (kind == kSingleEncode || kind == kSingleDecode) {
    const TileConfig c = single_config(kind == kSingleDecode, (uint64_t)std::max<int64_t>(total, 0));
    const int unit = kind == kSingleDecode ? 16 : 12;
    *out = b64_shape{c.threads, c.upt, c.stages, c.blocks_per_sm,
                     (int64_t)c.threads * c.upt * unit, 0.f};
  } else {
    const BatchConfig c = tuned_batch_config(kind == kBatchDecode, nmsg, total);
    *out = b64_shape{c.threads, c.kernel, c.stages, c.blocks_per_sm, c.tile, 0.f};
  }
  return B64_OK;
}

int b64_shape_set(int kind, int64_t total, int64_t nmsg, const b64_shape* s) {
  clear_error();
  if (kind < 0 || kind >= kKinds || !s) {
    set_error("bad kind or null shape");
    return B64_ERR_ARG;
  }
  if (!shape_valid(kind, *s)) {
    set_error("shape not valid for this kind");
    return B64_ERR_ARG;
  }
  if (kind == kSingleEncode || kind == kSingleDecode || kind == kDecodeWs) {
    // with a device present, the shape must fit its shared memory
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
      cudaError_t e;
      const DeviceInfo* di = device_info(&e);
      const TileConfig c{s->threads, s->units_per_thread, s->stages, s->blocks_per_sm};
      const size_t need = kind == kDecodeWs ? ws_lines_smem_bytes(c)
                                            : single_smem_bytes(kind == kSingleDecode, c);
      if (di && need + 1024 > (size_t)di->max_smem_optin) {
        set_error("shape needs %zu bytes of shared memory per CTA; the device allows %d", need,
                  di->max_smem_optin);
        return B64_ERR_ARG;
      }
    } else {
      cudaGetLastError();
    }
  }
  std::lock_guard<std::mutex> g(g_mu);
  load_env_once_locked();
  Entry& e = g_table[kind][bucket_of(kind, total, nmsg)];
  e.set = true;
  e.s = *s;
  return B64_OK;
}

int b64_tune_save(const char* path) {
  clear_error();
  if (!path) return B64_ERR_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  FILE* f = fopen(path, "w");
  if (!f) {
    set_error("cannot write %s", path);
    return B64_ERR_ARG;
  }
  for (int k = 0; k < kKinds; ++k)
    for (int b = 0; b < kBuckets; ++b)
      if (g_table[k][b].set) {
        const b64_shape& s = g_table[k][b].s;
        fprintf(f, "%d %d %d %d %d %d %lld %.5f\n", k, b, s.threads, s.units_per_thread, s.stages,
                s.blocks_per_sm, (long long)s.tile, s.ms);
      }
  fclose(f);
  return B64_OK;
}

int b64_tune_load(const char* path) {
  clear_error();
  if (!path) return B64_ERR_ARG;
  std::lock_guard<std::mutex> g(g_mu);
  g_loaded = true;
  const int rc = load_file_locked(path);
  if (rc != B64_OK) set_error("cannot read %s", path);
  return rc;
}

int b64_tune(int kind, int64_t total, int64_t nmsg, b64_shape* trials, int max_trials,
             int* ntrials, gb64_stream_t stream_) {
  clear_error();
  if (kind < 0 || kind >= kKinds || total <= 0 ||
      ((kind == kBatchEncode || kind == kBatchDecode) && (nmsg <= 0 || nmsg > total))) {
    set_error("bad kind, size or message count");
    return B64_ERR_ARG;
  }
  if (kind == kDecodeWs) {
    set_error("the line-model kernel's shape is set with b64_shape_set, not tuned");
    return B64_ERR_ARG;
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  cudaError_t e;
  const DeviceInfo* di = device_info(&e);
  if (!di) return cuda_status(e, "tune: device query");
  const bool decode = (kind == kSingleDecode || kind == kBatchDecode);
  const bool batch = (kind == kBatchEncode || kind == kBatchDecode);
  // Test data: `raw` random bytes, `enc` their encoding (the decode input).
  const uint64_t raw_n = decode ? (uint64_t)total / 4 * 3 : (uint64_t)total;
  const uint64_t enc_n = b64_encoded_len(raw_n);
  DeviceBuffers buf;
  uint8_t *raw = nullptr, *enc = nullptr, *dec = nullptr;
  b64_result* res = nullptr;
  e = buf.alloc(&raw, raw_n);
  if (e == cudaSuccess) e = buf.alloc(&enc, enc_n + 64 * (uint64_t)std::max<int64_t>(nmsg, 1));
  if (e == cudaSuccess) e = buf.alloc(&dec, raw_n + 16);
  if (e == cudaSuccess) e = buf.alloc(&res, sizeof(b64_result));
  if (e != cudaSuccess) return cuda_status(e, "tune: buffers");
  k_fill_random<<<di->sm_count * 4, 256, 0, stream>>>(raw, raw_n, 0x5eedull + (uint64_t)kind);
  // batch layout: nmsg messages, lengths spread around the mean (deterministic)
  int64_t *in_off = nullptr, *out_off = nullptr, *enc_off = nullptr, *fb = nullptr, *ol = nullptr;
  int32_t* st = nullptr;
  void* scratch = nullptr;
  if (batch) {
    std::vector<int64_t> off(nmsg + 1, 0);
    const int64_t mean = (int64_t)raw_n / nmsg;
    uint64_t x = 88172645463325252ull;
    for (int64_t j = 0; j < nmsg; ++j) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      const int64_t len = std::max<int64_t>(1, mean / 2 + (int64_t)(x % (uint64_t)(mean + 1)));
      off[j + 1] = std::min<int64_t>((int64_t)raw_n, off[j] + len);
    }
    e = buf.alloc(&in_off, (nmsg + 1) * 8);
    if (e == cudaSuccess) e = buf.alloc(&out_off, (nmsg + 1) * 8);
    if (e == cudaSuccess) e = buf.alloc(&enc_off, (nmsg + 1) * 8);
    if (e == cudaSuccess) e = buf.alloc(&fb, nmsg * 8);
    if (e == cudaSuccess) e = buf.alloc(&ol, nmsg * 8);
    if (e == cudaSuccess) e = buf.alloc(&st, nmsg * 4);
    if (e == cudaSuccess) e = buf.alloc(&scratch, batch_scratch_bytes(nmsg));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(in_off, off.data(), (nmsg + 1) * 8, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e, "tune: batch buffers");
  }
  BatchArgs ba;
  ba.in_off = in_off;
  ba.nmsg = nmsg;
  ba.stream = stream;
  ba.status = st;
  ba.first_bad = fb;
  ba.outlen = ol;
  if (batch) batch_scratch_split(scratch, nmsg, &ba.weight_off, &ba.parts);
  if (decode) {  // decode input = encoding of the random bytes
    if (batch) {
      BatchArgs ea = ba;
      ea.decode = 0;
      ea.src = raw;
      ea.dst = enc;
      ea.out_off = enc_off;
      e = batch_launch(ea, default_batch_config(0, (int64_t)raw_n / nmsg));
    } else {
      e = launch_encode(raw, raw_n, enc, stream, default_encode_config(raw_n));
    }
    if (e != cudaSuccess) return cuda_status(e, "tune: preparing the decode input");
  }
  std::vector<b64_shape> cand =
      batch ? batch_candidates(decode) : single_candidates(decode, di);
  int best = -1;
  int n = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    b64_shape& s = cand[i];
    auto run = [&]() -> cudaError_t {
      if (batch) {
        BatchArgs a = ba;
        a.decode = decode;
        a.src = decode ? enc : raw;
        a.in_off = decode ? enc_off : in_off;
        a.dst = decode ? dec : enc;
        a.out_off = decode ? out_off : enc_off;
        return batch_launch(a, batch_config_of(s));
      }
      const TileConfig c{s.threads, s.units_per_thread, s.stages, s.blocks_per_sm};
      if (!decode) return launch_encode(raw, raw_n, enc, stream, c);
      cudaError_t r = cudaMemsetAsync(res, 0xFF, sizeof(b64_result), stream);
      if (r == cudaSuccess) r = launch_decode(enc, enc_n, decode_body_end(enc_n), dec, res, stream, c);
      return r;
    };
    float ms = 0;
    e = time_median(run, stream, 7, &ms);
    if (e != cudaSuccess) return cuda_status(e, "tune: timing");
    s.ms = ms;
    if (trials && n < max_trials) trials[n] = s;
    ++n;
    if (best < 0 || ms < cand[best].ms) best = (int)i;
  }
  if (ntrials) *ntrials = n;
  if (best >= 0) {
    std::lock_guard<std::mutex> g(g_mu);
    load_env_once_locked();
    Entry& en = g_table[kind][bucket_of(kind, decode && !batch ? (int64_t)enc_n : total, nmsg)];
    en.set = true;
    en.s = cand[best];
  }
  return B64_OK;
}

}  // extern "C"
