// Serving engine: continuous batching of encode and decode requests.
//
// Requests name a device-resident payload (pointer + length) and arrive at
// any time (b64_server_submit, thread-safe). One engine thread
//   - admits requests by device memory: every batch takes one block of a
//     fixed arena (the memory budget) for its descriptors, weight offsets,
//     per-message results and outputs; a batch that does not fit waits until
//     earlier outputs are released (counted as a memory wait);
//   - forms a batch per free stream slot from the pending requests of one
//     kind (the kind whose oldest request is oldest), up to max_batch_msgs
//     requests and max_batch_bytes payload bytes, so requests that arrive
//     while other batches run join the next batch (continuous batching);
//   - builds the batch's message descriptors and weight offsets on the host
//     (from the request lengths; no device scan, no copy of the payloads),
//     then, with the lock released, issues one host-to-device copy, the
//     persistent batched codec kernel that reads each payload where it lives
//     (plus the per-message finish kernel and one device-to-host copy of the
//     results for decode) and an event; batches on different slots overlap
//     on the device;
//   - polls the events and turns finished batches into completions
//     (status, first_bad, outlen, a device pointer to the output, and the
//     arrival/admission/completion times).
// Outputs stay in the arena until the request is released.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"
#include "internal.h"
#include "tuner.h"

namespace gb64 {
namespace {

using Clock = std::chrono::steady_clock;

struct Arena {
  uint8_t* base = nullptr;
  uint64_t size = 0, used = 0, high_water = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> bytes

  static uint64_t round(uint64_t n) { return (n + 255) & ~255ull; }
  void init(uint8_t* b, uint64_t n) {
    base = b;
    size = n;
    free_.clear();
    free_[0] = n;
  }
  bool alloc(uint64_t n, uint64_t* off) {
    n = round(n);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const uint64_t o = it->first, rest = it->second - n;
      free_.erase(it);
      if (rest) free_[o + n] = rest;
      *off = o;
      used += n;
      high_water = std::max(high_water, used);
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    n = round(n);
    used -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Request {
  int kind = 0;
  const uint8_t* src = nullptr;
  int64_t len = 0;
  double t_arrival = 0, t_admit = 0;
  int64_t batch = -1;
  bool done = false, released = false;
};

// Block layout of one batch (offsets from the block start). The first
// h2d_bytes are copied from the host; the d2h region holds decode results.
struct Layout {
  uint64_t desc, weight_off, first_bad, outlen, status, out, total;
  uint64_t h2d_bytes, d2h_off, d2h_bytes;
};

Layout layout_for(int64_t n, int64_t out_bytes, int kind) {
  auto up = [](uint64_t x) { return (x + 255) & ~255ull; };
  Layout L;
  L.desc = 0;
  L.weight_off = L.desc + (uint64_t)n * sizeof(MsgDesc);
  L.first_bad = L.weight_off + (uint64_t)(n + 1) * 8;
  L.outlen = L.first_bad + (uint64_t)n * 8;
  L.status = L.outlen + (uint64_t)n * 8;
  L.out = up(L.status + (uint64_t)n * 4);
  L.total = L.out + (uint64_t)out_bytes + 16;
  L.h2d_bytes = kind ? L.status : L.first_bad;
  L.d2h_off = L.first_bad;
  L.d2h_bytes = L.out - L.first_bad;
  return L;
}

struct Member {
  int64_t id;
  const uint8_t* src;
  int64_t len;
  int64_t out_off;
};

struct Batch {
  int kind = 0;
  std::vector<Member> members;
  uint64_t block = 0, block_bytes = 0;
  Layout L{};
  BatchConfig cfg{};
  int slot = -1;
  int unreleased = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t* host = nullptr;  // pinned: staging of the h2d region, then the results
  uint64_t host_bytes = 0;
  int64_t batch = -1;
};

}  // namespace
}  // namespace gb64

struct b64_server {
  gb64::Arena arena;
  b64_server_config cfg{};
  int device = 0;
  std::vector<gb64::Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<gb64::Request> reqs;  // index = request id (stable references)
  std::deque<int64_t> pending[2];
  std::map<int64_t, gb64::Batch> batches;
  int64_t next_batch = 0;
  std::deque<b64_completion> done_q;
  b64_server_stats stats{};
  std::atomic<bool> stop{false};
  std::thread engine;
  gb64::Clock::time_point t0;
  int error = 0;

  double now_us() const {
    return std::chrono::duration<double, std::micro>(gb64::Clock::now() - t0).count();
  }
};

namespace gb64 {
namespace {

int64_t out_capacity(int kind, int64_t len) {
  return kind ? (int64_t)b64_decoded_cap((size_t)len) : (int64_t)b64_encoded_len((size_t)len);
}

void release_block_locked(b64_server* S, int64_t bid) {
  auto it = S->batches.find(bid);
  if (it == S->batches.end()) return;
  S->arena.release(it->second.block, it->second.block_bytes);
  S->batches.erase(it);
}

// Forms a batch for a free slot (lock held): pops its requests, allocates
// its block, copies what the launch needs. Returns the batch id or -1.
int64_t form_batch(b64_server* S) {
  int slot = -1;
  for (size_t i = 0; i < S->slots.size(); ++i)
    if (S->slots[i].batch < 0) {
      slot = (int)i;
      break;
    }
  if (slot < 0) return -1;
  int kind = -1;
  double oldest = 1e300;
  for (int k = 0; k < 2; ++k)
    if (!S->pending[k].empty() && S->reqs[S->pending[k].front()].t_arrival < oldest) {
      oldest = S->reqs[S->pending[k].front()].t_arrival;
      kind = k;
    }
  if (kind < 0) return -1;
  std::deque<int64_t>& q = S->pending[kind];
  int64_t n = 0, in_bytes = 0;
  while (n < (int64_t)q.size() && n < S->cfg.max_batch_msgs) {
    const int64_t len = S->reqs[q[n]].len;
    if (n > 0 && in_bytes + len > S->cfg.max_batch_bytes) break;
    in_bytes += len;
    ++n;
  }
  // admission by memory: shrink the batch until its block fits the arena
  uint64_t off = 0;
  Layout L{};
  while (n > 0) {
    int64_t out_bytes = 0;
    for (int64_t j = 0; j < n; ++j) out_bytes += out_capacity(kind, S->reqs[q[j]].len);
    L = layout_for(n, out_bytes, kind);
    if (S->arena.alloc(L.total, &off)) break;
    n = (n > 1) ? n / 2 : 0;
  }
  if (n == 0) {
    S->stats.memory_waits++;
    return -1;
  }
  const int64_t bid = S->next_batch++;
  Batch& B = S->batches[bid];
  B.kind = kind;
  B.block = off;
  B.block_bytes = L.total;
  B.L = L;
  B.slot = slot;
  B.unreleased = (int)n;
  const double t = S->now_us();
  int64_t out_off = 0;
  in_bytes = 0;
  B.members.reserve(n);
  for (int64_t j = 0; j < n; ++j) {
    const int64_t id = q.front();
    q.pop_front();
    Request& r = S->reqs[id];
    r.batch = bid;
    r.t_admit = t;
    B.members.push_back(Member{id, r.src, r.len, out_off});
    out_off += out_capacity(kind, r.len);
    in_bytes += r.len;
  }
  B.cfg = tuned_batch_config(kind, n, in_bytes);
  S->slots[slot].batch = bid;
  S->stats.batches++;
  S->stats.requests_launched += n;
  S->stats.bytes_in += in_bytes;
  S->stats.arena_high_water = (int64_t)S->arena.high_water;
  return bid;
}

// Stages and launches a formed batch (no lock needed: the batch and its
// slot are owned by the engine thread until it is reaped).
cudaError_t launch_batch(const Batch& B, Slot& sl, uint8_t* arena_base) {
  const int64_t n = (int64_t)B.members.size();
  uint8_t* blk = arena_base + B.block;
  MsgDesc* h_desc = reinterpret_cast<MsgDesc*>(sl.host + B.L.desc);
  int64_t* h_weight = reinterpret_cast<int64_t*>(sl.host + B.L.weight_off);
  h_weight[0] = 0;
  for (int64_t j = 0; j < n; ++j) {
    const Member& m = B.members[j];
    h_desc[j] = MsgDesc{m.src, m.len, m.out_off};
    const int64_t tiles = m.len > 0 ? (m.len + B.cfg.tile - 1) / B.cfg.tile : 0;
    h_weight[j + 1] = h_weight[j] + (tiles ? m.len + tiles * kBatchTileCost : 0);
  }
  if (B.kind) {
    int64_t* h_fb = reinterpret_cast<int64_t*>(sl.host + B.L.first_bad);
    int64_t* h_ol = reinterpret_cast<int64_t*>(sl.host + B.L.outlen);
    for (int64_t j = 0; j < n; ++j) {
      h_fb[j] = INT64_MAX;  // "no bad character yet"
      h_ol[j] = 0;
    }
  }
  cudaError_t e = cudaMemcpyAsync(blk, sl.host, B.L.h2d_bytes, cudaMemcpyHostToDevice, sl.stream);
  if (e != cudaSuccess) return e;
  e = batch_launch_desc(B.kind, reinterpret_cast<const MsgDesc*>(blk + B.L.desc), n,
                        blk + B.L.out, reinterpret_cast<const int64_t*>(blk + B.L.weight_off),
                        reinterpret_cast<int32_t*>(blk + B.L.status),
                        reinterpret_cast<int64_t*>(blk + B.L.first_bad),
                        reinterpret_cast<int64_t*>(blk + B.L.outlen), B.cfg, false, sl.stream);
  if (e != cudaSuccess) return e;
  if (B.kind) {
    e = cudaMemcpyAsync(sl.host + B.L.d2h_off, blk + B.L.d2h_off, B.L.d2h_bytes,
                        cudaMemcpyDeviceToHost, sl.stream);
    if (e != cudaSuccess) return e;
  }
  return cudaEventRecord(sl.done, sl.stream);
}

// Moves finished batches to completions (lock held). Returns how many.
int reap(b64_server* S) {
  int nb = 0;
  for (Slot& sl : S->slots) {
    if (sl.batch < 0) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) S->error = cuda_status(q, "server: batch");
    Batch& B = S->batches[sl.batch];
    const double t = S->now_us();
    const int64_t n = (int64_t)B.members.size();
    const int32_t* st = reinterpret_cast<const int32_t*>(sl.host + B.L.status);
    const int64_t* fb = reinterpret_cast<const int64_t*>(sl.host + B.L.first_bad);
    const int64_t* ol = reinterpret_cast<const int64_t*>(sl.host + B.L.outlen);
    uint8_t* out = S->arena.base + B.block + B.L.out;
    for (int64_t j = 0; j < n; ++j) {
      const Member& m = B.members[j];
      Request& r = S->reqs[m.id];
      r.done = true;
      b64_completion c{};
      c.id = m.id;
      c.kind = B.kind;
      if (q != cudaSuccess) {
        c.status = B64_ERR_CUDA;
      } else if (B.kind) {
        c.status = st[j];
        c.first_bad = fb[j];
        c.outlen = ol[j];
      } else {
        c.status = B64_OK;
        c.first_bad = -1;
        c.outlen = out_capacity(0, m.len);
      }
      c.out = out + m.out_off;
      c.len = m.len;
      c.batch = sl.batch;
      c.t_arrival_us = r.t_arrival;
      c.t_admit_us = r.t_admit;
      c.t_done_us = t;
      S->done_q.push_back(c);
    }
    sl.batch = -1;
    S->stats.requests_done += n;
    ++nb;
  }
  return nb;
}

void engine_main(b64_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    const int reaped = reap(S);
    if (reaped) S->cv.notify_all();
    const int64_t bid = form_batch(S);
    if (bid >= 0) {
      Batch& B = S->batches[bid];  // std::map: stable while the lock is dropped
      Slot& sl = S->slots[B.slot];
      uint8_t* base = S->arena.base;
      lk.unlock();
      const cudaError_t e = launch_batch(B, sl, base);
      lk.lock();
      if (e != cudaSuccess) S->error = cuda_status(e, "server: batch launch");
      continue;
    }
    bool busy = false;
    for (const Slot& sl : S->slots) busy |= sl.batch >= 0;
    if (!busy && S->pending[0].empty() && S->pending[1].empty()) {
      S->cv.wait_for(lk, std::chrono::milliseconds(5));
    } else if (!reaped) {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
  }
}

}  // namespace
}  // namespace gb64

using namespace gb64;

extern "C" {

b64_server* b64_server_create(const b64_server_config* cfg_in) {
  clear_error();
  if (!cfg_in) {
    set_error("config is null");
    return nullptr;
  }
  b64_server_config cfg = *cfg_in;
  if (cfg.memory_budget < (1 << 20) || cfg.streams < 1 || cfg.streams > 16 ||
      cfg.max_batch_msgs < 1 || cfg.max_batch_msgs > 65536 || cfg.max_batch_bytes < 1) {
    set_error("config out of range (budget >= 1 MiB, 1..16 streams, 1..65536 msgs per batch)");
    return nullptr;
  }
  std::unique_ptr<b64_server> S(new b64_server());
  S->cfg = cfg;
  cudaError_t e = cudaGetDevice(&S->device);
  uint8_t* mem = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&mem, (size_t)cfg.memory_budget);
  if (e != cudaSuccess) {
    cuda_status(e, "server: arena");
    return nullptr;
  }
  S->arena.init(mem, (uint64_t)cfg.memory_budget);
  S->stats.arena_bytes = cfg.memory_budget;
  const uint64_t host_bytes = layout_for(cfg.max_batch_msgs, 0, 1).out;
  S->slots.resize(cfg.streams);
  for (Slot& sl : S->slots) {
    e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&sl.host, host_bytes);
    if (e != cudaSuccess) {
      cuda_status(e, "server: streams");
      return nullptr;
    }
    sl.host_bytes = host_bytes;
  }
  S->t0 = Clock::now();
  b64_server* raw = S.release();
  raw->engine = std::thread(engine_main, raw);
  return raw;
}

double b64_server_now_us(b64_server* S) { return S ? S->now_us() : 0.0; }

int b64_server_submit(b64_server* S, int kind, const uint8_t* src, int64_t len,
                      double t_arrival_us, int64_t* id) {
  clear_error();
  if (!S || (kind != 0 && kind != 1) || len < 0 || (len > 0 && !src)) {
    set_error("bad server, kind, length or source");
    return B64_ERR_ARG;
  }
  const Layout L = layout_for(1, out_capacity(kind, len), kind);
  std::lock_guard<std::mutex> g(S->mu);
  if (S->error) return S->error;
  if (L.total > S->arena.size) {
    S->stats.rejected++;
    set_error("request of %lld bytes does not fit the memory budget", (long long)len);
    return B64_ERR_NOMEM;
  }
  const int64_t rid = (int64_t)S->reqs.size();
  Request r;
  r.kind = kind;
  r.src = src;
  r.len = len;
  r.t_arrival = t_arrival_us >= 0 ? t_arrival_us : S->now_us();
  S->reqs.push_back(r);
  S->pending[kind].push_back(rid);
  S->stats.requests_submitted++;
  if (id) *id = rid;
  S->cv.notify_all();
  return B64_OK;
}

static void release_locked(b64_server* S, int64_t id) {
  Request& r = S->reqs[id];
  if (r.released || !r.done) return;
  r.released = true;
  auto it = S->batches.find(r.batch);
  if (it == S->batches.end()) return;
  if (--it->second.unreleased == 0) release_block_locked(S, r.batch);
}

int b64_server_poll(b64_server* S, b64_completion* out, int max, int timeout_us) {
  clear_error();
  if (!S || (!out && max > 0)) return B64_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done_q.empty() && timeout_us > 0)
    S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !S->done_q.empty(); });
  int k = 0;
  while (k < max && !S->done_q.empty()) {
    out[k] = S->done_q.front();
    S->done_q.pop_front();
    if (S->cfg.auto_release) release_locked(S, out[k].id);
    ++k;
  }
  if (S->error && k == 0) return S->error;
  return k;
}

int b64_server_release(b64_server* S, int64_t id) {
  clear_error();
  if (!S) return B64_ERR_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  if (id < 0 || id >= (int64_t)S->reqs.size() || !S->reqs[id].done) {
    set_error("unknown or unfinished request");
    return B64_ERR_ARG;
  }
  release_locked(S, id);
  return B64_OK;
}

int b64_server_stats_get(b64_server* S, b64_server_stats* out) {
  if (!S || !out) return B64_ERR_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->stats;
  out->arena_in_use = (int64_t)S->arena.used;
  return B64_OK;
}

int b64_server_replay(b64_server* S, int64_t n, const double* t_arrival_us, const int32_t* kind,
                      const uint64_t* src, const int64_t* len, double* latency_us,
                      int32_t* status) {
  clear_error();
  if (!S || n < 0 || (n > 0 && (!t_arrival_us || !kind || !src || !len || !latency_us))) {
    set_error("bad replay arguments");
    return B64_ERR_ARG;
  }
  if (!S->cfg.auto_release) {
    set_error("replay needs a server created with auto_release");
    return B64_ERR_ARG;
  }
  int64_t first = -1;
  {
    std::lock_guard<std::mutex> g(S->mu);
    first = (int64_t)S->reqs.size();
  }
  const double base = S->now_us();
  std::atomic<int> submit_rc{B64_OK};
  std::atomic<int64_t> accepted{0};
  std::atomic<bool> submitted_all{false};
  std::thread submitter([&] {
    for (int64_t i = 0; i < n; ++i) {
      const double target = base + t_arrival_us[i];
      for (;;) {
        const double dt = target - S->now_us();
        if (dt <= 0) break;
        if (dt > 300) std::this_thread::sleep_for(std::chrono::microseconds((int64_t)(dt - 200)));
      }
      int64_t id;
      const int rc = b64_server_submit(S, kind[i], reinterpret_cast<const uint8_t*>(src[i]),
                                       len[i], target, &id);
      if (rc == B64_OK) {
        accepted++;
      } else {  // rejected (too large for the budget): never completes
        submit_rc = rc;
        latency_us[i] = -1;
        if (status) status[i] = rc;
      }
    }
    submitted_all = true;
  });
  std::vector<b64_completion> buf(4096);
  int64_t got = 0;
  int rc = B64_OK;
  while (!(submitted_all && got >= accepted)) {
    const int k = b64_server_poll(S, buf.data(), (int)buf.size(), 2000);
    if (k < 0) {
      rc = k;
      break;
    }
    for (int j = 0; j < k; ++j) {
      const int64_t i = buf[j].id - first;
      if (i < 0 || i >= n) continue;
      latency_us[i] = buf[j].t_done_us - buf[j].t_arrival_us;
      if (status) status[i] = buf[j].status;
      ++got;
    }
  }
  submitter.join();
  return rc != B64_OK ? rc : (int)submit_rc;
}

void b64_server_destroy(b64_server* S) {
  if (!S) return;
  S->stop = true;
  S->cv.notify_all();
  if (S->engine.joinable()) S->engine.join();
  for (Slot& sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.host) cudaFreeHost(sl.host);
  }
  cudaFree(S->arena.base);
  delete S;
}

}  // extern "C"
