/*
 * gb64 - base64 codec for NVIDIA GB300 (sm_103a): the C ABI.
 *
 * The operations follow Muła & Lemire, "Faster Base64 Encoding and Decoding
 * using AVX2 Instructions" (arXiv 1704.00605):
 *   encode  Algorithm 1 (Section 2): every 3 input bytes become four 6-bit
 *           values, each mapped to a character of Table 1; a final group of
 *           1 or 2 bytes gets "==" or "=" padding.
 *   decode  Algorithm 2 (Section 2): every 4 characters become 3 bytes; a
 *           character outside Table 1 is reported as an error (Section 2,
 *           "report an error when characters outside of this set are
 *           encountered"; Appendix B quotes RFC 4648 on the same rule).
 *
 * Conventions shared by every call:
 *   - Pointers named src/dst/in_off/out_off/status/first_bad/outlen/d_result
 *     are DEVICE pointers owned by the caller (any cudaMalloc/torch memory
 *     of the current device), unless the name starts with h_ (host memory).
 *   - stream is a cudaStream_t (NULL = the legacy default stream). Calls that
 *     do not say "synchronous" only enqueue work on it.
 *   - src and dst must not overlap. No output is NUL-terminated.
 *   - Argument errors are found on the host before anything is enqueued and
 *     return B64_ERR_ARG; CUDA runtime failures return B64_ERR_CUDA. The text
 *     of the last error of the calling thread is b64_last_error().
 *   - Decode status: B64_OK, B64_ERR_INVALID_CHAR (first_bad = index of the
 *     first character that is outside Table 1 and not an accepted padding
 *     '='), or B64_ERR_BAD_LENGTH (no invalid character, length not a
 *     multiple of 4; first_bad = m - m % 4). '=' is accepted only as the last
 *     character, or the last two, of an input whose length is a multiple of
 *     4. On B64_OK first_bad = m; on an error outlen = 0 and the contents of
 *     dst are unspecified. Non-zero trailing bits in the final group are
 *     accepted and dropped (Appendix A's extra check is not applied).
 */
#ifndef GB64_H
#define GB64_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream handle (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *gb64_stream_t;

typedef enum {
  B64_OK = 0,
  B64_ERR_INVALID_CHAR = 1,
  B64_ERR_BAD_LENGTH = 2,
  B64_ERR_NONCANONICAL = 3, /* B64_FLAG_STRICT_TAIL: non-zero trailing bits */
  B64_ERR_ARG = -1,
  B64_ERR_CUDA = -2,
  B64_ERR_NOMEM = -3,
  B64_ERR_TIMEOUT = -4
} b64_status;

/* Device-side result of one decode (written by b64_decode_async). */
typedef struct {
  int64_t first_bad; /* as for b64_decode */
  int64_t outlen;    /* bytes written on B64_OK, else 0 */
  int32_t status;    /* a b64_status */
  uint32_t internal; /* used by the library while the decode runs; afterwards
                        it names the kernel path that finished the decode
                        (an implementation detail, for tests) */
} b64_result;

/* Length of the encoding of n bytes: 4 * ceil(n / 3) (Section 2: three
 * bytes per four characters, padded). Returns SIZE_MAX if it overflows. */
size_t b64_encoded_len(size_t n);

/* Bytes a decode of m characters may write: 3 * (m / 4). */
size_t b64_decoded_cap(size_t m);

/* Encode n bytes at src into b64_encoded_len(n) characters at dst
 * (Algorithm 1). Asynchronous on stream. Returns the output length, or
 * SIZE_MAX on an argument or CUDA error (see b64_last_error()). n = 0 is
 * legal and returns 0 without enqueuing work. Any alignment of src and dst
 * is accepted; 16-byte aligned pointers take the TMA-pipelined kernel. */
size_t b64_encode(const uint8_t *src, size_t n, char *dst, gb64_stream_t stream);

/* Decode m characters at src into dst (capacity b64_decoded_cap(m) bytes)
 * (Algorithm 2, strict). SYNCHRONOUS: waits for stream, then stores the
 * decoded length in *outlen and the first bad index in *first_bad (host
 * pointers) and returns a b64_status. */
int b64_decode(const char *src, size_t m, uint8_t *dst, size_t *outlen, size_t *first_bad,
               gb64_stream_t stream);

/* Asynchronous decode: as b64_decode, but the result goes to the device
 * struct *d_result (caller-owned device memory, 8-byte aligned) and nothing
 * waits. Returns B64_OK when the work was enqueued, else an error code. */
int b64_decode_async(const char *src, size_t m, uint8_t *dst, b64_result *d_result,
                     gb64_stream_t stream);

/* Host-buffer forms: h_src and h_dst are HOST pointers (pinned memory gives
 * the full link bandwidth; pageable memory works but is slower). The input
 * is copied to the device in chunks, coded by the same kernels, and copied
 * back, with copies and kernels of different chunks overlapped on internal
 * streams ordered after `stream`. SYNCHRONOUS. The library keeps device and
 * pinned staging buffers per calling thread (allocated at first use). */
size_t b64_encode_host(const uint8_t *h_src, size_t n, char *h_dst, gb64_stream_t stream);
int b64_decode_host(const char *h_src, size_t m, uint8_t *h_dst, size_t *outlen,
                    size_t *first_bad, gb64_stream_t stream);

/* Batched forms: nmsg messages packed back to back in src, message j at
 * [in_off[j], in_off[j+1]) with in_off[0] = 0 (int64, device, nmsg + 1
 * entries, non-decreasing). The library writes out_off[0..nmsg] (device):
 * the exclusive prefix of b64_encoded_len (encode) or b64_decoded_cap
 * (decode) of the messages, and message j's output starts at dst +
 * out_off[j]. One persistent kernel codes every message: messages of up to
 * 256 bytes / 344 characters one thread each, longer ones cut into
 * fixed-size tiles that the warps share by bytes (a device prefix sum over
 * the messages' weights), and per-message padding and error positions are
 * handled inside the kernel (Section 2's rules per message). Asynchronous; per-message decode results go to
 * status[j], first_bad[j] (relative to the message start) and outlen[j].
 * dst must hold out_off[nmsg] bytes: call b64_batch_out_offsets first when
 * that total is not known. Temporary device memory is taken from the
 * stream-ordered allocator on `stream` and returned on it. */
int b64_batch_out_offsets(int decode, const int64_t *in_off, int64_t nmsg, int64_t *out_off,
                          gb64_stream_t stream);
int b64_encode_batch(const uint8_t *src, const int64_t *in_off, int64_t nmsg, char *dst,
                     int64_t *out_off, gb64_stream_t stream);
int b64_decode_batch(const char *src, const int64_t *in_off, int64_t nmsg, uint8_t *dst,
                     int64_t *out_off, int32_t *status, int64_t *first_bad, int64_t *outlen,
                     gb64_stream_t stream);

/* Batched decode that allocates nothing. The paper has no counterpart: this
 * is an interface for callers that must not allocate device memory inside
 * the call (a fixed memory budget or an allocator owned by someone else, or
 * a hot path that cannot afford cudaMalloc/cudaFree synchronizing the
 * device). Same arguments, kernels and results as b64_decode_batch, but the
 * scratch lives in a fixed array inside the library (about 576 KiB per GPU
 * that uses it, held until the process exits) instead of coming from the
 * stream-ordered allocator. At most 65536 messages per call; a larger nmsg
 * returns B64_ERR_ARG with nothing enqueued. Every call on a device shares
 * that array, so two calls that overlap on the GPU race: order them on one
 * stream or with events. The first call on a device looks up the array's
 * device address; make it before any stream capture. That address is kept
 * until the process exits: resetting the device (cudaDeviceReset) between
 * calls is not supported. Asynchronous. */
int b64_decode_batch_noalloc(const char *src, const int64_t *in_off, int64_t nmsg, uint8_t *dst,
                             int64_t *out_off, int32_t *status, int64_t *first_bad,
                             int64_t *outlen, gb64_stream_t stream);

/* ---- launch shapes and the autotuner (no counterpart in the paper) ----
 * Kernel families: */
enum {
  B64_KIND_ENCODE = 0,       /* b64_encode and the host-buffer encode */
  B64_KIND_DECODE = 1,       /* b64_decode(_async) and the host-buffer decode */
  B64_KIND_ENCODE_BATCH = 2, /* b64_encode_batch */
  B64_KIND_DECODE_BATCH = 3, /* b64_decode_batch(_noalloc) */
  B64_KIND_DECODE_WS = 4     /* the one-pass line-model kernel of B64_FLAG_SKIP_WS */
};

/* A launch shape. Single kinds use threads, units_per_thread (12 input
 * bytes or 16 characters each; tile = threads * units_per_thread * unit),
 * stages (TMA stages in shared memory) and blocks_per_sm (0 = as many as
 * fit). Batch kinds use units_per_thread as the kernel choice: 0 = messages
 * of up to 256 bytes (encode) or 344 characters (decode) one thread each
 * and per-warp tiles staged in shared memory for the longer ones, 1 =
 * staged tiles for every message, 2 = short messages one thread each and
 * unstaged tiles (read and written straight from and to global memory) for
 * the rest, 3 (the default for decode) = a batch whose encoded lengths are
 * all multiples of 4 (padded output; any padded encoding, decoding), of at
 * least 1 Ki characters on average and with src and dst 16-byte aligned,
 * coded as one buffer by a kernel of its own (messages then start on quads
 * of the encoded side, and decoding, every output at 3/4 of its input
 * offset), any other batch as 2. Then threads, tile (input bytes per warp tile, a multiple of
 * 384, or characters, a multiple of 512: up to 16 such rows staged, 64
 * unstaged), stages (staged input stages per warp, 2..6; 0 = 4) and
 * blocks_per_sm (0 = as many as fit); a staged shape's shared memory,
 * threads / 32 * (stages * (tile + 32) + (decode only) 3 * tile / 4 + 32)
 * bytes, must stay within 219 KiB. B64_KIND_DECODE_WS uses threads (256
 * or 512), units_per_thread (16 kept characters each; a tile of up to 64 Ki
 * characters) and stages (2..6). ms is a measured time. */
typedef struct {
  int32_t threads;
  int32_t units_per_thread;
  int32_t stages;
  int32_t blocks_per_sm;
  int64_t tile;
  float ms;
} b64_shape;

/* Shapes are kept per size bucket: single kinds by input size (total =
 * bytes or characters; nmsg ignored), batch kinds by mean message length
 * (total / nmsg; total < 0 = unknown). b64_shape_get returns the shape a
 * call of that size uses; b64_shape_set replaces it (B64_ERR_ARG if the
 * shape is not valid for the kind). */
int b64_shape_get(int kind, int64_t total, int64_t nmsg, b64_shape *out);
int b64_shape_set(int kind, int64_t total, int64_t nmsg, const b64_shape *shape);

/* Autotune one bucket (the kinds 0-3): generate `total` bytes (or characters) of random
 * test data on the device (as nmsg messages for batch kinds), time every
 * candidate shape of the kind with CUDA events (median of 7 runs), and keep
 * the fastest for that bucket. Up to max_trials timed shapes are written to
 * trials (host array, may be null) and their count to *ntrials. Allocates
 * its test buffers; synchronous on stream. */
int b64_tune(int kind, int64_t total, int64_t nmsg, b64_shape *trials, int max_trials,
             int *ntrials, gb64_stream_t stream);

/* Write / read the shape table (text). The file named by the environment
 * variable GB64_TUNE_FILE, if set, is read at first use. */
int b64_tune_save(const char *path);
int b64_tune_load(const char *path);

/* ---- serving engine (no counterpart in the paper) ----------------------
 * Continuous batching of encode/decode requests whose payloads are resident
 * in device memory. An engine thread admits requests by device memory (all
 * of a batch's buffers come from one arena of memory_budget bytes allocated
 * at creation; a batch that does not fit waits for earlier outputs to be
 * released), forms a batch per free stream slot from the requests that have
 * arrived, describes their payloads in place (one host-built descriptor per
 * request: address, length, output offset; no gather and no copy of the
 * payloads), runs the batched codec kernels on them, and reports
 * completions. Requests that arrive while batches run
 * join the next batch; batches on different slots overlap on the GPU. */
typedef struct b64_server b64_server;

typedef struct {
  int64_t memory_budget;   /* bytes of device memory the server may hold */
  int32_t streams;         /* batches in flight at once, 1..16 */
  int32_t max_batch_msgs;  /* requests per batch, 1..65536 */
  int64_t max_batch_bytes; /* payload bytes per batch (a larger request runs alone) */
  int32_t auto_release;    /* 1: outputs are freed when polled (out is then invalid) */
  int32_t reserved;
} b64_server_config;

typedef struct {
  int64_t id;           /* from b64_server_submit */
  int32_t kind;         /* 0 encode, 1 decode */
  int32_t status;       /* b64_status of the request */
  int64_t first_bad;    /* decode: as b64_decode; encode: -1 */
  int64_t outlen;       /* bytes (decode) or characters (encode) produced */
  const uint8_t *out;   /* device pointer to the output, valid until released */
  int64_t len;          /* payload length */
  int64_t batch;        /* batch sequence number */
  double t_arrival_us;  /* server clock: arrival, admission, completion seen */
  double t_admit_us;
  double t_done_us;
} b64_completion;

typedef struct {
  int64_t requests_submitted, requests_launched, requests_done, rejected;
  int64_t batches, memory_waits;
  int64_t arena_bytes, arena_in_use, arena_high_water, bytes_in;
} b64_server_stats;

/* Creates a server on the current device (allocates its arena and pinned
 * staging, starts the engine thread). NULL on error (b64_last_error()). */
b64_server *b64_server_create(const b64_server_config *cfg);
/* Microseconds since the server was created (the clock of all timestamps). */
double b64_server_now_us(b64_server *server);
/* Queues one request: kind 0 encode / 1 decode of len bytes at src (device
 * memory that must stay valid until the request completes). t_arrival_us < 0
 * means now. Thread-safe. B64_ERR_NOMEM if one request alone exceeds the
 * memory budget. */
int b64_server_submit(b64_server *server, int kind, const uint8_t *src, int64_t len,
                      double t_arrival_us, int64_t *id);
/* Up to max completions (waiting up to timeout_us for the first); returns
 * how many, or a negative b64_status. */
int b64_server_poll(b64_server *server, b64_completion *out, int max, int timeout_us);
/* Frees a completed request's output (its batch's memory is returned to
 * the arena when every request of the batch is released). */
int b64_server_release(b64_server *server, int64_t id);
int b64_server_stats_get(b64_server *server, b64_server_stats *out);
/* Open-loop replay from native threads: request i is submitted at
 * t_arrival_us[i] after the call starts (kind[i], src[i] as a device address,
 * len[i]); returns when all have completed, with latency_us[i] = completion
 * minus scheduled arrival and status[i] (may be null). Needs auto_release. */
int b64_server_replay(b64_server *server, int64_t n, const double *t_arrival_us,
                      const int32_t *kind, const uint64_t *src, const int64_t *len,
                      double *latency_us, int32_t *status);
/* Stops the engine, waits for work in flight, frees everything. */
void b64_server_destroy(b64_server *server);

/* ---- variants (Section 2: base64url, omitted padding; Appendix A) ----
 * Flags for the _ex calls (0 = the calls above):
 *   B64_FLAG_URL          base64url alphabet: values 62 and 63 are '-' and '_'
 *                         (then '+' and '/' are invalid characters).
 *   B64_FLAG_NOPAD        encode writes no '=' (output b64_encoded_len_ex);
 *                         decode also accepts a final group of 2 or 3
 *                         characters (1 or 2 bytes); padded input is still
 *                         accepted; a final group of 1 character is
 *                         B64_ERR_BAD_LENGTH at m - 1.
 *   B64_FLAG_STRICT_TAIL  decode applies Appendix A's check of the final
 *                         group: the bits dropped by the last data character
 *                         must be zero, else B64_ERR_NONCANONICAL with
 *                         first_bad = that character (invalid characters and
 *                         the length rule are reported first). Ignored by
 *                         encode, whose output always has zero bits. */
#define B64_FLAG_URL 1
#define B64_FLAG_NOPAD 2
#define B64_FLAG_STRICT_TAIL 4
/*   B64_FLAG_SKIP_WS      decode only, single buffer: space, line feed and
 *                         carriage return are removed before decoding
 *                         (Appendix B); first_bad is an index into the
 *                         original input, outlen counts decoded bytes. Uses
 *                         a scratch buffer of about m bytes that the library
 *                         keeps per device between calls (grown as needed,
 *                         freed by b64_release_scratch); calls on different
 *                         streams that use it run one after the other. While
 *                         the stream captures a graph the scratch comes from
 *                         the stream-ordered allocator instead. Not accepted
 *                         by encode or batches. */
#define B64_FLAG_SKIP_WS 8

size_t b64_encoded_len_ex(size_t n, int flags);
size_t b64_decoded_cap_ex(size_t m, int flags);
size_t b64_encode_ex(const uint8_t *src, size_t n, char *dst, int flags, gb64_stream_t stream);
int b64_decode_ex(const char *src, size_t m, uint8_t *dst, size_t *outlen, size_t *first_bad,
                  int flags, gb64_stream_t stream);
int b64_decode_async_ex(const char *src, size_t m, uint8_t *dst, b64_result *d_result, int flags,
                        gb64_stream_t stream);
int b64_batch_out_offsets_ex(int decode, const int64_t *in_off, int64_t nmsg, int64_t *out_off,
                             int flags, gb64_stream_t stream);
int b64_encode_batch_ex(const uint8_t *src, const int64_t *in_off, int64_t nmsg, char *dst,
                        int64_t *out_off, int flags, gb64_stream_t stream);
int b64_decode_batch_ex(const char *src, const int64_t *in_off, int64_t nmsg, uint8_t *dst,
                        int64_t *out_off, int32_t *status, int64_t *first_bad, int64_t *outlen,
                        int flags, gb64_stream_t stream);

/* Human-readable name of a b64_status value (static string). */
const char *b64_status_str(int status);

/* Text of the last error recorded by a call on the calling thread ("" if
 * none). The pointer stays valid until the thread's next gb64 call. */
const char *b64_last_error(void);

/* Reads and clears the device-side fault word of the current device: non-zero
 * when a pipelined kernel gave up on a bounded wait for its own copies
 * (B64_ERR_TIMEOUT) since the last query. Synchronizes the device. Returns 0,
 * B64_ERR_TIMEOUT or B64_ERR_CUDA. */
int b64_device_fault(void);

/* Frees the scratch buffer that the B64_FLAG_SKIP_WS decode keeps on the
 * current device, after the last call that uses it has finished (waits for
 * it); the next such call allocates it again. Returns B64_OK or
 * B64_ERR_CUDA. */
int b64_release_scratch(void);

/* Test hook of the bounded waits (no counterpart in the paper). While
 * stall != 0, every pipelined kernel launched afterwards (the TMA
 * single-buffer encode and decode, the whitespace decode's line kernel, and
 * the batched kernel that stages tiles in shared memory) leaves out the
 * first input copy of its first CTA (of the first warp, batched), so that
 * the wait on it runs out after wait_limit_ns
 * (0 = the default of 2 s): the kernel records the fault word, waits
 * (bounded) for its other copies in flight and returns, the call reports
 * B64_ERR_TIMEOUT (decode results; b64_device_fault()), and no GPU fault,
 * trap or hang is involved. stall = 0 restores normal operation, and
 * wait_limit_ns then sets the limit of every bounded wait (0 = 2 s).
 * Process-wide; for tests, not for concurrent use. Returns B64_OK. */
int b64_test_stall_copies(int stall, uint64_t wait_limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* GB64_H */
