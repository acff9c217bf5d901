/*
 * utf8gpu — UTF-8 validation on one GPU with the `lookup` algorithm of
 * J. Keiser and D. Lemire, "Validating UTF-8 In Less Than One Instruction Per
 * Byte" (Software: Practice and Experience, 2021; arXiv 2010.03090).
 *
 * The problem (Section 3): a byte sequence is valid UTF-8 iff it splits into
 * characters of Table 1 -- one ASCII byte 00..7F, or a lead byte with 2..4
 * header bits followed by 1..3 continuation bytes 10xxxxxx -- where the
 * decoded code point is not overlong (rule d), not above U+10FFFF (rule e)
 * and not a surrogate U+D800..U+DFFF (rule f).  The empty sequence is valid.
 * Every entry point computes exactly this predicate, with the three nibble
 * tables, the 3-4 byte check, the end-of-stream check and the ASCII early-out
 * of Section 6, in hand-written CUDA kernels.  There is no CPU fallback: a
 * machine without a usable GPU gets UTF8_ERR_CUDA.
 *
 * Conventions for every entry point
 *   - Pointers named `data`, `offsets`, `out_*` are DEVICE pointers (memory
 *     from cudaMalloc, or managed memory), unless the name says `host`.  The
 *     caller owns all buffers; the library keeps no reference after the work
 *     it queued has run.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     queued on it; entry points documented as asynchronous return before the
 *     GPU has finished and the caller must keep the buffers alive until the
 *     stream passes that point.
 *   - Status: 0 (UTF8_OK) or a UTF8_ERR_* code.  The status of the calling
 *     thread's last call is also kept for utf8_last_error(), which is the only
 *     way to see it for utf8_validate(), whose result is a bool.
 *   - The library allocates small per-device work areas on a device's first
 *     call (a ring of result bytes in pinned host memory mapped into the
 *     device; the staging buffer of utf8_validate_host on its first use); make
 *     that first call before capturing any stream into a CUDA graph.  It never
 *     frees caller memory.  Entry points are thread safe.
 */
#ifndef UTF8GPU_H
#define UTF8GPU_H

#include <stdbool.h>
#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum utf8_status {
    UTF8_OK = 0,
    UTF8_ERR_INVALID_ARG = 1, /* null pointer with len > 0, count < 0, host memory
                                 passed where device memory is required, ... */
    UTF8_ERR_CUDA = 2,        /* a CUDA call failed (no device, launch error, ...) */
    UTF8_ERR_TIMEOUT = 3,     /* a device-side wait ran past its deadline */
    UTF8_ERR_BUDGET = 4,      /* a request would exceed a memory budget */
    UTF8_ERR_NOMEM = 5        /* a library work area could not be allocated */
};

/*
 * Validates one buffer: data[0 .. len).  Returns true iff it is valid UTF-8.
 * Section 3 defines the predicate; Section 6 (Fig. 1, Table 7, Sections
 * 6.2-6.4) the algorithm.  len == 0 returns true without touching the GPU.
 * Synchronises `stream` before returning.  On any error returns false and
 * sets utf8_last_error() (UTF8_ERR_INVALID_ARG for data == NULL with len > 0
 * or for a pointer that is not device memory).
 */
bool utf8_validate(const uint8_t* data, size_t len, cudaStream_t stream);

/*
 * Asynchronous form of utf8_validate: queues the work on `stream` and writes
 * the result to the device byte *out_valid (1 = valid, 0 = invalid) when the
 * stream reaches it.  Makes no synchronisation and no allocation, so it can be
 * captured in a CUDA graph.  Returns a status.
 */
int utf8_validate_async(const uint8_t* data, size_t len, uint8_t* out_valid,
                        cudaStream_t stream);

/*
 * Many independent device buffers in one launch: out_valid[i] = 1 iff
 * data[i][0 .. lens[i]) is valid UTF-8, each buffer checked exactly as
 * utf8_validate checks it (Section 6).  data, lens: host arrays of `count`
 * entries (read during the call; a buffer with lens[i] == 0 may be NULL and
 * is valid); out_valid: device uint8[count].  The buffers' tiles are cut
 * into 128 KiB chunks interleaved across the buffers and taken by the warps
 * from a counter, so buffers bound by HBM bandwidth (ASCII text) and
 * buffers bound by the integer ALU (the classification of non-ASCII text)
 * are checked at the same time rather than one after the other.  Up to 64
 * buffers go in one launch; more are split into launches of 64.  Each
 * launch uses one of 1024 counters the library keeps per device (zeroed on
 * the stream before the launch): at most 1024 of these calls may run on
 * the GPU at once, and a CUDA graph holding this call must not be replayed
 * while it is still running.  Asynchronous, no allocation; returns a status
 * (UTF8_ERR_INVALID_ARG for count < 0, a null array, or a pointer that is
 * not device memory).
 */
int utf8_validate_buffers_async(const uint8_t* const* data, const size_t* lens, int count,
                                uint8_t* out_valid, cudaStream_t stream);

/*
 * The paper's finite-state validator (Section 5: nine states, the continuation
 * ranges 80..8F / 90..9F / A0..BF, one transition per byte) on the GPU, for
 * comparison with the `lookup` path of utf8_validate_async; same arguments,
 * result and status.  Each lane runs four machines over regions of 512 bytes
 * that start at character boundaries (the paper's interleaved regions); the
 * table lives in shared memory.  Asynchronous, no allocation.
 */
int utf8_validate_fsm_async(const uint8_t* data, size_t len, uint8_t* out_valid,
                            cudaStream_t stream);

/*
 * Validates `count` strings in one launch sequence.  String i is
 * data[offsets[i] .. offsets[i+1]) (int64 device array of count + 1
 * non-decreasing entries, offsets[0] >= 0); each string is checked on its own
 * (three virtual zero bytes before and after it, Section 6.3), never seeing
 * its neighbours' bytes.  out_valid: device uint8[count], 1 = valid, 0 =
 * invalid.  data must be non-null (and device memory) even when every string
 * is empty.  Asynchronous on `stream`.  count == 0 is a no-op.  Offsets are not
 * checked by default (utf8_check_offsets below, or UTF8GPU_CHECK_OFFSETS=1,
 * checks them); malformed offsets give unspecified flags, and only a
 * well-formed call is guaranteed to read nothing outside the aligned 16-byte
 * granules that hold bytes of [data + offsets[0], data + offsets[count]).
 * Returns a status.
 */
int utf8_validate_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                        uint8_t* out_valid, cudaStream_t stream);

/*
 * utf8_validate_batch with its arguments in a DEVICE descriptor that the
 * kernels read when they run (count and pointers are not baked into the
 * launch), so a CUDA graph that captures this call replays for any batch
 * written into the descriptor between replays: other pointers, another count.
 * desc: device memory, read on the stream; its fields follow the rules of
 * utf8_validate_batch.  Two kernels: one sets the count flags to 1, the batch
 * pass clears those of invalid strings.  Asynchronous; returns a status
 * (UTF8_ERR_INVALID_ARG for a null or host desc; the descriptor's contents
 * are not checked on the host).
 */
typedef struct {
    const uint8_t* data;    /* device */
    const int64_t* offsets; /* device, count + 1 entries */
    int64_t count;
    uint8_t* out_valid;     /* device, count entries */
} utf8_batch_desc;

int utf8_validate_batch_desc(const utf8_batch_desc* desc, cudaStream_t stream);

/*
 * Checks batch offsets on the device (one pass): offsets[0] >= 0 and
 * offsets[0 .. count] non-decreasing.  Synchronises `stream`; returns
 * UTF8_OK or UTF8_ERR_INVALID_ARG (also for a null or host pointer).
 * With the environment variable UTF8GPU_CHECK_OFFSETS=1 (read once per
 * process) utf8_validate_batch and utf8_locate_errors_batch run this check
 * first and return its error instead of launching: an opt-in debug mode that
 * makes those calls synchronous.
 */
int utf8_check_offsets(const int64_t* offsets, int64_t count, cudaStream_t stream);

/*
 * Where validation fails (the paper's validators answer valid / invalid;
 * these report where and why, from the same `lookup` pass).
 *
 * position: the length of the longest prefix of the input that is valid
 *   UTF-8; it equals the input's length exactly when the input is valid.
 * rule: the Section 3 rule that the character starting at `position` breaks,
 *   numbered as the paper letters the rules a-f (utf8_rule); UTF8_RULE_NONE
 *   when the input is valid.  Rules are taken in decoding order: the lead's
 *   header bits (a, c), then each continuation byte (b), then the decoded
 *   code point (d, e, f; at most one of them can hold).
 *
 * How it is computed: the `lookup` classification (Section 6) marks the first
 * erroneous position p, which lies 0..3 bytes after the failing character's
 * start; the position is the last m <= p at which no character is cut (the
 * end-of-stream check of Section 6.3 applied to the prefix), and the rule
 * comes from decoding the at most four bytes at m.
 */
enum utf8_rule {
    UTF8_RULE_NONE = 0,
    UTF8_RULE_5PLUS_BYTE = 1, /* a: lead byte with five or more header bits (F8..FF) */
    UTF8_RULE_TOO_SHORT = 2,  /* b: fewer continuation bytes than the lead announces */
    UTF8_RULE_TOO_LONG = 3,   /* c: continuation byte where a character must start */
    UTF8_RULE_OVERLONG = 4,   /* d: code point below the minimum for its length */
    UTF8_RULE_TOO_LARGE = 5,  /* e: code point above U+10FFFF */
    UTF8_RULE_SURROGATE = 6   /* f: code point in U+D800..U+DFFF */
};

typedef struct {
    uint64_t position; /* length of the longest valid prefix */
    int32_t rule;      /* enum utf8_rule */
    int32_t reserved;  /* 0 */
} utf8_error_info;

/*
 * Locates the first error of data[0 .. len) (device memory).  *out (device
 * memory, 8-byte aligned, 16 bytes) receives the result when the stream
 * reaches it; it is also the work area of the call, so nothing else may use
 * it until then.  No allocation and no synchronisation (graph capturable).
 * Asynchronous; returns a status (UTF8_ERR_INVALID_ARG for a null or host
 * pointer or a misaligned out).
 */
int utf8_locate_error_async(const uint8_t* data, size_t len, utf8_error_info* out,
                            cudaStream_t stream);

/*
 * Synchronous form: *out_host (host memory) receives the result.  Uses a
 * library ring of device result slots; synchronises `stream`.
 */
int utf8_locate_error(const uint8_t* data, size_t len, utf8_error_info* out_host,
                      cudaStream_t stream);

/*
 * Per string of a batch (the layout and rules of utf8_validate_batch): out is
 * a device array of `count` utf8_error_info (8-byte aligned), position
 * relative to the string's start.  All strings in one launch sequence: the
 * batch pass marks each string's first erroneous position with an atomic
 * minimum in out[i].position, then one thread per string settles position and
 * rule.  Asynchronous; returns a status.
 */
int utf8_locate_errors_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                             utf8_error_info* out, cudaStream_t stream);

/*
 * Validates a buffer in HOST memory: copies it to the GPU through a
 * library-owned staging ring (pinned or pageable source; chunks of the copy
 * overlap with validation of earlier chunks, the 3 bytes before each chunk
 * carried across) and returns true iff it is valid UTF-8.  Synchronous.  On
 * error returns false and sets utf8_last_error().
 */
bool utf8_validate_host(const uint8_t* host_data, size_t len, cudaStream_t stream);

/*
 * Copies src[0 .. len) to dst and validates it in the same pass (the bytes
 * are read from HBM once): the ingest step "copy into place, then validate"
 * fused.  dst, src: device memory, not overlapping (UTF8_ERR_INVALID_ARG
 * otherwise); *out_valid (device byte) = 1 if valid, 0 if not.  When dst and
 * src differ in alignment modulo 16 the call copies first and validates the
 * copy (two passes, still on the GPU).  Asynchronous.
 */
int utf8_copy_validate(uint8_t* dst, const uint8_t* src, size_t len, uint8_t* out_valid,
                       cudaStream_t stream);

/*
 * One chunk of a longer stream (the paper's loop carries the previous block
 * and checks the end of the stream once: Section 6, Section 6.3).  data[0 ..
 * len) (device memory) is checked as it would be inside the whole stream:
 * `prefix` holds the prefix_len (0..3) bytes that precede the chunk in the
 * stream, the byte just before it in bits 0..7, the one before that in bits
 * 8..15, then bits 16..23 (prefix_len = 0 at the start of a stream).  With
 * final_chunk != 0 the end of the stream after this chunk is checked too
 * (an empty final chunk checks only the end).  The result is AND-ed into the
 * device byte *out_valid: it is cleared on an error and never set, so the
 * caller sets it to 1 first and any number of chunks (also on other streams or
 * other GPUs, e.g. shards of one buffer) may share it.  Asynchronous.
 */
int utf8_validate_chunk(const uint8_t* data, size_t len, uint32_t prefix, int prefix_len,
                        int final_chunk, uint8_t* out_valid, cudaStream_t stream);

/*
 * Stream validation with the carried state on the device (no host sync
 * between chunks): the last three bytes of the stream so far and the result.
 * utf8_stream_create allocates it (NULL on error), reset starts a new stream,
 * update validates the next chunk (device memory; asynchronous; chunks may be
 * reused buffers, the state keeps what it needs), finish checks the end of the
 * stream and writes the result (1 = valid) to the device byte *out_valid.
 * Calls on one state must be ordered (same stream, or synchronised).  Apart
 * from create and destroy none of them allocates or synchronises, so a whole
 * sequence reset, updates, finish can be captured in one CUDA graph and
 * replayed (which device slot each update uses is fixed when it is captured;
 * do not mix replays with direct calls on the same state).
 */
typedef struct utf8_stream utf8_stream;
utf8_stream* utf8_stream_create(void);
int utf8_stream_reset(utf8_stream* s, cudaStream_t stream);
int utf8_stream_update(utf8_stream* s, const uint8_t* chunk, size_t len, cudaStream_t stream);
int utf8_stream_finish(utf8_stream* s, uint8_t* out_valid, cudaStream_t stream);
void utf8_stream_destroy(utf8_stream* s);

/*
 * utf8_validate_host without any allocation, for callers that cannot allocate
 * GPU memory when they validate: services whose GPU memory is reserved up
 * front by a pool or another framework, latency-critical paths where
 * cudaMalloc/cudaFree could synchronise the device, code that must keep a
 * fixed footprint.  The paper has no counterpart; it is a packaging of the
 * same kernel.  The input (host memory, len <= 32 MiB; longer inputs are
 * rejected with UTF8_ERR_BUDGET) is staged through a fixed 32 MiB + 4 KiB
 * array compiled into the library.  Under CUDA's lazy module loading (the
 * default) a device gets its copy of the array, and the validation kernels,
 * when the first call on that device loads them, and keeps them until exit:
 * make one call on each device (len 0 is enough; host_data may be NULL)
 * before reserving the device's memory, and before any stream capture
 * begins.  A first call that fails (UTF8_ERR_CUDA, e.g. no memory left to
 * load the module) is retried by the next one.  All calls share the array:
 * calls whose work overlaps on the GPU race on it (serialise them); the array
 * keeps the previous call's bytes, which never affect a later result.
 * Synchronous (waits for `stream`); returns true iff valid, false with
 * utf8_last_error() set otherwise.
 */
bool utf8_validate_host_noalloc(const uint8_t* host_data, size_t len, cudaStream_t stream);

/*
 * Debug view of the classification (Section 6.1, Fig. 1, Table 7; Section
 * 6.2) of one buffer, from the device code the validators run: for each
 * position i in 0 .. len+2 (the buffer followed by its three zero padding
 * bytes, zeros before it) writes
 *   out_special[i] = the second-byte rows of Table 7 that (data[i-1], data[i])
 *     matches, through the three AND-ed nibble tables: bit 0 overlong
 *     2-byte (C0, C1), bit 1 overlong 3-byte (E0 80..9F), bit 2 surrogate
 *     (ED A0..BF), bit 3 too large (F4..FF 90..BF), bit 4 overlong 4-byte or
 *     too large (F0 or F5..FF, then 80..8F).  Where data[i-1] is ASCII and
 *     data[i] a continuation (an error in any case) the bits are unspecified;
 *   out_cont[i] = bit 0: a continuation is expected at i: data[i-1] >= 0xC0
 *     (TOO_SHORT), or exactly one of data[i-2] >= 0xE0 and data[i-3] >= 0xF0
 *     (must_be_2_3; both hold only where a lead follows a 4-byte lead, an
 *     error that position i-2 shows); bit 1: data[i] is a continuation.
 * Position i is an error iff out_special[i] != 0 or its two cont bits differ.
 * out_special, out_cont: device uint8[len + 3].  Asynchronous.
 */
int utf8_classify_debug(const uint8_t* data, size_t len, uint8_t* out_special,
                        uint8_t* out_cont, cudaStream_t stream);

/*
 * Continuous-batching server.  Requests are device-resident buffers submitted
 * from any thread; each is validated exactly as utf8_validate would, but many
 * requests share one launch (a segment batch: each buffer checked on its
 * own, the batch's tiles split evenly across the GPU).  A request is admitted
 * while the bytes of admitted, unfinished requests stay within budget_bytes;
 * later ones wait in arrival order.  A batch is launched when its oldest
 * request has waited window_min_us and no batch is on the GPU, or has waited
 * window_max_us, or max_batch requests are ready; up to `streams` batches run
 * at once, so requests arriving while others are on the GPU are batched and
 * launched without waiting for them.  The buffer of a request must stay
 * valid until its result has been taken.
 */
typedef struct utf8_server utf8_server;

typedef struct {
    uint64_t budget_bytes;  /* default 8 GiB */
    uint32_t window_min_us; /* default 50 */
    uint32_t window_max_us; /* default 500 */
    uint32_t max_batch;     /* requests per launch, default 4096 */
    uint32_t streams;       /* batches in flight, default 4 (max 64) */
} utf8_server_config;

typedef struct {
    uint64_t submitted, completed, batches, bytes, max_admitted_bytes, max_batch_seen;
} utf8_server_stats;

void utf8_server_default_config(utf8_server_config* cfg);

/* NULL on error (utf8_last_error: UTF8_ERR_INVALID_ARG or UTF8_ERR_CUDA).
 * Uses the current device; allocates its streams and descriptor buffers. */
utf8_server* utf8_server_create(const utf8_server_config* cfg);

/* Queues data[0 .. len) (device memory); *ticket identifies the request.
 * UTF8_ERR_BUDGET if len alone exceeds the budget. */
int utf8_server_submit(utf8_server* s, const uint8_t* data, size_t len, uint64_t* ticket);

/* Waits up to timeout_us (< 0: forever) for a request; *valid = 1/0 and
 * *latency_ns = time from arrival to result.  UTF8_ERR_TIMEOUT if not done. */
int utf8_server_result(utf8_server* s, uint64_t ticket, int64_t timeout_us, int* valid,
                       int64_t* latency_ns);

/* Load replay (benchmarks and tests): submits request i (host arrays of
 * device pointers and lengths) arrival_ns[i] after the call starts (busy
 * wait), then waits for all; latency counts from the scheduled arrival. */
int utf8_server_replay(utf8_server* s, const uint8_t* const* datas, const size_t* lens,
                       const int64_t* arrival_ns, int64_t count, uint8_t* out_valid,
                       int64_t* out_latency_ns);

int utf8_server_stats_get(utf8_server* s, utf8_server_stats* out);

/* Finishes all submitted requests, then frees the server. */
void utf8_server_destroy(utf8_server* s);

/* Status of the calling thread's last utf8_* call. */
int utf8_last_error(void);

/* Static, human-readable text for a status code. */
const char* utf8_error_string(int code);

/*
 * Autotuning of the launch configuration (tile rows per warp and resident
 * CTAs per SM, for the single-buffer and the batch kernel) on synthetic data
 * generated on the current device.
 * flags: 0 = use the cached entry of this GPU if there is one (and apply it
 * to the current device), else tune; 1 = retune.  The cache is keyed by GPU
 * name and SM count; it can be saved to and loaded from a JSON file.  Loaded
 * entries apply to devices first used afterwards, and to the current device
 * on utf8_autotune(0).  Return a status.
 */
int utf8_autotune(int flags);
int utf8_tune_cache_load(const char* path);
int utf8_tune_cache_save(const char* path);

/*
 * Writes the launch configuration in use on the current device as a short
 * JSON object into buf (at most cap bytes, NUL terminated): tile rows and
 * CTAs per SM of the single-buffer and batch kernels, the SM count, whether
 * early exit is on, and "staged": whether the 8-row single- and multi-buffer
 * passes stage their tiles through shared memory (the default where the
 * device allows it; UTF8GPU_STAGED=0 keeps them in registers).  Returns the
 * length it needed, or -1.
 */
int utf8_config_json(char* buf, size_t cap);

/*
 * Early exit of single-buffer validation (utf8_validate, utf8_validate_async,
 * the host-memory calls), process-wide.  When on, the warps of the lookup
 * pass look at the buffer's result byte every 16 KiB of their share and stop
 * once another warp has found an error, so an invalid buffer whose first
 * error lies early is rejected after reading a fraction of it.  The answer is
 * the same either way; on valid text the polling loop runs about 2% slower,
 * so the default is off.  The initial setting is the environment variable
 * UTF8GPU_EARLY_EXIT (non-zero = on).  A launch takes the setting in force
 * when it is issued; a captured CUDA graph keeps the one of its capture.
 * Error location (utf8_locate_error*) always stops early: a warp whose
 * remaining bytes all lie after an error already found stops.
 * enable: 0 = off, anything else = on.  Returns the previous setting (0/1).
 */
int utf8_set_early_exit(int enable);

#ifdef __cplusplus
}
#endif

#endif /* UTF8GPU_H */
