/*
 * Seeded synthetic UTF-8 text for tests and benchmarks.
 *
 * This module only produces input bytes; it holds none of the validation
 * arithmetic and is shared, as an input source only, by the GPU tests, the
 * oracle checks and the benchmark.
 *
 * Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used as a counter-based generator:
 * draw i of stream s is mix(s + (i + 1) * golden), so every segment of every
 * buffer or string has its own reproducible stream and the output does not
 * depend on the number of threads.
 *
 * Content models (uniform choice of the encoded length per character, then a
 * uniform code point in that length's range, as the paper's generator does
 * in Section 7.3; surrogates never drawn):
 *   0 ASCII   : 0x20..0x7E with a newline on average every 80 bytes
 *   1 LATIN   : 85% printable ASCII, 15% U+0080..U+07FF
 *   2 CJK     : 20% printable ASCII, 80% U+4E00..U+9FFF
 *   3 EMOJI   : 50% printable ASCII, 50% U+1F300..U+1FAFF
 *   4 UNIFORM : length 1..4 uniform, code point uniform in its range
 *   5 RAND12  : length 1..2 uniform (the paper's "1-2 bytes" input)
 *   6 RAND13  : length 1..3 uniform
 * Every segment is filled to its exact length: when the next character does
 * not fit, the rest is printable ASCII.
 */
#include <stddef.h>
#include <stdint.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s; } rng_t;

static inline uint64_t next64(rng_t* r) { r->s += GOLDEN; return mix64(r->s); }

/* uniform integer in [0, n) (n < 2^32), by the high half of a 64x32 product */
static inline uint32_t below(rng_t* r, uint32_t n)
{
    return (uint32_t)(((next64(r) >> 32) * (uint64_t)n) >> 32);
}

static int put_cp(uint8_t* out, uint32_t cp)
{
    if (cp < 0x80) { out[0] = (uint8_t)cp; return 1; }
    if (cp < 0x800) {
        out[0] = (uint8_t)(0xC0 | (cp >> 6));
        out[1] = (uint8_t)(0x80 | (cp & 0x3F));
        return 2;
    }
    if (cp < 0x10000) {
        out[0] = (uint8_t)(0xE0 | (cp >> 12));
        out[1] = (uint8_t)(0x80 | ((cp >> 6) & 0x3F));
        out[2] = (uint8_t)(0x80 | (cp & 0x3F));
        return 3;
    }
    out[0] = (uint8_t)(0xF0 | (cp >> 18));
    out[1] = (uint8_t)(0x80 | ((cp >> 12) & 0x3F));
    out[2] = (uint8_t)(0x80 | ((cp >> 6) & 0x3F));
    out[3] = (uint8_t)(0x80 | (cp & 0x3F));
    return 4;
}

static uint32_t printable(rng_t* r) { return 0x20 + below(r, 0x5F); }

static uint32_t uniform_of_len(rng_t* r, int len)
{
    switch (len) {
    case 1: return below(r, 0x80);
    case 2: return 0x80 + below(r, 0x800 - 0x80);
    case 3: {   /* U+0800..U+FFFF without U+D800..U+DFFF */
        uint32_t v = 0x800 + below(r, 0x10000 - 0x800 - 0x800);
        return v >= 0xD800 ? v + 0x800 : v;
    }
    default: return 0x10000 + below(r, 0x110000 - 0x10000);
    }
}

static uint32_t draw_cp(rng_t* r, int model)
{
    switch (model) {
    case 0:
        return below(r, 80) == 0 ? 0x0A : printable(r);
    case 1:
        return below(r, 100) < 85 ? printable(r) : 0x80 + below(r, 0x800 - 0x80);
    case 2:
        return below(r, 100) < 20 ? printable(r) : 0x4E00 + below(r, 0xA000 - 0x4E00);
    case 3:
        return below(r, 2) == 0 ? printable(r) : 0x1F300 + below(r, 0x1FB00 - 0x1F300);
    case 5:
        return uniform_of_len(r, 1 + (int)below(r, 2));
    case 6:
        return uniform_of_len(r, 1 + (int)below(r, 3));
    default:
        return uniform_of_len(r, 1 + (int)below(r, 4));
    }
}

/* Fills exactly n bytes of valid UTF-8 from one stream. */
void synth_fill(uint8_t* out, size_t n, uint64_t stream, int model)
{
    rng_t r = { mix64(stream) };
    uint8_t tmp[4];
    size_t i = 0;
    while (i < n) {
        int len = put_cp(tmp, draw_cp(&r, model));
        if ((size_t)len > n - i) break;
        for (int k = 0; k < len; ++k) out[i + k] = tmp[k];
        i += (size_t)len;
    }
    while (i < n) out[i++] = (uint8_t)printable(&r);
}

/* A string (or a whole buffer) is cut into segments of `seg` bytes; segment j
 * of string k draws from stream mix(seed ^ mix(k)) + j. */
typedef struct {
    uint8_t* data; const int64_t* offsets; const uint8_t* models; int model;
    int64_t count; uint64_t seed; int64_t seg;
    const int64_t* work_string; const int64_t* work_first;   /* prefix over segments */
    int64_t nwork; volatile int64_t next;
    pthread_mutex_t lock;
} fill_job;

static void fill_segment(fill_job* J, int64_t k, int64_t j)
{
    int64_t lo = J->offsets[k] + j * J->seg;
    int64_t hi = lo + J->seg;
    if (hi > J->offsets[k + 1]) hi = J->offsets[k + 1];
    int model = J->models ? J->models[k] : J->model;
    uint64_t stream = (J->seed ^ mix64((uint64_t)k + 1)) + (uint64_t)j * GOLDEN;
    synth_fill(J->data + lo, (size_t)(hi - lo), stream, model);
}

static void* fill_worker(void* arg)
{
    fill_job* J = (fill_job*)arg;
    const int64_t batch = 16;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t w0 = J->next;
        J->next = w0 + batch;
        pthread_mutex_unlock(&J->lock);
        if (w0 >= J->nwork) return NULL;
        int64_t w1 = w0 + batch < J->nwork ? w0 + batch : J->nwork;
        /* locate the string owning segment w0 (binary search), then walk */
        int64_t lo = 0, hi = J->count;        /* work_first[k] <= w < work_first[k+1] */
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (J->work_first[mid] <= w0) lo = mid; else hi = mid;
        }
        int64_t k = lo;
        for (int64_t w = w0; w < w1; ++w) {
            while (J->work_first[k + 1] <= w) ++k;
            fill_segment(J, k, w - J->work_first[k]);
        }
    }
}

/* Fills `count` strings; string k is data[offsets[k] .. offsets[k+1]) and uses
 * content model models[k] (or `model` when models is NULL).  work_first must
 * have count+1 entries of scratch space. */
void synth_fill_strings(uint8_t* data, const int64_t* offsets, int64_t count,
                        const uint8_t* models, int model, uint64_t seed,
                        int64_t seg, int threads, int64_t* work_first)
{
    if (count <= 0) return;
    if (seg <= 0) seg = 1 << 20;
    work_first[0] = 0;
    for (int64_t k = 0; k < count; ++k) {
        int64_t len = offsets[k + 1] - offsets[k];
        work_first[k + 1] = work_first[k] + (len + seg - 1) / seg;
    }
    fill_job J;
    J.data = data; J.offsets = offsets; J.models = models; J.model = model;
    J.count = count; J.seed = seed; J.seg = seg; J.work_string = NULL;
    J.work_first = work_first; J.nwork = work_first[count]; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (threads < 1) threads = 1;
    if (threads > 128) threads = 128;
    pthread_t tid[128];
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, fill_worker, &J);
    fill_worker(&J);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&J.lock);
}
