/*
 * The paper's `lookup` validator (Section 6) on the host CPU, 16 bytes at a
 * time -- a CPU baseline for context, beside the GPU library.  It is neither
 * the oracle nor a fallback: only the tests and the benchmark load it.
 *
 * Written with GCC vector extensions, so the same source builds on x86-64
 * and on Arm: on aarch64 the variable 16-byte shuffles become the table
 * lookup instruction (tbl) and the two-vector shuffles that form the previous
 * bytes become ext, which is the NEON form of the algorithm the paper
 * describes for ARM; on a baseline x86-64 build without SSSE3 the compiler
 * expands them into scalar code (same results, slower).
 *
 * Per 16-byte vector v, with p the vector before it (zeros at the start):
 *   prev1, prev2, prev3 = v shifted in from p by 1, 2, 3 bytes
 *   special = byte_1_high[prev1 >> 4] & byte_1_low[prev1 & 15] & byte_2_high[v >> 4]
 *                                                        (Fig. 1, Table 7)
 *   must_be_2_3 = 0x80 where prev2 >= 0xE0 or prev3 >= 0xF0   (Section 6.2)
 *   error |= special ^ must_be_2_3
 * A 64-byte block that is all ASCII skips the classification but must not
 * follow an unfinished character (Section 6.4); one zero vector after the
 * data checks the end of the stream (Section 6.3).
 *
 * Build: gcc -O3 -shared -fPIC -o libcpulookup.so lookup_vec.c -lpthread
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#include <pthread.h>

typedef uint8_t u8x16 __attribute__((vector_size(16)));
typedef uint64_t u64x2 __attribute__((vector_size(16)));

/* Table 8's values of the three 16-entry tables (bit 0 TOO_SHORT, 1 TOO_LONG,
 * 2 OVERLONG_3, 3 TOO_LARGE, 4 SURROGATE, 5 OVERLONG_2, 6 OVERLONG_4 |
 * TOO_LARGE_1000, 7 TWO_CONTS), indexed by nibble value. */
static const u8x16 kByte1High = {0x02, 0x02, 0x02, 0x02, 0x02, 0x02, 0x02, 0x02,
                                 0x80, 0x80, 0x80, 0x80, 0x21, 0x01, 0x15, 0x49};
static const u8x16 kByte1Low = {0xE7, 0xA3, 0x83, 0x83, 0x8B, 0xCB, 0xCB, 0xCB,
                                0xCB, 0xCB, 0xCB, 0xCB, 0xCB, 0xDB, 0xCB, 0xCB};
static const u8x16 kByte2High = {0x01, 0x01, 0x01, 0x01, 0x01, 0x01, 0x01, 0x01,
                                 0xE6, 0xAE, 0xBA, 0xBA, 0x01, 0x01, 0x01, 0x01};

static inline u8x16 load16(const uint8_t* p) {
    u8x16 v;
    memcpy(&v, p, 16);
    return v;
}

/* (p, v) shifted so that lane i holds the byte k positions before v[i]. */
#define PREV(p, v, k)                                                          \
    __builtin_shuffle((p), (v), (u8x16){16 - (k), 17 - (k), 18 - (k), 19 - (k), \
                                        20 - (k), 21 - (k), 22 - (k), 23 - (k), \
                                        24 - (k), 25 - (k), 26 - (k), 27 - (k), \
                                        28 - (k), 29 - (k), 30 - (k), 31 - (k)})

static inline u8x16 check16(u8x16 p, u8x16 v) {
    const u8x16 prev1 = PREV(p, v, 1), prev2 = PREV(p, v, 2), prev3 = PREV(p, v, 3);
    const u8x16 byte_1_high = __builtin_shuffle(kByte1High, prev1 >> 4);
    const u8x16 byte_1_low = __builtin_shuffle(kByte1Low, prev1 & 0x0F);
    const u8x16 byte_2_high = __builtin_shuffle(kByte2High, v >> 4);
    const u8x16 special = byte_1_high & byte_1_low & byte_2_high;
    const u8x16 must_be_2_3 = (u8x16)((prev2 >= 0xE0) | (prev3 >= 0xF0)) & 0x80;
    return special ^ must_be_2_3;
}

/* Some byte of v is non-zero. */
static inline int any16(u8x16 v) {
    const u64x2 w = (u64x2)v;
    return (w[0] | w[1]) != 0;
}

/* The last vector ends inside a character: one of its last three bytes
 * starts a character longer than the bytes left. */
static inline int unfinished(u8x16 v) {
    return v[15] >= 0xC0 || v[14] >= 0xE0 || v[13] >= 0xF0;
}

int cpu_lookup_valid(const uint8_t* s, size_t n) {
    u8x16 prev = {0}, err = {0};
    size_t i = 0;
    for (; i + 64 <= n; i += 64) {
        const u8x16 a = load16(s + i), b = load16(s + i + 16), c = load16(s + i + 32),
                    d = load16(s + i + 48);
        if (!any16((a | b | c | d) & 0x80)) {          /* Section 6.4 */
            if (unfinished(prev)) return 0;
            prev = d;
            continue;
        }
        err |= check16(prev, a) | check16(a, b) | check16(b, c) | check16(c, d);
        prev = d;
    }
    for (; i < n; i += 16) {                           /* zero-padded tail */
        uint8_t buf[16] = {0};
        memcpy(buf, s + i, n - i < 16 ? n - i : 16);
        const u8x16 v = load16(buf);
        err |= check16(prev, v);
        prev = v;
    }
    err |= check16(prev, (u8x16){0});                  /* Section 6.3 */
    return !any16(err);
}

/* One flag per string k = s[offsets[k] .. offsets[k+1]); `threads` POSIX
 * threads take equal contiguous slices of the strings. */
typedef struct {
    const uint8_t* s; const int64_t* offsets; int64_t lo, hi; uint8_t* out;
} job_t;

static void* run_job(void* arg) {
    job_t* j = (job_t*)arg;
    for (int64_t k = j->lo; k < j->hi; ++k)
        j->out[k] = (uint8_t)cpu_lookup_valid(j->s + j->offsets[k],
                                              (size_t)(j->offsets[k + 1] - j->offsets[k]));
    return NULL;
}

void cpu_lookup_valid_batch(const uint8_t* s, const int64_t* offsets, int64_t count,
                            uint8_t* out, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (count < 2 * threads) threads = 1;
    pthread_t tid[256];
    job_t job[256];
    for (int t = 0; t < threads; ++t) {
        job[t] = (job_t){s, offsets, count * t / threads, count * (t + 1) / threads, out};
        if (threads > 1) pthread_create(&tid[t], NULL, run_job, &job[t]);
        else run_job(&job[t]);
    }
    if (threads > 1)
        for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
}
