/*
 * CPU oracle for UTF-8 validation — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product path (the CUDA kernels behind
 * libutf8gpu.so) never calls it and shares no code, header or table with it.
 *
 * What it computes: the RFC 3629 well-formedness predicate that the paper
 * states in Section 3 (Table 1: the valid code-point ranges and their byte
 * forms; rules a-f: 5+ byte, too short, too long, overlong, too large,
 * surrogate).  The `lookup` algorithm of Section 6 reaches exactly this
 * boolean, so the oracle is that definition written out as a plain decode
 * loop: read a lead byte, decide the sequence length from its header bits,
 * check and accumulate the continuation bytes, then range-check the decoded
 * code point.  It is branchy and slow on purpose.
 *
 * oracle_locate extends the boolean with where it fails: the length of the
 * longest valid prefix and the Section 3 rule (a-f) that the next character
 * breaks, by the same kind of plain decode loop.
 *
 * A second, independent validator, the finite-state machine of Section 5
 * (its state-transition table), lives here as well.  It is not the oracle;
 * the tests use it as one more pin on the oracle (exhaustive agreement on
 * short strings).
 *
 * Build: gcc -O2 -shared -fPIC -o liboracle.so utf8_oracle.c -lpthread
 * With -DORACLE_MUTANT=k one deliberate mistake is planted (tests only),
 * to show that the pins catch it.
 */
#include <stddef.h>
#include <stdint.h>
#include <pthread.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ------------------------------------------------------------------------ */
/* The oracle: decode and range-check (Section 3, Table 1, rules a-f).       */
/* ------------------------------------------------------------------------ */
int oracle_valid(const uint8_t* s, size_t n)
{
    size_t i = 0;
    while (i < n) {
        uint32_t lead = s[i];
        uint32_t len, cp, min_cp;
        if (lead < 0x80) {                 /* 1 byte: ASCII U+0000..U+007F */
            i += 1;
            continue;
        } else if ((lead >> 5) == 0x6) {   /* 110xxxxx: 2 bytes, >= U+0080 */
            len = 2; cp = lead & 0x1F; min_cp = 0x80;
        } else if ((lead >> 4) == 0xE) {   /* 1110xxxx: 3 bytes, >= U+0800 */
            len = 3; cp = lead & 0x0F; min_cp = 0x800;
#if ORACLE_MUTANT == 1                      /* mutant: wrong overlong bound */
            min_cp = 0x80;
#endif
        } else if ((lead >> 3) == 0x1E) {  /* 11110xxx: 4 bytes, >= U+10000 */
            len = 4; cp = lead & 0x07; min_cp = 0x10000;
#if ORACLE_MUTANT == 2                      /* mutant: 5-byte leads admitted */
        } else if ((lead >> 2) == 0x3E) {
            len = 4; cp = lead & 0x03; min_cp = 0x10000;
#endif
        } else {
            /* rule c (a continuation byte 10xxxxxx cannot lead) or
             * rule a (five or more header bits: 11111xxx) */
            return 0;
        }
#if ORACLE_MUTANT == 3                      /* mutant: truncated tail ignored */
        if (n - i < len) return 1;
#else
        if (n - i < len) return 0;         /* rule b: too short at the end */
#endif
        for (uint32_t k = 1; k < len; ++k) {
            uint32_t c = s[i + k];
#if ORACLE_MUTANT == 4                      /* mutant: any byte >= 0x80 continues */
            if (c < 0x80) return 0;
#else
            if ((c >> 6) != 0x2) return 0; /* rule b: not a continuation */
#endif
            cp = (cp << 6) | (c & 0x3F);
        }
        if (cp < min_cp) return 0;         /* rule d: overlong */
#if ORACLE_MUTANT == 5                      /* mutant: off-by-one upper bound */
        if (cp > 0x110000) return 0;
#else
        if (cp > 0x10FFFF) return 0;       /* rule e: too large */
#endif
#if ORACLE_MUTANT != 6                      /* mutant 6: surrogates admitted */
        if (cp >= 0xD800 && cp <= 0xDFFF) return 0;  /* rule f: surrogate */
#endif
        i += len;
    }
    return 1;                              /* the empty string is valid */
}

/* One flag per string: string k is s[offsets[k] .. offsets[k+1]). */
static void batch_range(const uint8_t* data, const int64_t* offsets,
                        int64_t lo, int64_t hi, uint8_t* out)
{
    for (int64_t k = lo; k < hi; ++k)
        out[k] = (uint8_t)oracle_valid(data + offsets[k],
                                       (size_t)(offsets[k + 1] - offsets[k]));
}

typedef struct {
    const uint8_t* data; const int64_t* offsets; int64_t lo, hi; uint8_t* out;
} batch_job;

static void* batch_worker(void* arg)
{
    batch_job* j = (batch_job*)arg;
    batch_range(j->data, j->offsets, j->lo, j->hi, j->out);
    return NULL;
}

/* Validates `count` strings; `threads` > 1 splits the string list into equal
 * contiguous slices, one POSIX thread each (strings are independent). */
void oracle_valid_batch(const uint8_t* data, const int64_t* offsets,
                        int64_t count, uint8_t* out, int threads)
{
    if (threads <= 1 || count < 2 * threads) {
        batch_range(data, offsets, 0, count, out);
        return;
    }
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    batch_job job[256];
    for (int t = 0; t < threads; ++t) {
        job[t].data = data; job[t].offsets = offsets; job[t].out = out;
        job[t].lo = count * t / threads;
        job[t].hi = count * (t + 1) / threads;
        pthread_create(&tid[t], NULL, batch_worker, &job[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Independent pin: the finite-state validator of Section 5.                */
/*                                                                          */
/* Byte categories: the three continuation ranges (the reading taken is     */
/* Low 80..8F, Mid 90..9F, High A0..BF, the one consistent with the         */
/* transitions) and the nine first-byte rows of the transition table.       */
/* ------------------------------------------------------------------------ */
enum { C_LOW, C_MID, C_HIGH,                     /* continuation bytes */
       F_ASCII, F_2, F_3, F_4, F_E0, F_ED, F_F0, F_F4, F_BAD, N_CAT };
enum { S_VALID, S_1, S_2, S_3, S_E0, S_ED, S_F0, S_F4, S_ERROR, N_STATE };

static int fsm_category(uint32_t b)
{
    if (b <= 0x7F) return F_ASCII;
    if (b <= 0x8F) return C_LOW;
    if (b <= 0x9F) return C_MID;
    if (b <= 0xBF) return C_HIGH;
    if (b <= 0xC1) return F_BAD;                 /* 110 00000..00001 */
    if (b <= 0xDF) return F_2;                   /* 110 00010..11111 */
    if (b == 0xE0) return F_E0;
    if (b == 0xED) return F_ED;
    if (b <= 0xEF) return F_3;                   /* E1..EC, EE..EF */
    if (b == 0xF0) return F_F0;
    if (b <= 0xF3) return F_4;                   /* F1..F3 */
    if (b == 0xF4) return F_F4;
    return F_BAD;                                /* F5..FF */
}

static int fsm_next(int state, int cat)
{
    int cont = (cat == C_LOW || cat == C_MID || cat == C_HIGH);
    switch (state) {
    case S_VALID:
        switch (cat) {
        case F_ASCII: return S_VALID;
        case F_2: return S_1;
        case F_3: return S_2;
        case F_4: return S_3;
        case F_E0: return S_E0;
        case F_ED: return S_ED;
        case F_F0: return S_F0;
        case F_F4: return S_F4;
        default: return S_ERROR;                 /* continuation or bad lead */
        }
    case S_1: return cont ? S_VALID : S_ERROR;
    case S_2: return cont ? S_1 : S_ERROR;
    case S_3: return cont ? S_2 : S_ERROR;
    case S_E0: return cat == C_HIGH ? S_1 : S_ERROR;           /* 3-byte overlong */
    case S_ED: return (cat == C_LOW || cat == C_MID) ? S_1 : S_ERROR; /* surrogate */
    case S_F0: return (cat == C_MID || cat == C_HIGH) ? S_2 : S_ERROR; /* 4-byte overlong */
    case S_F4: return cat == C_LOW ? S_2 : S_ERROR;            /* too large */
    default: return S_ERROR;                                    /* sticky */
    }
}

int oracle_fsm_valid(const uint8_t* s, size_t n)
{
    int state = S_VALID;
    for (size_t i = 0; i < n; ++i) state = fsm_next(state, fsm_category(s[i]));
    return state == S_VALID;     /* ending mid-character is an error */
}

/* ------------------------------------------------------------------------ */
/* Enumeration helpers for the exhaustive pins (tests only).                */
/* ------------------------------------------------------------------------ */

/* Counts valid strings among all byte strings of length `len` (1..4) whose
 * first byte is >= lead_min, using the decode oracle (which = 0) or the
 * finite-state validator (which = 1). */
int64_t oracle_count_valid(int len, int lead_min, int which)
{
    uint8_t s[4];
    int64_t count = 0;
    uint64_t total = 1;
    for (int k = 1; k < len; ++k) total <<= 8;
    for (uint32_t b0 = (uint32_t)lead_min; b0 < 256; ++b0) {
        s[0] = (uint8_t)b0;
        for (uint64_t r = 0; r < total; ++r) {
            for (int k = 1; k < len; ++k) s[k] = (uint8_t)(r >> (8 * (k - 1)));
            int v = which ? oracle_fsm_valid(s, (size_t)len) : oracle_valid(s, (size_t)len);
            count += v;
        }
    }
    return count;
}

/* Writes validity of every string of length `len` (1..3) into out[256^len],
 * indexed by the string read as a little-endian integer. */
void oracle_valid_all(int len, uint8_t* out, int which)
{
    uint8_t s[3];
    uint64_t total = 1;
    for (int k = 0; k < len; ++k) total <<= 8;
    for (uint64_t r = 0; r < total; ++r) {
        for (int k = 0; k < len; ++k) s[k] = (uint8_t)(r >> (8 * k));
        out[r] = (uint8_t)(which ? oracle_fsm_valid(s, (size_t)len)
                                 : oracle_valid(s, (size_t)len));
    }
}

/* Agreement of the decode oracle and the finite-state validator over every
 * string of byte classes of length 1..max_len, one representative byte per
 * class taken from reps[0..nreps).  Returns the number of disagreements. */
int64_t oracle_class_disagreements(const uint8_t* reps, int nreps, int max_len)
{
    uint8_t s[16];
    int idx[16];
    int64_t bad = 0;
    if (max_len > 16) max_len = 16;
    for (int len = 1; len <= max_len; ++len) {
        for (int k = 0; k < len; ++k) idx[k] = 0;
        for (;;) {
            for (int k = 0; k < len; ++k) s[k] = reps[idx[k]];
            if (oracle_valid(s, (size_t)len) != oracle_fsm_valid(s, (size_t)len)) ++bad;
            int k = 0;
            while (k < len && ++idx[k] == nreps) idx[k++] = 0;
            if (k == len) break;
        }
    }
    return bad;
}

/* ------------------------------------------------------------------------ */
/* Where validity ends (reported beside the paper's boolean).               */
/*                                                                          */
/* position: the length of the longest prefix of s that is valid under the */
/* Section 3 predicate; it is n exactly when s is valid.  rule: which of    */
/* the Section 3 rules the character starting at `position` breaks,         */
/* numbered as the paper letters them: 1 = a (5+ byte: a lead with five or  */
/* more header bits), 2 = b (too short: fewer continuation bytes than the   */
/* lead announces, before another byte or the end), 3 = c (too long: a      */
/* continuation byte where a character must start), 4 = d (overlong),       */
/* 5 = e (too large), 6 = f (surrogate); 0 when s is valid.  The rules are  */
/* checked in decoding order (header bits, then each continuation byte,     */
/* then the decoded code point), and on a character whose continuation      */
/* bytes are all present at most one of d, e and f can hold.                */
/* ------------------------------------------------------------------------ */
int64_t oracle_locate(const uint8_t* s, size_t n, int32_t* rule)
{
    size_t i = 0;
    while (i < n) {
        uint32_t lead = s[i];
        uint32_t len, cp, min_cp;
        if (lead < 0x80) {
            i += 1;
            continue;
        }
        if ((lead >> 6) == 0x2) { *rule = 3; return (int64_t)i; }      /* rule c */
        if ((lead >> 5) == 0x6) {
            len = 2; cp = lead & 0x1F; min_cp = 0x80;
        } else if ((lead >> 4) == 0xE) {
            len = 3; cp = lead & 0x0F; min_cp = 0x800;
        } else if ((lead >> 3) == 0x1E) {
            len = 4; cp = lead & 0x07; min_cp = 0x10000;
        } else {
            *rule = 1; return (int64_t)i;                              /* rule a */
        }
        for (uint32_t k = 1; k < len; ++k) {
            if (i + k >= n || (s[i + k] >> 6) != 0x2) {
                *rule = 2;                                             /* rule b */
#if ORACLE_MUTANT == 7                      /* mutant: the missing byte's index */
                return (int64_t)(i + k);
#else
                return (int64_t)i;
#endif
            }
            cp = (cp << 6) | (s[i + k] & 0x3F);
        }
#if ORACLE_MUTANT == 8                      /* mutant: C0/C1 leads taken as rule a */
        if (lead == 0xC0 || lead == 0xC1) { *rule = 1; return (int64_t)i; }
#endif
        if (cp < min_cp) { *rule = 4; return (int64_t)i; }             /* rule d */
        if (cp > 0x10FFFF) { *rule = 5; return (int64_t)i; }           /* rule e */
        if (cp >= 0xD800 && cp <= 0xDFFF) { *rule = 6; return (int64_t)i; }  /* f */
        i += len;
    }
    *rule = 0;
    return (int64_t)n;
}

/* Per string k of a batch: position relative to the string's start, rule. */
typedef struct {
    const uint8_t* data; const int64_t* offsets; int64_t lo, hi;
    int64_t* pos; int32_t* rule;
} locate_job;

static void* locate_worker(void* arg)
{
    locate_job* j = (locate_job*)arg;
    for (int64_t k = j->lo; k < j->hi; ++k)
        j->pos[k] = oracle_locate(j->data + j->offsets[k],
                                  (size_t)(j->offsets[k + 1] - j->offsets[k]), &j->rule[k]);
    return NULL;
}

void oracle_locate_batch(const uint8_t* data, const int64_t* offsets, int64_t count,
                         int64_t* pos, int32_t* rule, int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (count < 2 * threads) threads = 1;
    pthread_t tid[256];
    locate_job job[256];
    for (int t = 0; t < threads; ++t) {
        job[t].data = data; job[t].offsets = offsets; job[t].pos = pos; job[t].rule = rule;
        job[t].lo = count * t / threads;
        job[t].hi = count * (t + 1) / threads;
        if (threads > 1) pthread_create(&tid[t], NULL, locate_worker, &job[t]);
        else locate_worker(&job[t]);
    }
    if (threads > 1)
        for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
}
