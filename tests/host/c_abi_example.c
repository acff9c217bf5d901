/* A plain C99 user of the C-ABI (include/utf8gpu.h): validate device buffers,
 * locate an error, validate a small batch.  Exits 0 when every result is the
 * expected one. */
#include <stdio.h>
#include <string.h>

#include <cuda_runtime.h>

#include "utf8gpu.h"

static int upload(uint8_t** d, const void* src, size_t n) {
    if (cudaMalloc((void**)d, n ? n : 1) != cudaSuccess) return 0;
    return cudaMemcpy(*d, src, n, cudaMemcpyHostToDevice) == cudaSuccess;
}

int main(void) {
    const char good[] = "h\xc3\xa9llo w\xc3\xb6rld \xe4\xb8\x96\xe7\x95\x8c \xf0\x9f\x98\x80";
    const char bad[] = "abc\xed\xa0\x80xyz"; /* a surrogate at byte 3 (rule f) */
    const char batch[] = "ok\xc3" "fine\xe2\x82\xac";
    const int64_t offsets[] = {0, 2, 3, 10}; /* "ok", a cut character, "fine" + euro sign */
    uint8_t *d_good, *d_bad, *d_batch, *d_flags;
    int64_t* d_off;
    uint8_t flags[3] = {9, 9, 9};
    utf8_error_info info;
    int fails = 0;

    if (!upload(&d_good, good, strlen(good)) || !upload(&d_bad, bad, strlen(bad)) ||
        !upload(&d_batch, batch, sizeof batch - 1) ||
        cudaMalloc((void**)&d_off, sizeof offsets) != cudaSuccess ||
        cudaMemcpy(d_off, offsets, sizeof offsets, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc((void**)&d_flags, 3) != cudaSuccess) {
        printf("cuda setup failed\n");
        return 2;
    }
    if (!utf8_validate(d_good, strlen(good), NULL)) { printf("good: invalid\n"); ++fails; }
    if (utf8_validate(d_bad, strlen(bad), NULL)) { printf("bad: valid\n"); ++fails; }
    if (utf8_last_error() != UTF8_OK) { printf("status %d\n", utf8_last_error()); ++fails; }
    if (utf8_locate_error(d_bad, strlen(bad), &info, NULL) != UTF8_OK ||
        info.position != 3 || info.rule != UTF8_RULE_SURROGATE) {
        printf("locate: %llu %d\n", (unsigned long long)info.position, info.rule);
        ++fails;
    }
    if (utf8_validate_batch(d_batch, d_off, 3, d_flags, NULL) != UTF8_OK ||
        cudaMemcpy(flags, d_flags, 3, cudaMemcpyDeviceToHost) != cudaSuccess ||
        flags[0] != 1 || flags[1] != 0 || flags[2] != 1) {
        printf("batch: %d %d %d\n", flags[0], flags[1], flags[2]);
        ++fails;
    }
    if (utf8_validate_batch(d_batch, d_off, -1, d_flags, NULL) != UTF8_ERR_INVALID_ARG) {
        printf("count -1 accepted\n");
        ++fails;
    }
    printf("%s (%s)\n", fails ? "FAIL" : "ok", utf8_error_string(UTF8_OK));
    cudaFree(d_good); cudaFree(d_bad); cudaFree(d_batch); cudaFree(d_off); cudaFree(d_flags);
    return fails ? 1 : 0;
}
