/*
 * A plain C client of libga (include/ga.h), built with gcc and linked against libga.so: no
 * Python, no PyTorch.  It runs a synchronous 16x16-island run (checkpointed and resumed
 * half way), its pairwise MRCA bounds, and an asynchronous run on the reproducible
 * schedule, and prints FNV-1a hashes of the records and bounds for the test to compare with
 * the Python binding's.  Exit status: 0, or the first failing call's error code negated.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "ga.h"

static uint64_t fnv1a(const void *data, size_t n, uint64_t h)
{
    const unsigned char *p = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

#define CHECK(call)                                                                      \
    do {                                                                                 \
        int rc_ = (call);                                                                \
        if (rc_ != GA_OK) {                                                              \
            fprintf(stderr, "%s failed: %s (%d)\n", #call, ga_strerror(rc_), rc_);       \
            return -rc_;                                                                 \
        }                                                                                \
    } while (0)

int main(void)
{
    ga_config cfg;
    CHECK(ga_config_default(&cfg));
    cfg.rows = 16;
    cfg.cols = 16;
    cfg.seed = 1234;
    cfg.run_id = 7;
    CHECK(ga_config_check(&cfg));

    ga_run *run = NULL;
    CHECK(ga_create(&cfg, NULL, 0, &run));
    CHECK(ga_step(run, 60));
    uint32_t record_bytes = 0;
    CHECK(ga_record_bytes(&cfg, &record_bytes));
    size_t bytes = (size_t)cfg.rows * cfg.cols * cfg.island_size * record_bytes;
    uint8_t probe[1];
    size_t need = 0;
    if (ga_snapshot(run, probe, sizeof probe, &need) != GA_ERANGE || need != bytes) return 3;
    void *half = malloc(bytes), *rec = malloc(bytes);
    if (!half || !rec) return 2;
    CHECK(ga_snapshot(run, half, bytes, &bytes));
    CHECK(ga_step(run, 60));
    CHECK(ga_snapshot(run, rec, bytes, &bytes));
    printf("sync %016llx\n", (unsigned long long)fnv1a(rec, bytes, 1469598103934665603ull));

    /* resume from the checkpoint: the same end state */
    ga_run *again = NULL;
    CHECK(ga_create(&cfg, NULL, 0, &again));
    CHECK(ga_load(again, half, bytes, 60));
    CHECK(ga_step(again, 60));
    void *rec2 = malloc(bytes);
    if (!rec2) return 2;
    CHECK(ga_snapshot(again, rec2, bytes, &bytes));
    printf("resume %016llx\n", (unsigned long long)fnv1a(rec2, bytes, 1469598103934665603ull));

    uint32_t ids[64];
    for (uint32_t i = 0; i < 64; ++i) ids[i] = i * 127u % (16u * 16u * 32u);
    uint32_t lo[64 * 63 / 2], hi[64 * 63 / 2];
    CHECK(ga_mrca_bounds(run, ids, 64, lo, hi));
    uint64_t h = fnv1a(lo, sizeof lo, 1469598103934665603ull);
    printf("mrca %016llx\n", (unsigned long long)fnv1a(hi, sizeof hi, h));

    cfg.mode = GA_ASYNC_SEQUENTIAL;
    ga_run *arun = NULL;
    CHECK(ga_create(&cfg, NULL, 0, &arun));
    CHECK(ga_async_window(arun, 4));
    CHECK(ga_step(arun, 40));
    CHECK(ga_snapshot(arun, rec, bytes, &bytes));
    printf("async %016llx\n", (unsigned long long)fnv1a(rec, bytes, 1469598103934665603ull));

    CHECK(ga_destroy(arun));
    CHECK(ga_destroy(again));
    CHECK(ga_destroy(run));
    free(half);
    free(rec);
    free(rec2);
    return 0;
}
