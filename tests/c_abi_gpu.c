/* One alignment through the C ABI from plain C, host buffers in and out:
   align_create -> align_submit_host -> align_poll -> align_destroy.
   Usage: c_abi_gpu <dir>; reads <dir>/lp.bin (float32 [T][C]), <dir>/tg.bin
   (int32 [L]) and <dir>/dims.txt ("T C L"), writes <dir>/path.bin,
   <dir>/scores.bin (T values each) and <dir>/total.bin. Run by
   tests/test_gpu_c_abi.py, which checks the outputs against the oracle. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "align.h"

static int read_all(const char *dir, const char *name, void *buf, size_t bytes) {
    char p[4096];
    FILE *f;
    size_t got;
    snprintf(p, sizeof p, "%s/%s", dir, name);
    f = fopen(p, "rb");
    if (!f) return -1;
    got = fread(buf, 1, bytes, f);
    fclose(f);
    return got == bytes ? 0 : -1;
}

static int write_all(const char *dir, const char *name, const void *buf, size_t bytes) {
    char p[4096];
    FILE *f;
    size_t put;
    snprintf(p, sizeof p, "%s/%s", dir, name);
    f = fopen(p, "wb");
    if (!f) return -1;
    put = fwrite(buf, 1, bytes, f);
    fclose(f);
    return put == bytes ? 0 : -1;
}

int main(int argc, char **argv) {
    char p[4096];
    long long T = 0, C = 0, L = 0;
    FILE *f;
    float *lp, *scores, total = 0.0f;
    int32_t *tg, *path, status = 1;
    uint64_t id = 0;
    align_ctx *ctx = NULL;
    align_config cfg;
    align_out out;
    int rc;
    if (argc != 2) return 2;
    snprintf(p, sizeof p, "%s/dims.txt", argv[1]);
    f = fopen(p, "r");
    if (!f || fscanf(f, "%lld %lld %lld", &T, &C, &L) != 3) return 3;
    fclose(f);
    lp = (float *)malloc((size_t)(T * C) * sizeof(float));
    tg = (int32_t *)malloc((size_t)(L > 0 ? L : 1) * sizeof(int32_t));
    path = (int32_t *)malloc((size_t)T * sizeof(int32_t));
    scores = (float *)malloc((size_t)T * sizeof(float));
    if (!lp || !tg || !path || !scores) return 4;
    if (read_all(argv[1], "lp.bin", lp, (size_t)(T * C) * sizeof(float)) ||
        (L > 0 && read_all(argv[1], "tg.bin", tg, (size_t)L * sizeof(int32_t))))
        return 5;
    memset(&cfg, 0, sizeof cfg);
    cfg.device = 0;
    rc = align_create(&ctx, &cfg);
    if (rc != ALIGN_OK) {
        fprintf(stderr, "align_create: %s (%s)\n", align_status_string(rc), align_last_error());
        return 6;
    }
    memset(&out, 0, sizeof out);
    out.path = path;
    out.scores = scores;
    out.total = &total;
    rc = align_submit_host(ctx, lp, T, C, tg, L, 0, out, &id);
    if (rc == ALIGN_OK || rc == ALIGN_PENDING) rc = align_poll(ctx, id, -1, &status);
    if (rc != ALIGN_OK) {
        fprintf(stderr, "submit/poll: %s (%s)\n", align_status_string(rc), align_last_error());
        align_destroy(ctx);
        return 7;
    }
    align_destroy(ctx);
    if (write_all(argv[1], "path.bin", path, (size_t)T * sizeof(int32_t)) ||
        write_all(argv[1], "scores.bin", scores, (size_t)T * sizeof(float)) ||
        write_all(argv[1], "total.bin", &total, sizeof total))
        return 8;
    printf("status %d total %.9g\n", (int)status, (double)total);
    return status == ALIGN_OK ? 0 : 9;
}
