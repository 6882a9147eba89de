/*
 * The C ABI used from a plain C99 program, with no Python or PyTorch in the
 * process.  Test infrastructure: it links the CUDA library and, to check it,
 * the CPU oracle (whose two entry points it declares itself below).
 *
 *   abi_parity host   calls that need no GPU: the version string, default
 *                     options, argument errors and their messages;
 *   abi_parity gpu    a 12-bit pair in host memory, a context with 64 bins,
 *                     joint histograms of several 16.16 affines on both
 *                     paths against the oracle's bit for bit, and MI through
 *                     mi_eval_q16 against an FP64 reduction of the oracle's
 *                     histogram (Eq. 1 and Eq. 2, Shannon, nats).
 * Exit status 0 when every check holds; the first failure is printed.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mi.h"

/* oracle entry points (CPU, FP64 / integer; oracle/mi_oracle.c) */
void orc_bin_volume(const void *data, int dtype, int depth, int64_t nvox, int bins, uint8_t *out);
int64_t orc_joint_hist(const uint8_t *fbins, const int nf[3], const void *mov, int mdtype, int mdepth,
                       const int nm[3], const int32_t q[12], int bins, uint64_t *hist);

static int fail(const char *what, const char *detail) {
    fprintf(stderr, "abi_parity: %s%s%s\n", what, detail ? ": " : "", detail ? detail : "");
    return 1;
}

static int host_checks(void) {
    const char *v = mi_version();
    if (!v || !strstr(v, "sm_103a")) return fail("mi_version does not name sm_103a", v);
    mi_options o;
    mi_options_default(&o);
    if (o.kernel != MI_HARD || o.hist_variant != MI_HV_AUTO || o.path != MI_PATH_AUTO || o.use_graphs != 1)
        return fail("mi_options_default gave unexpected defaults", NULL);
    mi_ctx *ctx = (mi_ctx *)1;
    if (mi_create(&ctx, NULL, NULL, 64, NULL) == MI_OK) return fail("mi_create accepted NULL volumes", NULL);
    if (ctx != NULL) return fail("mi_create left a context behind on error", NULL);
    const char *msg = mi_last_error(NULL);
    if (!msg || !msg[0]) return fail("no error message after a rejected call", NULL);
    if (mi_transform_size(NULL) != -1) return fail("mi_transform_size(NULL) is not -1", NULL);
    return 0;
}

/* 12-bit values from a 32-bit linear congruential generator (multiplier 1664525, increment
 * 1013904223), smoothed along x so that neighbouring voxels correlate like image data */
static void fill12(uint16_t *v, int64_t n, uint32_t seed) {
    uint32_t s = seed;
    uint32_t prev = 0;
    for (int64_t i = 0; i < n; ++i) {
        s = s * 1664525u + 1013904223u;
        const uint32_t r = s >> 20; /* 12 bits */
        prev = (prev * 3u + r) / 4u;
        v[i] = (uint16_t)prev;
    }
}

static double shannon_mi(const uint64_t *h, int bins) {
    double N = 0.0;
    for (int c = 0; c < bins * bins; ++c) N += (double)h[c];
    double hf = 0.0, hm = 0.0, hj = 0.0;
    for (int r = 0; r < bins; ++r) {
        double row = 0.0, col = 0.0;
        for (int c = 0; c < bins; ++c) {
            row += (double)h[r * bins + c];
            col += (double)h[c * bins + r];
            const double p = (double)h[r * bins + c] / N;
            if (p > 0.0) hj -= p * log(p);
        }
        if (row > 0.0) hf -= row / N * log(row / N);
        if (col > 0.0) hm -= col / N * log(col / N);
    }
    return hf + hm - hj;
}

static int gpu_checks(void) {
    enum { BINS = 64, NT = 4 };
    const int nf[3] = {37, 29, 23}, nm[3] = {31, 27, 19};
    const int64_t nvf = (int64_t)nf[0] * nf[1] * nf[2], nvm = (int64_t)nm[0] * nm[1] * nm[2];
    uint16_t *f = (uint16_t *)malloc((size_t)nvf * 2), *m = (uint16_t *)malloc((size_t)nvm * 2);
    uint8_t *fb = (uint8_t *)malloc((size_t)nvf);
    uint64_t *want = (uint64_t *)malloc(sizeof(uint64_t) * BINS * BINS);
    uint32_t *got = (uint32_t *)malloc(sizeof(uint32_t) * NT * BINS * BINS);
    if (!f || !m || !fb || !want || !got) return fail("host allocation", NULL);
    fill12(f, nvf, 1u);
    fill12(m, nvm, 2u);
    /* identity; a sub-voxel translation; a shear-rotation-scale mix; a shift whose x lands on the
     * moving volume's last column exactly */
    const int32_t q16[NT][12] = {
        {65536, 0, 0, 0, 0, 65536, 0, 0, 0, 0, 65536, 0},
        {65536, 0, 0, 81920, 0, 65536, 0, -32768, 0, 0, 65536, 49152},
        {64000, 5000, -3000, 20000, -4000, 66000, 2000, -15000, 1000, -2000, 65000, 30000},
        {65536, 0, 0, -6 * 65536, 0, 65536, 0, 0x4000, 0, 0, 65536, 0x8000}};
    mi_volume vf = {f, MI_U16, {nf[0], nf[1], nf[2]}, 12, {1.0f, 1.0f, 1.0f}};
    mi_volume vm = {m, MI_U16, {nm[0], nm[1], nm[2]}, 12, {1.0f, 1.0f, 1.0f}};
    mi_ctx *ctx = NULL;
    if (mi_create(&ctx, &vf, &vm, BINS, NULL) != MI_OK) return fail("mi_create", mi_last_error(NULL));
    orc_bin_volume(f, MI_U16, 12, nvf, BINS, fb);
    const int paths[2] = {MI_PATH_PLAIN, MI_PATH_BATCHED};
    for (int p = 0; p < 2; ++p) {
        if (mi_hist(ctx, 0, NULL, &q16[0][0], NT, paths[p], got) != MI_OK) return fail("mi_hist", mi_last_error(ctx));
        for (int t = 0; t < NT; ++t) {
            orc_joint_hist(fb, nf, m, MI_U16, 12, nm, q16[t], BINS, want);
            for (int c = 0; c < BINS * BINS; ++c)
                if ((uint64_t)got[(size_t)t * BINS * BINS + c] != want[c]) {
                    char buf[96];
                    snprintf(buf, sizeof buf, "path %d, transform %d, cell %d: %u against %llu", paths[p], t, c,
                             got[(size_t)t * BINS * BINS + c], (unsigned long long)want[c]);
                    return fail("histogram differs from the oracle's", buf);
                }
        }
    }
    const float q[1] = {1.0f};
    double mi[NT];
    int64_t cnt[NT];
    if (mi_eval_q16(ctx, &q16[0][0], NT, q, 1, mi, NULL, cnt) != MI_OK) return fail("mi_eval_q16", mi_last_error(ctx));
    for (int t = 0; t < NT; ++t) {
        const int64_t n = orc_joint_hist(fb, nf, m, MI_U16, 12, nm, q16[t], BINS, want);
        const double ref = shannon_mi(want, BINS);
        if (cnt[t] != n) return fail("overlap count differs from the oracle's", NULL);
        if (!(fabs(mi[t] - ref) <= 1e-9 * fmax(1.0, fabs(ref)))) {
            char buf[96];
            snprintf(buf, sizeof buf, "transform %d: %.15g against %.15g", t, mi[t], ref);
            return fail("MI differs from the FP64 reduction of the oracle's histogram", buf);
        }
    }
    mi_destroy(ctx);
    free(f);
    free(m);
    free(fb);
    free(want);
    free(got);
    return 0;
}

int main(int argc, char **argv) {
    if (argc != 2) return fail("usage: abi_parity host|gpu", NULL);
    if (!strcmp(argv[1], "host")) return host_checks();
    if (!strcmp(argv[1], "gpu")) return host_checks() || gpu_checks();
    return fail("unknown mode", argv[1]);
}
