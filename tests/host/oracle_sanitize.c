/* oracle_sanitize.c -- drives every entry point of the CPU oracle on small
 * random inputs, built with AddressSanitizer and UndefinedBehaviorSanitizer by
 * tests/test_oracle_sanitizers.py: any out-of-bounds access, leak, signed
 * overflow or other undefined behaviour in the oracle aborts the run.  It
 * checks no values (the pins do that); it only exercises the code paths:
 * bands with and without given slopes, both end modes, FP32 and FP64, brute
 * force, anchors, traceback and the whole-batch mapping with both strands. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "rawalign_oracle.h"

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t next(void)
{
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return st;
}
static int64_t uni(int64_t lo, int64_t hi) { return lo + (int64_t)(next() % (uint64_t)(hi - lo + 1)); }
static float unif(void) { return (float)((next() >> 11) * (1.0 / 9007199254740992.0)) * 4.0f - 2.0f; }

int main(void)
{
    long calls = 0;
    for (int rep = 0; rep < 3000; ++rep) {
        const int64_t n = uni(1, rep < 2000 ? 7 : 60), m = uni(1, rep < 2000 ? 7 : 60);
        float e[64], r[64];
        double e64[64], r64[64];
        for (int64_t i = 0; i < n; ++i)
            e64[i] = e[i] = unif();
        for (int64_t j = 0; j < m; ++j)
            r64[j] = r[j] = unif();
        const int64_t bw = uni(-1, 6), given = uni(0, 2) == 0;
        const int64_t num = given ? uni(0, 5) : 0, den = given ? uni(1, 5) : 0;
        for (int end = 0; end < 2; ++end) {
            float c32;
            double c64;
            int64_t ei, ej, we;
            uint64_t cells, paths;
            ora_dtw_f32(e, n, r, m, bw, num, den, end, &c32, &ei, &ej, &cells, &we, NULL);
            float *full = malloc(sizeof(float) * (size_t)(n * m));
            ora_dtw_f32(e, n, r, m, bw, num, den, end, &c32, &ei, &ej, &cells, &we, full);
            free(full);
            ora_dtw_f64(e64, n, r64, m, bw, num, den, end, &c64, &ei, &ej, &cells, &we, NULL);
            if (n <= 7 && m <= 7) {
                ora_brute_f32(e, n, r, m, bw, num, den, end, &c32, &ej, &paths);
                ora_brute_f64(e64, n, r64, m, bw, num, den, end, &c64, &ej, &paths);
            }
            int32_t pi[128], pj[128];
            int64_t len;
            ora_traceback_f32(e, n, r, m, bw, num, den, end, pi, pj, 128, &len, &c32);
            calls += 6;
        }
        /* anchors: sorted, disjoint runs inside the table (and some invalid) */
        ora_anchor_t A[4];
        int64_t K = 0, q = 0, t = 0;
        while (K < 4 && q < n && t < m && uni(0, 3)) {
            const int64_t q0 = uni(q, n - 1), t0 = uni(t, m - 1);
            const int64_t ln = uni(1, (n - q0 < m - t0 ? n - q0 : m - t0));
            A[K].q = (uint32_t)q0;
            A[K].t = (uint32_t)t0;
            A[K].len = (uint32_t)ln;
            ++K;
            q = q0 + ln;
            t = t0 + ln;
        }
        float ca;
        double cad;
        uint64_t cells;
        ora_anchored_f32(e, n, r, m, A, K, bw, &ca, &cells);
        ora_anchored_f64(e64, n, r64, m, A, K, bw, &cad, &cells);
        if (n <= 7 && m <= 7)
            ora_anchored_brute(e64, n, r64, m, A, K, &cad);
        if (K) {
            ora_anchor_t bad = A[0];
            bad.len = (uint32_t)(n + m);
            ora_anchored_f32(e, n, r, m, &bad, 1, bw, &ca, &cells);
        }
        calls += 4;
    }
    /* a whole batch: random reference, pore table, reads and candidates */
    const int k = 6;
    const uint64_t ref_len = 5000;
    uint8_t *ref = malloc((ref_len + 3) / 4);
    for (uint64_t x = 0; x < (ref_len + 3) / 4; ++x)
        ref[x] = (uint8_t)next();
    float *pore = malloc(sizeof(float) * 4096);
    for (int x = 0; x < 4096; ++x)
        pore[x] = unif();
    enum { NR = 20, NC = 60 };
    uint64_t offs[NR + 1];
    offs[0] = 0;
    for (int x = 0; x < NR; ++x)
        offs[x + 1] = offs[x] + (uint64_t)uni(1, 80);
    float *ev = malloc(sizeof(float) * offs[NR]);
    for (uint64_t x = 0; x < offs[NR]; ++x)
        ev[x] = unif();
    ora_candidate_t c[NC];
    ora_anchor_t an[NC * 2];
    uint64_t aoff[NC + 1];
    aoff[0] = 0;
    memset(c, 0, sizeof c);
    for (int x = 0; x < NC; ++x) {
        c[x].read_id = (uint64_t)uni(0, NR - 1);
        c[x].ref_len_bases = (uint32_t)uni(k, 120);
        c[x].ref_offset = (uint64_t)uni(0, (int64_t)(ref_len - c[x].ref_len_bases));
        c[x].strand = (uint8_t)uni(0, 1);
        c[x].band_w = (int32_t)uni(-1, 30);
        aoff[x + 1] = aoff[x];
        const int64_t nn = (int64_t)(offs[c[x].read_id + 1] - offs[c[x].read_id]);
        const int64_t mm = (int64_t)c[x].ref_len_bases - k + 1;
        if (nn > 2 && mm > 2) {
            an[aoff[x + 1]].q = 1;
            an[aoff[x + 1]].t = 1;
            an[aoff[x + 1]].len = 1;
            aoff[x + 1]++;
        }
    }
    ora_result_t out[NC];
    for (int end = 0; end < 2; ++end)
        for (int f64 = 0; f64 < 2; ++f64)
            ora_map_batch(k, 0.4f, 20.0f, end, pore, ref, ref_len, ev, offs, NR, c, NC, out, f64);
    ora_map_anchored(k, 0.4f, 20.0f, pore, ref, ref_len, ev, offs, NR, c, NC, an, aoff, out, 0);
    ora_map_anchored(k, 0.4f, 20.0f, pore, ref, ref_len, ev, offs, NR, c, NC, an, aoff, out, 1);
    free(ref);
    free(pore);
    free(ev);
    printf("oracle sanitizer run: %ld calls, no report\n", calls + 6);
    return 0;
}
