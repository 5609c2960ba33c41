/*
 * rawalign_oracle.c -- plain, slow, single-threaded CPU oracle for the RawAlign
 * DTW alignment path (Lindegger et al., "RawAlign", arXiv 2310.05037).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; the two meet only at the seeded synthetic inputs.
 *
 * Every function writes out the plain definition of one step of the method:
 *   - expected event values from the pore (k-mer) model   Sup. A.1.1
 *   - the sloped band                                      Sec. 2.4.3
 *   - the DTW recurrence and its corner cell               Sec. 2.2
 *   - the score  B_Match * N_Read - C_DTW                  Sec. 2.3
 *   - the mapping decision (best candidate >= threshold)   Sec. 2.3, Sec. 3.1
 * Readings of points the paper leaves open (absolute difference as the
 * distance, anchored start, half-width band around the line through (0,0)
 * and (n-1,m-1), ties resolved towards the smaller index) are listed in the
 * design notes; each is restated where it is used below.
 *
 * Arithmetic: IEEE-754 binary32 (or binary64 for the *_f64 run), round to
 * nearest even, compiled with -ffp-contract=off and without fast-math, so that
 * every add, subtract and multiply is one correctly rounded operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "rawalign_oracle.h"

/* ---------------------------------------------------------------------------
 * Expected event generation (Sup. A.1.1): a noise-free sequencer would report,
 * for the k-mer that starts at reference position j, the pore model's mean
 * current for that k-mer.  Bases are coded A=0, C=1, G=2, T=3 and the k-mer's
 * first base is its most significant base-4 digit.
 * ------------------------------------------------------------------------- */
int64_t ora_kmer_index(const uint8_t *codes, int k)
{
    int64_t idx = 0;
    for (int t = 0; t < k; ++t) {
        int64_t place = 1;
        for (int u = 0; u < k - 1 - t; ++u)
            place *= 4;
        idx += (int64_t)codes[t] * place;
    }
    return idx;
}

int64_t ora_expected_signal(const uint8_t *codes, int64_t n_bases, int k,
                            const float *pore, float *r_out)
{
    if (k < 1 || n_bases < k)
        return 0;
    int64_t m = n_bases - k + 1;
    for (int64_t j = 0; j < m; ++j)
        r_out[j] = pore[ora_kmer_index(codes + j, k)];
    return m;
}

/* Reference segment [off, off+len) of a reference stored four bases per byte,
 * base p in bits 2*(p%4)..2*(p%4)+1 of byte p/4.  strand 1 = reverse
 * complement of the segment (complement of code c is 3-c). */
int ora_segment_codes(const uint8_t *ref2bit, uint64_t ref_len, uint64_t off,
                      uint64_t len, int strand, uint8_t *out)
{
    if (off > ref_len || len > ref_len - off)
        return -1;
    for (uint64_t q = 0; q < len; ++q) {
        uint64_t p = off + q;
        uint8_t c = (uint8_t)((ref2bit[p / 4] >> (2 * (p % 4))) & 3u);
        if (strand == 0)
            out[q] = c;
        else
            out[len - 1 - q] = (uint8_t)(3 - c);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Band (Sec. 2.4.3).  The band follows the line through (0,0) with slope
 * num/den reference values per read event; by default that is the ratio of
 * the two segment lengths, (m-1)/(n-1), so the line ends in the corner cell.
 * A cell (i,j) is kept when its column lies within w columns of the line:
 *     |j*den - i*num| <= w*den          (exact in 64-bit integers)
 * w is raised to w_eff = max(w, ceil(num/(2*den)), 1): consecutive rows then
 * overlap or touch, so a monotone path from (0,0) always exists.
 * band_w < 0, or a single row or column, means no band.
 * ------------------------------------------------------------------------- */
int ora_band_params(int64_t n, int64_t m, int64_t band_w, int64_t num_in,
                    int64_t den_in, ora_band_t *b)
{
    memset(b, 0, sizeof *b);
    if (n < 1 || m < 1)
        return -1;
    if (band_w < 0 || n == 1 || m == 1) {
        b->unbanded = 1;
        b->w_eff = -1;
        return 0;
    }
    int64_t num = num_in, den = den_in;
    if (num == 0 && den == 0) {
        num = m - 1;
        den = n - 1;
    }
    if (num < 0 || den <= 0)
        return -1;
    int64_t half = (num + 2 * den - 1) / (2 * den); /* ceil(num / (2 den)) */
    int64_t w = band_w;
    if (w < half)
        w = half;
    if (w < 1)
        w = 1;
    b->unbanded = 0;
    b->num = num;
    b->den = den;
    b->w_eff = w;
    return 0;
}

int ora_in_band(const ora_band_t *b, int64_t i, int64_t j)
{
    if (b->unbanded)
        return 1;
    int64_t dev = j * b->den - i * b->num;
    if (dev < 0)
        dev = -dev;
    return dev <= b->w_eff * b->den;
}

uint64_t ora_band_cells(const ora_band_t *b, int64_t n, int64_t m)
{
    uint64_t cells = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j)
            cells += (uint64_t)ora_in_band(b, i, j);
    return cells;
}

/* ---------------------------------------------------------------------------
 * DTW (Sec. 2.2).  Rows i are read events e[i], columns j expected values r[j].
 *   d(i,j) = |e[i] - r[j]|                     (absolute signal difference)
 *   D(0,0) = d(0,0)                             (anchored start)
 *   D(i,j) = d(i,j) + min(D(i-1,j-1), D(i-1,j), D(i,j-1))   (NW, N, W)
 * Cells outside the band, and neighbours outside the table, count as +inf.
 * GLOBAL:   C = D(n-1, m-1)  (the corner cell: the paper's "southwest" corner
 *           is read as the last cell, the only one reachable by N/NW/W moves).
 * FREE_END: C = min_j D(n-1, j), the smallest such j on ties (prefix of a read
 *           against a longer reference window).
 * ------------------------------------------------------------------------- */
#define ORA_DTW_BODY(T, ABS, INF)                                               \
    ora_band_t band;                                                            \
    if (ora_band_params(n, m, band_w, num, den, &band) != 0)                    \
        return -1;                                                              \
    T *prev = (T *)malloc(sizeof(T) * (size_t)m);                               \
    T *cur = (T *)malloc(sizeof(T) * (size_t)m);                                \
    if (!prev || !cur) {                                                        \
        free(prev);                                                             \
        free(cur);                                                              \
        return -2;                                                              \
    }                                                                           \
    uint64_t ncell = 0;                                                         \
    for (int64_t i = 0; i < n; ++i) {                                           \
        for (int64_t j = 0; j < m; ++j) {                                       \
            if (!ora_in_band(&band, i, j)) {                                    \
                cur[j] = INF;                                                   \
                continue;                                                       \
            }                                                                   \
            T diff = e[i] - r[j];                                               \
            T dd = ABS(diff);                                                   \
            T best;                                                             \
            if (i == 0 && j == 0) {                                             \
                best = (T)0;                                                    \
            } else {                                                            \
                T nw = (i > 0 && j > 0) ? prev[j - 1] : INF;                    \
                T no = (i > 0) ? prev[j] : INF;                                 \
                T we = (j > 0) ? cur[j - 1] : INF;                              \
                best = nw;                                                      \
                if (no < best)                                                  \
                    best = no;                                                  \
                if (we < best)                                                  \
                    best = we;                                                  \
            }                                                                   \
            cur[j] = dd + best;                                                 \
            ncell++;                                                            \
        }                                                                       \
        if (full)                                                               \
            memcpy(full + (size_t)i * (size_t)m, cur, sizeof(T) * (size_t)m);   \
        T *tmp = prev;                                                          \
        prev = cur;                                                             \
        cur = tmp;                                                              \
    }                                                                           \
    /* prev now holds row n-1 */                                                \
    if (end_mode == ORA_END_GLOBAL) {                                           \
        *cost = prev[m - 1];                                                    \
        *end_i = n - 1;                                                         \
        *end_j = m - 1;                                                         \
    } else {                                                                    \
        T c = INF;                                                              \
        int64_t cj = -1;                                                        \
        for (int64_t j = 0; j < m; ++j)                                         \
            if (prev[j] < c) {                                                  \
                c = prev[j];                                                    \
                cj = j;                                                         \
            }                                                                   \
        *cost = c;                                                              \
        *end_i = (cj < 0) ? -1 : n - 1;                                         \
        *end_j = cj;                                                            \
    }                                                                           \
    *cells = ncell;                                                             \
    if (w_eff)                                                                  \
        *w_eff = band.w_eff;                                                    \
    free(prev);                                                                 \
    free(cur);                                                                  \
    return 0;

int ora_dtw_f32(const float *e, int64_t n, const float *r, int64_t m,
                int64_t band_w, int64_t num, int64_t den, int end_mode,
                float *cost, int64_t *end_i, int64_t *end_j, uint64_t *cells,
                int64_t *w_eff, float *full)
{
    ORA_DTW_BODY(float, fabsf, INFINITY)
}

int ora_dtw_f64(const double *e, int64_t n, const double *r, int64_t m,
                int64_t band_w, int64_t num, int64_t den, int end_mode,
                double *cost, int64_t *end_i, int64_t *end_j, uint64_t *cells,
                int64_t *w_eff, double *full)
{
    ORA_DTW_BODY(double, fabs, (double)INFINITY)
}

/* ---------------------------------------------------------------------------
 * Brute force: the DTW cost is the minimum, over monotone warping paths from
 * (0,0) that step E, S or SE through in-band cells, of the path's cost summed
 * from the start (S <- fl(d + S)).  Because round-to-nearest addition is
 * monotone in S, this minimum equals the DP value bit for bit.  Exponential:
 * tiny inputs only (n, m <= 8).
 * ------------------------------------------------------------------------- */
typedef struct {
    const void *e, *r;
    int64_t n, m;
    const ora_band_t *band;
    int end_mode;
    int dbl;
    double best; /* stored as double; f32 results are exact in double */
    int64_t best_j;
    uint64_t paths;
} ora_bf_t;

static void bf_walk_f32(ora_bf_t *s, int64_t i, int64_t j, float acc)
{
    const float *e = (const float *)s->e, *r = (const float *)s->r;
    if (i == s->n - 1) {
        int end_ok = (s->end_mode == ORA_END_FREE) || (j == s->m - 1);
        if (end_ok) {
            s->paths++;
            if ((double)acc < s->best || ((double)acc == s->best && j < s->best_j)) {
                s->best = (double)acc;
                s->best_j = j;
            }
        }
    }
    static const int di[3] = {0, 1, 1}, dj[3] = {1, 0, 1};
    for (int mv = 0; mv < 3; ++mv) {
        int64_t ni = i + di[mv], nj = j + dj[mv];
        if (ni >= s->n || nj >= s->m || !ora_in_band(s->band, ni, nj))
            continue;
        float diff = e[ni] - r[nj];
        float dd = fabsf(diff);
        bf_walk_f32(s, ni, nj, dd + acc);
    }
}

static void bf_walk_f64(ora_bf_t *s, int64_t i, int64_t j, double acc)
{
    const double *e = (const double *)s->e, *r = (const double *)s->r;
    if (i == s->n - 1) {
        int end_ok = (s->end_mode == ORA_END_FREE) || (j == s->m - 1);
        if (end_ok) {
            s->paths++;
            if (acc < s->best || (acc == s->best && j < s->best_j)) {
                s->best = acc;
                s->best_j = j;
            }
        }
    }
    static const int di[3] = {0, 1, 1}, dj[3] = {1, 0, 1};
    for (int mv = 0; mv < 3; ++mv) {
        int64_t ni = i + di[mv], nj = j + dj[mv];
        if (ni >= s->n || nj >= s->m || !ora_in_band(s->band, ni, nj))
            continue;
        double diff = e[ni] - r[nj];
        double dd = fabs(diff);
        bf_walk_f64(s, ni, nj, dd + acc);
    }
}

static int ora_brute(const void *e, int64_t n, const void *r, int64_t m,
                     int64_t band_w, int64_t num, int64_t den, int end_mode,
                     int dbl, double *cost, int64_t *end_j, uint64_t *paths)
{
    ora_band_t band;
    if (n < 1 || m < 1 || n > 9 || m > 9)
        return -1;
    if (ora_band_params(n, m, band_w, num, den, &band) != 0)
        return -1;
    ora_bf_t s = {e, r, n, m, &band, end_mode, dbl, (double)INFINITY, -1, 0};
    if (ora_in_band(&band, 0, 0)) {
        if (dbl) {
            double d0 = fabs(((const double *)e)[0] - ((const double *)r)[0]);
            bf_walk_f64(&s, 0, 0, d0);
        } else {
            float diff = ((const float *)e)[0] - ((const float *)r)[0];
            bf_walk_f32(&s, 0, 0, fabsf(diff));
        }
    }
    *cost = s.best;
    *end_j = s.best_j;
    *paths = s.paths;
    return 0;
}

int ora_brute_f32(const float *e, int64_t n, const float *r, int64_t m,
                  int64_t band_w, int64_t num, int64_t den, int end_mode,
                  float *cost, int64_t *end_j, uint64_t *paths)
{
    double c;
    int rc = ora_brute(e, n, r, m, band_w, num, den, end_mode, 0, &c, end_j, paths);
    *cost = (float)c;
    return rc;
}

int ora_brute_f64(const double *e, int64_t n, const double *r, int64_t m,
                  int64_t band_w, int64_t num, int64_t den, int end_mode,
                  double *cost, int64_t *end_j, uint64_t *paths)
{
    return ora_brute(e, n, r, m, band_w, num, den, end_mode, 1, cost, end_j, paths);
}

/* ---------------------------------------------------------------------------
 * Score (Sec. 2.3): Score = B_Match * N_Read - C_DTW, as two separately rounded
 * operations (product first), N_Read = the number of read events aligned.
 * ------------------------------------------------------------------------- */
float ora_score_f32(float b_match, int64_t n_read, float cost)
{
    volatile float prod = b_match * (float)n_read;
    return prod - cost;
}

double ora_score_f64(double b_match, int64_t n_read, double cost)
{
    volatile double prod = b_match * (double)n_read;
    return prod - cost;
}

/* ---------------------------------------------------------------------------
 * Whole path for a batch of reads and candidate reference regions, with the
 * semantics of the library's batch call: expected signal, band, DTW, score per
 * candidate; then per read the best score (smallest candidate index on ties)
 * is mapped when it is at least Score_Threshold (Sec. 2.3; defaults
 * B_Match = 0.4, Score_Threshold = 20 in Sec. 3.1).
 * Returns 0, or a negative code for an invalid input (checked before any
 * work): non-finite event, empty read, segment outside the reference,
 * segment shorter than k, read index out of range, bad band slope.
 * ------------------------------------------------------------------------- */
static void ora_decide(uint32_t n_reads, const ora_candidate_t *cands, uint32_t n_cands,
                       float score_threshold, ora_result_t *out, int use_f64);

int ora_map_batch(int k, float b_match, float score_threshold, int end_mode,
                  const float *pore, const uint8_t *ref2bit, uint64_t ref_len,
                  const float *events, const uint64_t *read_offsets,
                  uint32_t n_reads, const ora_candidate_t *cands,
                  uint32_t n_cands, ora_result_t *out, int use_f64)
{
    if (k < 1 || k > 12)
        return -1;
    for (uint32_t q = 0; q < n_reads; ++q) {
        if (read_offsets[q + 1] <= read_offsets[q])
            return -1;
        for (uint64_t x = read_offsets[q]; x < read_offsets[q + 1]; ++x)
            if (!isfinite(events[x]))
                return -1;
    }
    for (uint32_t c = 0; c < n_cands; ++c) {
        const ora_candidate_t *cd = &cands[c];
        if (cd->read_id >= n_reads)
            return -1;
        if (cd->ref_offset > ref_len || cd->ref_len_bases > ref_len - cd->ref_offset)
            return -1;
        if ((int64_t)cd->ref_len_bases < k)
            return -1;
        if (cd->strand > 1)
            return -1;
        int64_t n = (int64_t)(read_offsets[cd->read_id + 1] - read_offsets[cd->read_id]);
        int64_t m = (int64_t)cd->ref_len_bases - k + 1;
        ora_band_t band;
        if (ora_band_params(n, m, cd->band_w, cd->slope_num, cd->slope_den, &band) != 0)
            return -1;
    }

    for (uint32_t c = 0; c < n_cands; ++c) {
        const ora_candidate_t *cd = &cands[c];
        int64_t n = (int64_t)(read_offsets[cd->read_id + 1] - read_offsets[cd->read_id]);
        const float *e = events + read_offsets[cd->read_id];
        uint8_t *codes = (uint8_t *)malloc(cd->ref_len_bases);
        int64_t m = (int64_t)cd->ref_len_bases - k + 1;
        float *r = (float *)malloc(sizeof(float) * (size_t)m);
        ora_segment_codes(ref2bit, ref_len, cd->ref_offset, cd->ref_len_bases,
                          cd->strand, codes);
        ora_expected_signal(codes, cd->ref_len_bases, k, pore, r);
        ora_result_t *o = &out[c];
        memset(o, 0, sizeof *o);
        o->read_id = cd->read_id;
        o->cand_idx = c;
        int64_t ei, ej, weff;
        uint64_t cells;
        if (!use_f64) {
            float cost;
            ora_dtw_f32(e, n, r, m, cd->band_w, cd->slope_num, cd->slope_den,
                        end_mode, &cost, &ei, &ej, &cells, &weff, NULL);
            o->cost = cost;
            o->score = ora_score_f32(b_match, n, cost);
            o->cost64 = cost;
            o->score64 = o->score;
        } else {
            double *e64 = (double *)malloc(sizeof(double) * (size_t)n);
            double *r64 = (double *)malloc(sizeof(double) * (size_t)m);
            for (int64_t x = 0; x < n; ++x)
                e64[x] = e[x];
            for (int64_t x = 0; x < m; ++x)
                r64[x] = r[x];
            double cost;
            ora_dtw_f64(e64, n, r64, m, cd->band_w, cd->slope_num, cd->slope_den,
                        end_mode, &cost, &ei, &ej, &cells, &weff, NULL);
            o->cost64 = cost;
            o->score64 = ora_score_f64((double)b_match, n, cost);
            o->cost = (float)cost;
            o->score = (float)o->score64;
            free(e64);
            free(r64);
        }
        o->end_i = (int32_t)ei;
        o->end_j = (int32_t)ej;
        o->cells = cells;
        o->w_eff = (int32_t)weff;
        o->status = 0;
        free(codes);
        free(r);
    }

    ora_decide(n_reads, cands, n_cands, score_threshold, out, use_f64);
    return 0;
}

/* Per-read decision (Sec. 2.3, Sec. 3.1): scan candidates in index order,
 * keep the first maximum score; the read is mapped iff it is >= threshold. */
static void ora_decide(uint32_t n_reads, const ora_candidate_t *cands, uint32_t n_cands,
                       float score_threshold, ora_result_t *out, int use_f64)
{
    int64_t *best = (int64_t *)malloc(sizeof(int64_t) * (n_reads ? n_reads : 1));
    for (uint32_t q = 0; q < n_reads; ++q)
        best[q] = -1;
    for (uint32_t c = 0; c < n_cands; ++c) {
        uint64_t q = cands[c].read_id;
        double sc = use_f64 ? out[c].score64 : (double)out[c].score;
        if (best[q] < 0) {
            best[q] = c;
        } else {
            double bs = use_f64 ? out[best[q]].score64 : (double)out[best[q]].score;
            if (sc > bs)
                best[q] = c;
        }
    }
    for (uint32_t c = 0; c < n_cands; ++c) {
        uint64_t q = cands[c].read_id;
        double bs = use_f64 ? out[best[q]].score64 : (double)out[best[q]].score;
        out[c].is_best = (best[q] == (int64_t)c);
        out[c].decision = (bs >= (double)score_threshold) ? ORA_MAPPED : ORA_UNMAPPED;
    }
    free(best);
}

/* ---------------------------------------------------------------------------
 * Anchor-guided alignment (Sec. 2.4.2).  A chain gives K anchors, each a run
 * of L events e[q..q+L-1] matched one to one to expected values r[t..t+L-1]
 * (the anchor's diagonal), sorted and disjoint in both sequences.  Only the
 * gaps between anchors are aligned by DTW; the anchors' own cells lie on the
 * diagonal.  Reading taken where the paper leaves details open:
 *   - the alignment runs from (0,0) to (n-1,m-1) and visits, in order,
 *     gap 0, anchor 1, gap 1, ..., anchor K, gap K;
 *   - gap k covers rows [end of anchor k, start of anchor k+1) and the same
 *     for columns (anchor 0 ends at (0,0), anchor K+1 starts at (n,m));
 *   - a gap with rows and columns is a global DTW of its own (anchored start
 *     at its first cell, corner end), banded around the line through its own
 *     corners with the candidate's half-width;
 *   - a gap with rows but no columns aligns each of its events to one
 *     expected value: the previous anchor's last value (the first anchor's
 *     first value for gap 0); symmetrically for columns without rows;
 *   - an anchor adds |e - r| of its diagonal cells, summed in order;
 *   - C = the pieces' costs added in path order, starting from the first
 *     piece; N_Read = n (every event is on the path).
 * Each piece's cost is a sum accumulated from its own first cell, so C is
 * the minimum path cost over paths that stay inside the gap rectangles and
 * anchor diagonals, evaluated piece by piece.
 * ------------------------------------------------------------------------- */
static int ora_anchors_valid(int64_t n, int64_t m, const ora_anchor_t *A, int64_t K)
{
    int64_t pq = 0, pt = 0;
    for (int64_t a = 0; a < K; ++a) {
        if (A[a].len < 1)
            return 0;
        if ((int64_t)A[a].q < pq || (int64_t)A[a].t < pt)
            return 0;
        pq = (int64_t)A[a].q + A[a].len;
        pt = (int64_t)A[a].t + A[a].len;
        if (pq > n || pt > m)
            return 0;
    }
    return 1;
}

#define ORA_ANCHORED_BODY(T, ABS, DTW)                                          \
    if (!ora_anchors_valid(n, m, A, K))                                         \
        return -1;                                                              \
    T C = 0;                                                                    \
    int first = 1;                                                              \
    uint64_t cl = 0;                                                            \
    int64_t pq = 0, pt = 0;                                                     \
    for (int64_t a = 0; a <= K; ++a) {                                          \
        const int64_t q1 = (a < K) ? (int64_t)A[a].q : n;                       \
        const int64_t t1 = (a < K) ? (int64_t)A[a].t : m;                       \
        const int64_t nr = q1 - pq, nc = t1 - pt;                               \
        int has = 0;                                                            \
        T piece = 0;                                                            \
        if (nr > 0 && nc > 0) {                                                 \
            T g;                                                                \
            int64_t ei, ej, we;                                                 \
            uint64_t gc;                                                        \
            if (DTW(e + pq, nr, r + pt, nc, band_w, 0, 0, ORA_END_GLOBAL, &g,   \
                    &ei, &ej, &gc, &we, NULL) != 0)                             \
                return -1;                                                      \
            piece = g;                                                          \
            cl += gc;                                                           \
            has = 1;                                                            \
        } else if (nr > 0) {                                                    \
            const int64_t col = (a > 0) ? pt - 1 : t1;                          \
            T s = 0;                                                            \
            for (int64_t i = pq; i < q1; ++i) {                                 \
                T diff = e[i] - r[col];                                         \
                T dd = ABS(diff);                                               \
                s = (i == pq) ? dd : s + dd;                                    \
            }                                                                   \
            piece = s;                                                          \
            cl += (uint64_t)nr;                                                 \
            has = 1;                                                            \
        } else if (nc > 0) {                                                    \
            const int64_t row = (a > 0) ? pq - 1 : q1;                          \
            T s = 0;                                                            \
            for (int64_t j = pt; j < t1; ++j) {                                 \
                T diff = e[row] - r[j];                                         \
                T dd = ABS(diff);                                               \
                s = (j == pt) ? dd : s + dd;                                    \
            }                                                                   \
            piece = s;                                                          \
            cl += (uint64_t)nc;                                                 \
            has = 1;                                                            \
        }                                                                       \
        if (has) {                                                              \
            C = first ? piece : C + piece;                                      \
            first = 0;                                                          \
        }                                                                       \
        if (a < K) {                                                            \
            T s = 0;                                                            \
            for (int64_t x = 0; x < (int64_t)A[a].len; ++x) {                   \
                T diff = e[A[a].q + x] - r[A[a].t + x];                         \
                T dd = ABS(diff);                                               \
                s = (x == 0) ? dd : s + dd;                                     \
            }                                                                   \
            C = first ? s : C + s;                                              \
            first = 0;                                                          \
            cl += A[a].len;                                                     \
            pq = (int64_t)A[a].q + A[a].len;                                    \
            pt = (int64_t)A[a].t + A[a].len;                                    \
        }                                                                       \
    }                                                                           \
    *cost = C;                                                                  \
    *cells = cl;                                                                \
    return 0;

int ora_anchored_f32(const float *e, int64_t n, const float *r, int64_t m,
                     const ora_anchor_t *A, int64_t K, int64_t band_w,
                     float *cost, uint64_t *cells)
{
    ORA_ANCHORED_BODY(float, fabsf, ora_dtw_f32)
}

int ora_anchored_f64(const double *e, int64_t n, const double *r, int64_t m,
                     const ora_anchor_t *A, int64_t K, int64_t band_w,
                     double *cost, uint64_t *cells)
{
    ORA_ANCHORED_BODY(double, fabs, ora_dtw_f64)
}

/* Brute force for the anchored reading: every N / W / NW path from (0,0) to
 * (n-1,m-1) that visits every anchor cell and whose cells all lie in a gap
 * rectangle, on a one-sided gap's line, or on an anchor's diagonal; the
 * minimum path sum (FP64, tiny tables). */
typedef struct {
    const double *e, *r;
    int64_t n, m;
    const uint8_t *ok;  /* 1: gap cell, 2: anchor cell */
    int64_t n_anchor_cells;
    double best;
} ora_abf_t;

static void abf_walk(ora_abf_t *s, int64_t i, int64_t j, double acc, int64_t seen)
{
    if (i == s->n - 1 && j == s->m - 1) {
        if (seen == s->n_anchor_cells && acc < s->best)
            s->best = acc;
        return;
    }
    static const int di[3] = {0, 1, 1}, dj[3] = {1, 0, 1};
    for (int mv = 0; mv < 3; ++mv) {
        int64_t ni = i + di[mv], nj = j + dj[mv];
        if (ni >= s->n || nj >= s->m || !s->ok[ni * s->m + nj])
            continue;
        abf_walk(s, ni, nj, acc + fabs(s->e[ni] - s->r[nj]), seen + (s->ok[ni * s->m + nj] == 2));
    }
}

int ora_anchored_brute(const double *e, int64_t n, const double *r, int64_t m,
                       const ora_anchor_t *A, int64_t K, double *cost)
{
    if (n < 1 || m < 1 || n > 9 || m > 9 || !ora_anchors_valid(n, m, A, K))
        return -1;
    uint8_t ok[81];
    memset(ok, 0, sizeof ok);
    int64_t pq = 0, pt = 0;
    for (int64_t a = 0; a <= K; ++a) {
        const int64_t q1 = (a < K) ? (int64_t)A[a].q : n;
        const int64_t t1 = (a < K) ? (int64_t)A[a].t : m;
        if (q1 > pq && t1 > pt) {
            for (int64_t i = pq; i < q1; ++i)
                for (int64_t j = pt; j < t1; ++j)
                    ok[i * m + j] = 1;
        } else if (q1 > pq) {
            const int64_t col = (a > 0) ? pt - 1 : t1;
            for (int64_t i = pq; i < q1; ++i)
                ok[i * m + col] = 1;
        } else if (t1 > pt) {
            const int64_t row = (a > 0) ? pq - 1 : q1;
            for (int64_t j = pt; j < t1; ++j)
                ok[row * m + j] = 1;
        }
        if (a < K) {
            for (int64_t x = 0; x < (int64_t)A[a].len; ++x)
                ok[(A[a].q + x) * m + A[a].t + x] = 2;
            pq = (int64_t)A[a].q + A[a].len;
            pt = (int64_t)A[a].t + A[a].len;
        }
    }
    int64_t n_anchor_cells = 0;
    for (int64_t a = 0; a < K; ++a)
        n_anchor_cells += A[a].len;
    ora_abf_t s = {e, r, n, m, ok, n_anchor_cells, (double)INFINITY};
    if (ok[0])
        abf_walk(&s, 0, 0, fabs(e[0] - r[0]), ok[0] == 2);
    *cost = s.best;
    return 0;
}

/* Whole-path oracle for a batch in anchor-guided mode: as ora_map_batch with
 * GLOBAL ends, each candidate c aligned through its anchors
 * anchors[anchor_offsets[c] .. anchor_offsets[c+1]) (columns relative to the
 * candidate's expected-signal row).  end = (n-1, m-1); w_eff reports the
 * given half-width (-1 without a band); cells = DP cells of the gaps plus the
 * cells on anchors and one-sided gaps. */
int ora_map_anchored(int k, float b_match, float score_threshold,
                     const float *pore, const uint8_t *ref2bit, uint64_t ref_len,
                     const float *events, const uint64_t *read_offsets,
                     uint32_t n_reads, const ora_candidate_t *cands,
                     uint32_t n_cands, const ora_anchor_t *anchors,
                     const uint64_t *anchor_offsets, ora_result_t *out, int use_f64)
{
    if (k < 1 || k > 12)
        return -1;
    for (uint32_t q = 0; q < n_reads; ++q) {
        if (read_offsets[q + 1] <= read_offsets[q])
            return -1;
        for (uint64_t x = read_offsets[q]; x < read_offsets[q + 1]; ++x)
            if (!isfinite(events[x]))
                return -1;
    }
    for (uint32_t c = 0; c < n_cands; ++c) {
        const ora_candidate_t *cd = &cands[c];
        if (cd->read_id >= n_reads || cd->strand > 1)
            return -1;
        if (cd->ref_offset > ref_len || cd->ref_len_bases > ref_len - cd->ref_offset)
            return -1;
        if ((int64_t)cd->ref_len_bases < k)
            return -1;
        if (anchor_offsets[c + 1] < anchor_offsets[c])
            return -1;
        int64_t n = (int64_t)(read_offsets[cd->read_id + 1] - read_offsets[cd->read_id]);
        int64_t m = (int64_t)cd->ref_len_bases - k + 1;
        if (!ora_anchors_valid(n, m, anchors + anchor_offsets[c],
                               (int64_t)(anchor_offsets[c + 1] - anchor_offsets[c])))
            return -1;
    }
    for (uint32_t c = 0; c < n_cands; ++c) {
        const ora_candidate_t *cd = &cands[c];
        int64_t n = (int64_t)(read_offsets[cd->read_id + 1] - read_offsets[cd->read_id]);
        const float *e = events + read_offsets[cd->read_id];
        int64_t m = (int64_t)cd->ref_len_bases - k + 1;
        uint8_t *codes = (uint8_t *)malloc(cd->ref_len_bases);
        float *r = (float *)malloc(sizeof(float) * (size_t)m);
        ora_segment_codes(ref2bit, ref_len, cd->ref_offset, cd->ref_len_bases, cd->strand, codes);
        ora_expected_signal(codes, cd->ref_len_bases, k, pore, r);
        const ora_anchor_t *A = anchors + anchor_offsets[c];
        int64_t K = (int64_t)(anchor_offsets[c + 1] - anchor_offsets[c]);
        ora_result_t *o = &out[c];
        memset(o, 0, sizeof *o);
        o->read_id = cd->read_id;
        o->cand_idx = c;
        uint64_t cells = 0;
        int rc;
        if (!use_f64) {
            float cost;
            rc = ora_anchored_f32(e, n, r, m, A, K, cd->band_w, &cost, &cells);
            o->cost = cost;
            o->score = ora_score_f32(b_match, n, cost);
            o->cost64 = cost;
            o->score64 = o->score;
        } else {
            double *e64 = (double *)malloc(sizeof(double) * (size_t)n);
            double *r64 = (double *)malloc(sizeof(double) * (size_t)m);
            for (int64_t x = 0; x < n; ++x)
                e64[x] = e[x];
            for (int64_t x = 0; x < m; ++x)
                r64[x] = r[x];
            double cost;
            rc = ora_anchored_f64(e64, n, r64, m, A, K, cd->band_w, &cost, &cells);
            o->cost64 = cost;
            o->score64 = ora_score_f64((double)b_match, n, cost);
            o->cost = (float)cost;
            o->score = (float)o->score64;
            free(e64);
            free(r64);
        }
        free(codes);
        free(r);
        if (rc != 0)
            return -1;
        o->end_i = (int32_t)(n - 1);
        o->end_j = (int32_t)(m - 1);
        o->cells = cells;
        o->w_eff = cd->band_w < 0 ? -1 : cd->band_w;
        o->status = 0;
    }
    ora_decide(n_reads, cands, n_cands, score_threshold, out, use_f64);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Traceback (the warping path; the paper computes it only on request,
 * Sec. 2.4): from the end cell, step to the predecessor whose DP value is
 * the minimum the recurrence took, preferring NW, then N, then W on ties,
 * until (0,0).  The path is returned from (0,0) to the end cell.  Every cell
 * of the full FP32 table comes from ora_dtw_f32.
 * ------------------------------------------------------------------------- */
int ora_traceback_f32(const float *e, int64_t n, const float *r, int64_t m,
                      int64_t band_w, int64_t num, int64_t den, int end_mode,
                      int32_t *path_i, int32_t *path_j, int64_t cap,
                      int64_t *path_len, float *cost)
{
    if (n < 1 || m < 1 || cap < n + m - 1)
        return -1;
    float *D = (float *)malloc(sizeof(float) * (size_t)n * (size_t)m);
    if (!D)
        return -2;
    int64_t ei, ej, we;
    uint64_t cells;
    if (ora_dtw_f32(e, n, r, m, band_w, num, den, end_mode, cost, &ei, &ej, &cells, &we, D) != 0) {
        free(D);
        return -1;
    }
    *path_len = 0;
    if (!(*cost < INFINITY) || ei < 0) {
        free(D);
        return 0;
    }
    int64_t i = ei, j = ej, len = 0;
    while (1) {
        path_i[len] = (int32_t)i;
        path_j[len] = (int32_t)j;
        ++len;
        if (i == 0 && j == 0)
            break;
        float nw = (i > 0 && j > 0) ? D[(i - 1) * m + (j - 1)] : INFINITY;
        float no = (i > 0) ? D[(i - 1) * m + j] : INFINITY;
        float wv = (j > 0) ? D[i * m + (j - 1)] : INFINITY;
        float best = nw;
        if (no < best)
            best = no;
        if (wv < best)
            best = wv;
        if (nw == best) {
            --i;
            --j;
        } else if (no == best) {
            --i;
        } else {
            --j;
        }
    }
    for (int64_t a = 0, b = len - 1; a < b; ++a, --b) {
        int32_t t = path_i[a];
        path_i[a] = path_i[b];
        path_i[b] = t;
        t = path_j[a];
        path_j[a] = path_j[b];
        path_j[b] = t;
    }
    *path_len = len;
    free(D);
    return 0;
}
