/*
 * rawalign_oracle.h -- declarations of the CPU oracle (test infrastructure
 * only; see rawalign_oracle.c).  This header belongs to the oracle alone: the
 * CUDA library neither includes it nor shares any of its types.
 */
#ifndef RAWALIGN_ORACLE_H
#define RAWALIGN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_END_GLOBAL = 0, ORA_END_FREE = 1 };
enum { ORA_UNMAPPED = 0, ORA_MAPPED = 1, ORA_PENDING = 2 };

typedef struct {
    int unbanded;
    int64_t num, den; /* slope num/den reference values per event */
    int64_t w_eff;    /* half-width in columns after the connectivity raise */
} ora_band_t;

/* One candidate reference region for one read (same field order as the
 * library's candidate record, declared independently here). */
typedef struct {
    uint64_t read_id;
    uint64_t ref_offset;
    uint32_t ref_len_bases;
    uint8_t strand;
    uint8_t pad0[3];
    int32_t band_w;
    int32_t pad1;
    int64_t slope_num;
    int64_t slope_den;
} ora_candidate_t;

typedef struct {
    uint64_t read_id;
    uint32_t cand_idx;
    float cost;
    float score;
    int32_t end_i, end_j;
    int32_t w_eff;
    uint64_t cells;
    int32_t status;
    int32_t is_best;
    int32_t decision;
    int32_t pad;
    double cost64;
    double score64;
} ora_result_t;

int64_t ora_kmer_index(const uint8_t *codes, int k);
int64_t ora_expected_signal(const uint8_t *codes, int64_t n_bases, int k,
                            const float *pore, float *r_out);
int ora_segment_codes(const uint8_t *ref2bit, uint64_t ref_len, uint64_t off,
                      uint64_t len, int strand, uint8_t *out);
int ora_band_params(int64_t n, int64_t m, int64_t band_w, int64_t num,
                    int64_t den, ora_band_t *b);
int ora_in_band(const ora_band_t *b, int64_t i, int64_t j);
uint64_t ora_band_cells(const ora_band_t *b, int64_t n, int64_t m);
int ora_dtw_f32(const float *e, int64_t n, const float *r, int64_t m,
                int64_t band_w, int64_t num, int64_t den, int end_mode,
                float *cost, int64_t *end_i, int64_t *end_j, uint64_t *cells,
                int64_t *w_eff, float *full);
int ora_dtw_f64(const double *e, int64_t n, const double *r, int64_t m,
                int64_t band_w, int64_t num, int64_t den, int end_mode,
                double *cost, int64_t *end_i, int64_t *end_j, uint64_t *cells,
                int64_t *w_eff, double *full);
int ora_brute_f32(const float *e, int64_t n, const float *r, int64_t m,
                  int64_t band_w, int64_t num, int64_t den, int end_mode,
                  float *cost, int64_t *end_j, uint64_t *paths);
int ora_brute_f64(const double *e, int64_t n, const double *r, int64_t m,
                  int64_t band_w, int64_t num, int64_t den, int end_mode,
                  double *cost, int64_t *end_j, uint64_t *paths);
float ora_score_f32(float b_match, int64_t n_read, float cost);
double ora_score_f64(double b_match, int64_t n_read, double cost);
/* One anchor of a chain (Sec. 2.4.2): events q..q+len-1 on the diagonal
 * with expected values t..t+len-1 of the candidate's region. */
typedef struct {
    uint32_t q, t, len;
} ora_anchor_t;

int ora_anchored_f32(const float *e, int64_t n, const float *r, int64_t m,
                     const ora_anchor_t *A, int64_t K, int64_t band_w,
                     float *cost, uint64_t *cells);
int ora_anchored_f64(const double *e, int64_t n, const double *r, int64_t m,
                     const ora_anchor_t *A, int64_t K, int64_t band_w,
                     double *cost, uint64_t *cells);
int ora_anchored_brute(const double *e, int64_t n, const double *r, int64_t m,
                       const ora_anchor_t *A, int64_t K, double *cost);
int ora_map_anchored(int k, float b_match, float score_threshold,
                     const float *pore, const uint8_t *ref2bit, uint64_t ref_len,
                     const float *events, const uint64_t *read_offsets,
                     uint32_t n_reads, const ora_candidate_t *cands,
                     uint32_t n_cands, const ora_anchor_t *anchors,
                     const uint64_t *anchor_offsets, ora_result_t *out, int use_f64);
int ora_traceback_f32(const float *e, int64_t n, const float *r, int64_t m,
                      int64_t band_w, int64_t num, int64_t den, int end_mode,
                      int32_t *path_i, int32_t *path_j, int64_t cap,
                      int64_t *path_len, float *cost);
int ora_map_batch(int k, float b_match, float score_threshold, int end_mode,
                  const float *pore, const uint8_t *ref2bit, uint64_t ref_len,
                  const float *events, const uint64_t *read_offsets,
                  uint32_t n_reads, const ora_candidate_t *cands,
                  uint32_t n_cands, ora_result_t *out, int use_f64);

#ifdef __cplusplus
}
#endif
#endif
