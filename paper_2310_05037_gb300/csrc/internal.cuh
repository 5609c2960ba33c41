// internal.cuh -- device-side records shared by the kernels and the host engine
// of librawalign_dtw (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rawalign_dtw.h"

namespace ra {

constexpr float kInf = __builtin_huge_valf();
constexpr int kBigCol = 0x3FFFFFFF;  // column index no band reaches: masks a row off
// Columns by which lane t of a striped group trails lane t-1 (the planner's
// schedule and the kernel must agree).
constexpr int kLaneLag = 2;

// One alignment, or one chunk of rows of one alignment (serving).
// Rows are read events (global index row0 .. row0+nrows-1); columns are the
// candidate's expected values 0..m-1; the band is |j*den - i*num| <= w*den
// with global row index i (Sec. 2.4.3).
struct WorkDesc {
    uint64_t ev_off;    // index in the events array of row row0
    uint64_t r_off;     // index in r_all of column 0
    uint64_t fin_off;   // frontier store index of the row above row0 (its first band column)
    uint64_t fout_off;  // frontier store index for the last row (serving)
    int64_t num, den;   // band slope (unbanded: 0, 1 with w = m)
    int32_t row0;       // first row (global index)
    int32_t nrows;      // rows in this piece
    int32_t m;          // columns
    int32_t w;          // band half-width w_eff (>= 1)
    int32_t cand;       // result slot (candidate index)
    int32_t read;       // read slot for the per-read best
    int32_t n_read;     // N_Read for the score
    int32_t fin_lo;     // first column of the stored row above (row0-1); -1 = virtual start
    int32_t fin_wid;    // stored columns - 1 (0 with the virtual start)
    int32_t fout_lo;    // first column of the last row's band (serving)
    int32_t dC;         // stripe period (steps between a lane's stripes)
    int32_t w_report;   // w_eff reported in the result (-1 = no band)
    int32_t a0;         // first in-band column of row0
    int32_t s_end;      // steps until the group is done (<= 0: no in-band cell)
    uint64_t cells;     // in-band cells of the piece (the host counts them exactly)
};
static_assert(sizeof(WorkDesc) == 112, "WorkDesc layout");

// Per-candidate description for the expected-signal step.
struct SigDesc {
    uint64_t ref_off;   // first base in the reference
    uint64_t r_off;     // first output value in r_all
    uint32_t len;       // bases in the region
    uint32_t strand;    // 1 = reverse complement
};

struct StripeParams {
    const WorkDesc *work;
    int n_work;
    int *queue;                    // next work item (atomic counter)
    const float *events;
    const float *r_all;
    const float *fstore;           // frontier store (rows above row0)
    float *fstore_out;             // frontier store for the last rows (serving)
    rawalign_result_t *results;
    unsigned long long *best_keys; // per read: (ordered score << 32) | ~cand
    float *gring;                  // global ring buffers when not in shared memory
    int ring_cap;                  // power of two, floats per group
    int ring_in_smem;
    float b_match;
    int end_free;                  // 1: FREE end (min over the last row)
    int *err;                      // error word (first failing work item + 1)
    int early_term;                // 1: branch and bound against the per-read best (GLOBAL end)
    // extents the checked build tests every work item against (floats for
    // the arrays, records for results and keys)
    uint64_t n_events, n_r, n_fstore;
    int n_results, n_keys;
    int stall_handoff;             // tests only: the split kernel's stripes never publish their bottom rows
};

// Anchor-guided alignment (Sec. 2.4.2): one candidate's cost is the sum, in
// path order, of its pieces: gaps aligned by their own DTW (kind 0, result
// of work item idx) and runs of cells summed directly (kind 1: an anchor's
// diagonal, ev_step = r_step = 1; a gap with rows only, r_step = 0; a gap
// with columns only, ev_step = 0).
struct PieceRef {
    uint64_t ev;      // first event (index in the events array)
    uint64_t r;       // first expected value (index in r_all)
    uint32_t kind;    // 0: DTW gap, 1: run of cells
    uint32_t len;     // cells of a run
    uint32_t idx;     // work item of a DTW gap
    uint16_t ev_step, r_step;
};
static_assert(sizeof(PieceRef) == 32, "PieceRef layout");

struct CombineDesc {
    uint32_t first, count;  // pieces of the candidate in the plan array
    int32_t n, m;           // table size (N_Read = n)
    int32_t read;           // read slot for the per-read best
    int32_t w_report;       // half-width reported (-1 = no band)
};

// Host-side launchers (dtw_kernels.cu).
cudaError_t launch_expected_signal(const SigDesc *d, int n, const uint8_t *ref2bit, const float *pore,
                                   int k, float *r_all, cudaStream_t s);
cudaError_t launch_check_events(const float *ev, uint64_t n, int *err, cudaStream_t s);
// dependent: launched as a programmatic dependent of the stream's previous
// kernel (its blocks start as SM slots free up; see pdl_allow_next)
cudaError_t launch_stripe(int G, int HR, const StripeParams &p, int grid, int block, size_t smem,
                          cudaStream_t s, bool dependent = false);
cudaError_t launch_maybe_dependent(const void *fn, int grid, int block, size_t smem, cudaStream_t s, void **args,
                                   bool dependent);
int stripe_max_blocks_per_sm(int G, int HR, int block, size_t smem);
// the block-split kernel for long alignments (split_kernel.cu): four warps,
// HR rows per lane, one alignment per block
int split_max_blocks_per_sm(int HR);
size_t split_smem_bytes();
cudaError_t launch_split(int HR, const StripeParams &p, int grid, cudaStream_t s, bool dependent = false);
void *pick_stripe_et(int G, int HR, bool smem_ring);  // stripe_kernel_et.cu
cudaError_t launch_plain(const WorkDesc *w, const float *events, const float *r_all, float *diag,
                         rawalign_result_t *results, unsigned long long *best_keys, float b_match,
                         int end_free, cudaStream_t s);
cudaError_t launch_plain_byval(const WorkDesc &w, const float *events, const float *r_all, float *diag,
                               rawalign_result_t *results, unsigned long long *best_keys, float b_match,
                               int end_free, cudaStream_t s);
int host_band(int64_t n, int64_t m, int32_t band_w, int64_t num, int64_t den, int64_t *num_out,
              int64_t *den_out, int64_t *w_out, int32_t *w_report);
cudaError_t launch_combine(const CombineDesc *d, int n, const PieceRef *plan, const rawalign_result_t *pieces,
                           const float *events, const float *r_all, rawalign_result_t *results,
                           unsigned long long *best_keys, float b_match, cudaStream_t s);
cudaError_t launch_decide(rawalign_result_t *results, int n, const unsigned long long *best_keys,
                          const int *read_of, float thr, int final_decision, cudaStream_t s);

// Row-wise band DDA, r rows on: (Q0, R0) is floor and remainder of a band
// edge at some row (0 <= R0 < den), (q1, r1) = divmod(num, den) the step per
// row; (Q, R) receive the edge r rows further.  For r < 32 the carry
// floor((R0 + r r1) / den) is at most r, so a 5-bit binary search finds it.
__host__ __device__ __forceinline__ void row_dda(int Q0, int R0, int q1, int r1, int den, int r, int &Q, int &R)
{
    const long long x = (long long)R0 + (long long)r * r1;
    int c = 0;
#pragma unroll
    for (int bit = 16; bit >= 1; bit >>= 1)
        if ((long long)(c + bit) * den <= x)
            c += bit;
    Q = Q0 + r * q1 + c;
    R = (int)(x - (long long)c * den);
}

}  // namespace ra
