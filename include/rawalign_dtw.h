/*
 * rawalign_dtw.h -- C ABI of the GB300 library for the alignment step of
 * RawAlign (Lindegger et al., arXiv 2310.05037): banded dynamic time warping
 * of a read's normalised events against the expected signal of candidate
 * reference regions, the alignment score and the per-read mapping decision.
 *
 * What each call computes, and the passage that defines it:
 *   expected signal  r[j] = pore[k-mer at j]              Sup. A.1.1
 *   band             |j*den - i*num| <= w_eff*den         Sec. 2.4.3
 *   DTW              D(i,j) = |e_i - r_j| + min(NW,N,W)   Sec. 2.2
 *   cost             D(n-1,m-1), or min over the last row Sec. 2.2
 *   score            B_Match * N_Read - C_DTW             Sec. 2.3
 *   decision         best candidate mapped iff >= thr     Sec. 2.3, Sec. 3.1
 *
 * Conventions (all calls):
 *   - Every call returns a rawalign_status_t; nothing is thrown across the ABI.
 *   - Host pointers passed to submit_* / prepare_* are read before the call
 *     returns; the caller may free or reuse them afterwards.
 *   - Device memory: the library places everything in the caller's arena
 *     (config.arena_dev, arena_bytes), a block of device memory the caller
 *     owns and keeps alive until rawalign_dtw_destroy returns.  The library
 *     itself calls no cudaMalloc for device memory.  On the host it keeps
 *     pinned staging memory (cudaHostAlloc): a pool for serving's copies and
 *     one buffer, grown on demand, for each batch's planned records; events
 *     and results are copied from and to the caller's buffers directly.
 *     Result buffers belong to the caller.
 *   - All work runs on config.cuda_stream (a cudaStream_t; NULL = the legacy
 *     default stream) on the device current at create time.
 *   - One handle is not thread-safe: the caller serialises calls on it.
 *   - Floating point: IEEE binary32, round to nearest even, no FMA contraction,
 *     no flush-to-zero.  Results are bit-identical to a sequential evaluation
 *     of the definitions above.
 *   - Base codes: A=0, C=1, G=2, T=3; the reference is packed four bases per
 *     byte, base p in bits 2*(p%4) and 2*(p%4)+1 of byte p/4.  The k-mer index
 *     takes the first base as the most significant base-4 digit.
 */
#ifndef RAWALIGN_DTW_H
#define RAWALIGN_DTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rawalign_dtw rawalign_dtw_t; /* opaque handle */

/* Status codes.  -7 is not used: serving has no cancel call (a read is
 * stopped by closing it with an empty last chunk). */
typedef enum {
    RA_OK = 0,
    RA_EINVAL = -1,     /* invalid argument or input data */
    RA_ENOMEM = -2,     /* the arena (or the frontier store) is too small */
    RA_EAGAIN = -3,     /* admission refused for now: retry after polling */
    RA_ENOTREADY = -4,  /* poll: the ticket has not completed yet */
    RA_ETIMEDOUT = -5,  /* per-result status: a bounded wait between the warps that share one long
                           alignment gave up (the result is not valid) */
    RA_EDEVICE = -6     /* a CUDA call failed (checked build: a work item failed its checks) */
} rawalign_status_t;

enum { RA_END_GLOBAL = 0, RA_END_FREE = 1 };            /* end of the DTW */
enum { RA_UNMAPPED = 0, RA_MAPPED = 1, RA_PENDING = 2 };/* decision */
/* result.status besides RA_OK: the candidate was stopped by early
 * termination (config.early_termination); cost then holds a lower bound of
 * its cost, score the matching upper bound of its score, end = (-1,-1). */
enum { RA_RESULT_PRUNED = 1 };
/* kernel choice: AUTO picks a striped variant per alignment (and, when the
 * tuning file's "block_split X" is above 0, gives the alignments that would
 * take over X times the batch's balanced length on one warp to a block of
 * four warps, each computing every fourth stripe); PLAIN runs one
 * alignment per launch; SPLIT runs every alignment of a batch on a block of
 * four warps (tests); RA_KERNEL_VARIANT0 + v forces striped variant v for
 * every alignment (tuning and tests): v = 0..9 are (lanes per alignment, rows
 * per lane) = (32,16) (16,16) (32,8) (16,8) (8,8) (4,8) (16,24) (8,24) (32,24)
 * (4,24). */
enum { RA_KERNEL_AUTO = 0, RA_KERNEL_PLAIN = 1, RA_KERNEL_SPLIT = 2, RA_KERNEL_VARIANT0 = 16 };

typedef struct {
    int32_t k;                 /* k-mer length, 1..8; pore table has 4^k entries */
    float b_match;             /* B_Match (paper default 0.4) */
    float score_threshold;     /* Score_Threshold (paper default 20) */
    int32_t end_mode;          /* RA_END_GLOBAL or RA_END_FREE for batches */
    void *arena_dev;           /* caller-owned device memory, 256-byte aligned */
    uint64_t arena_bytes;
    void *cuda_stream;         /* cudaStream_t */
    int32_t max_candidates;    /* serving: candidates per read (<= 64) */
    int32_t kernel;            /* RA_KERNEL_* */
    int32_t serve_slots;       /* serving: reads admitted at once (0 = none) */
    int32_t serve_max_events;  /* serving: events per read at most */
    const char *autotune_path; /* optional tuning table written by the tuner */
    int32_t early_termination; /* 1: branch and bound in GLOBAL batches (Sec. 2.4.1), see prepare_batch */
    int32_t serve_early_reject;/* serving: 1 = decide RA_UNMAPPED as soon as no candidate can reach the
                                  threshold within serve_max_events events (see submit_chunk) */
    int32_t test_stall_handoff;/* tests only, 0 otherwise: in the block-split kernel no stripe publishes
                                  its bottom row, so the next stripe's bounded wait gives up and the
                                  alignment's result comes back with status RA_ETIMEDOUT */
    int32_t pad;
} rawalign_dtw_config_t;

/* One candidate region of the reference for one read (48 bytes). */
typedef struct {
    uint64_t read_id;          /* batch: index of the read in the batch */
    uint64_t ref_offset;       /* first base of the region in the reference */
    uint32_t ref_len_bases;    /* bases; m = ref_len_bases - k + 1 >= 1 */
    uint8_t strand;            /* 0 forward, 1 reverse complement of the region */
    uint8_t pad0[3];
    int32_t band_w;            /* band half-width in columns; < 0: no band */
    int32_t pad1;
    int64_t slope_num;         /* band slope num/den reference values per event; */
    int64_t slope_den;         /* 0,0 = (m-1)/(n-1), the paper's length ratio  */
} rawalign_candidate_t;

/* One anchor of a chain (Sec. 2.4.2), 12 bytes: read events q .. q+len-1
 * matched one to one, on the diagonal, to the expected values t .. t+len-1
 * of the candidate's region (columns counted from the region's first k-mer). */
typedef struct {
    uint32_t q;
    uint32_t t;
    uint32_t len;
} rawalign_anchor_t;

/* Result of one candidate (56 bytes). */
typedef struct {
    uint64_t read_id;
    uint32_t cand_idx;         /* index of the candidate in the submitted array */
    float cost;                /* C_DTW (+inf when no in-band path reaches the end) */
    float score;               /* B_Match * N_Read - C_DTW */
    int32_t end_i, end_j;      /* end cell of the alignment (-1,-1 if none) */
    int32_t w_eff;             /* band half-width used (-1 = no band) */
    uint64_t cells;            /* in-band cells computed */
    int32_t status;            /* RA_OK or a per-alignment error */
    int32_t is_best;           /* 1 for the read's best candidate */
    int32_t decision;          /* the read's decision: RA_MAPPED / RA_UNMAPPED / RA_PENDING */
    int32_t pad;
} rawalign_result_t;

/* Creates a handle.  pore_model: 4^k floats (host).  ref_2bit: the packed
 * reference (host, (ref_len+3)/4 bytes), copied into the arena once.
 * Errors: RA_EINVAL (bad config or pointers), RA_ENOMEM (arena too small),
 * RA_EDEVICE.  Cited: Sup. A.1.1 (pore model), Sec. 2.1.3 (candidates). */
int rawalign_dtw_create(const rawalign_dtw_config_t *config, const float *pore_model,
                        const uint8_t *ref_2bit, uint64_t ref_len, rawalign_dtw_t **out);

/* Aligns a batch: every candidate against its read (Sec. 2.2-2.4.3), scores it
 * (Sec. 2.3) and decides each read (best score >= threshold).  events: all
 * reads' events back to back (host floats); read_offsets: n_reads+1 offsets
 * into events; cands: n_cands candidates (host).  The work is queued on the
 * stream; the results come from rawalign_dtw_poll(ticket).  Errors: RA_EINVAL
 * (empty read, candidate outside the reference or shorter than k, read_id out
 * of range, bad slope), RA_ENOMEM / RA_EAGAIN (arena full: poll earlier
 * tickets first), RA_EDEVICE.  Non-finite events are detected on the device:
 * the poll of that ticket returns RA_EINVAL. */
int rawalign_dtw_submit_batch(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                              uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                              uint64_t *ticket);

/* Serving (Read-Until, Sec. 1 and Sec. 3.1): appends n_events events of read
 * read_id and advances every candidate's DTW by those rows, keeping each
 * candidate's last DTW row (its frontier) in the arena between chunks.  The
 * first chunk of a read gives its candidates (cands, n_cands <=
 * max_candidates), later chunks pass NULL, 0.  Each candidate uses its own
 * band slope (slope_num/den must be given) and the FREE end (min over the
 * last row).  last = 1 closes the read after this chunk.  Returns RA_EAGAIN
 * when no read slot or frontier memory is free (admission), RA_EINVAL for
 * unknown reads or bad data.  The chunk's results (one per candidate, with the
 * read's decision so far: RA_MAPPED, or RA_PENDING / RA_UNMAPPED when last)
 * come from rawalign_dtw_poll(ticket).  With config.serve_early_reject = 1 a
 * chunk that is not the last one is also decided RA_UNMAPPED when no
 * candidate can reach the threshold any more: for every candidate
 * fl(fl(B_Match * serve_max_events) - cost) < Score_Threshold.  Costs only
 * grow as rows are added (every term is non-negative and rounding is
 * monotone), so such a read can never be mapped; the caller stops it (an
 * empty chunk with last = 1 returns its slot and memory). */
int rawalign_dtw_submit_chunk(rawalign_dtw_t *h, uint64_t read_id, const float *events,
                              uint32_t n_events, const rawalign_candidate_t *cands,
                              uint32_t n_cands, int last, uint64_t *ticket);

/* Launches all chunks submitted since the last flush as one continuous batch
 * (serving); submit_chunk queues, flush runs.  Returns RA_OK when nothing is
 * pending. */
int rawalign_dtw_flush(rawalign_dtw_t *h);

/* One chunk of a batched serving submission (32 bytes): events
 * events[ev_offset .. ev_offset+n_events) of read read_id; on the read's first
 * chunk its candidates cands[cand_offset .. cand_offset+n_cands), later
 * chunks n_cands = 0; last = 1 closes the read after this chunk (an empty
 * chunk with last = 1 closes a read that the caller stops early). */
typedef struct {
    uint64_t read_id;
    uint64_t ev_offset;
    uint32_t n_events;
    uint32_t cand_offset;
    uint32_t n_cands;
    int32_t last;
} rawalign_chunk_t;

/* Serving, many reads per call (Sec. 3.1: every pore delivers its next chunk
 * at about the same time): the same as rawalign_dtw_submit_chunk for each of
 * chunks[0 .. n_chunks) in order, from one events array and one candidates
 * array (host memory, read before return).  tickets[i] and status[i] receive
 * each chunk's ticket (0 when refused) and status (RA_OK, RA_EAGAIN when the
 * read was not admitted: no read slot or arena memory free, RA_EINVAL for bad
 * data); a refused chunk changes nothing.  Returns RA_OK, or RA_EINVAL for
 * bad arguments (then nothing was queued). */
int rawalign_dtw_submit_chunks(rawalign_dtw_t *h, const rawalign_chunk_t *chunks, uint32_t n_chunks,
                               const float *events, const rawalign_candidate_t *cands, uint64_t *tickets,
                               int32_t *status);

/* Serving: waits up to timeout_us (0 = do not wait, < 0 = forever) until every
 * ticket of tickets[0 .. n_tickets) has completed, then writes their results
 * back to back, in ticket order, into out (host, cap entries) and each
 * ticket's result count into counts[i].  Returns RA_ENOTREADY when some ticket
 * is still running (nothing is consumed), RA_EINVAL for an unknown or repeated
 * ticket or when cap is too small (nothing is consumed), RA_EDEVICE.  Each
 * ticket is consumed once, as with rawalign_dtw_poll. */
int rawalign_dtw_poll_chunks(rawalign_dtw_t *h, const uint64_t *tickets, uint32_t n_tickets,
                             rawalign_result_t *out, uint32_t cap, uint32_t *counts, int64_t timeout_us);

/* Serving counters since the handle was created (or the last reset): flushes,
 * chunks and per-candidate pieces launched, in-band cells, host time spent
 * queueing and planning (submit and flush calls), and per-flush device
 * intervals measured with CUDA events: input copies, kernels, result copy. */
typedef struct {
    uint64_t flushes, chunks, pieces, cells;
    double host_submit_ms;     /* in submit_chunk / submit_chunks */
    double host_flush_ms;      /* in flush: planning, staging, launching */
    double h2d_ms;             /* device time of the input copies */
    double device_ms;          /* device time from the first kernel to the last */
    double d2h_ms;             /* device time of the result copy */
    double host_launch_ms;     /* the part of host_flush_ms spent in CUDA calls (copies, launches, events) */
    double host_plan_ms;       /* the part of host_flush_ms spent planning the pieces and packing the inputs */
    double host_reap_ms;       /* taking finished flushes' results (in flush and in the polls) */
} rawalign_dtw_serve_stats_t;
int rawalign_dtw_serve_stats(rawalign_dtw_t *h, rawalign_dtw_serve_stats_t *out, int reset);

/* Waits up to timeout_us microseconds (0 = do not wait, < 0 = wait forever)
 * for a ticket, then copies up to cap results into out (host) and sets n_out.
 * Returns RA_ENOTREADY if the ticket is still running, RA_EINVAL for an
 * unknown ticket, RA_EDEVICE on a device error.  A ticket can be polled once
 * successfully; its memory is recycled afterwards. */
int rawalign_dtw_poll(rawalign_dtw_t *h, uint64_t ticket, rawalign_result_t *out, uint32_t cap,
                      uint32_t *n_out, int64_t timeout_us);

/* Device-resident batches for repeated runs (the timing harness): prepare
 * copies the inputs into the arena and plans the work once; run re-executes
 * every step of the path on the resident inputs (as one CUDA graph) and
 * returns a ticket; release frees the batch.
 *
 * Early termination (config.early_termination = 1; batches with GLOBAL end,
 * not anchor-guided; Sec. 2.4.1): the first candidate of each read, in the
 * order given (callers sort candidates by chaining score, as the paper
 * does), is queued ahead of the others; every candidate stops after any
 * stripe (a block of rows) whose last row shows that even the smallest cost
 * still reachable cannot beat the read's best score found so far.  Stopped candidates come back with status RA_RESULT_PRUNED.  The
 * read's best candidate, its result and the read's decision are the same as
 * without early termination; which other candidates are stopped, and their
 * bounds, may vary from run to run.  Unstopped results are unchanged. */
int rawalign_dtw_prepare_batch(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                               uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                               uint64_t *batch);
int rawalign_dtw_run_batch(rawalign_dtw_t *h, uint64_t batch, uint64_t *ticket);
int rawalign_dtw_release_batch(rawalign_dtw_t *h, uint64_t batch);

/* Destroys the handle after waiting for all queued work.  The arena can be
 * freed by the caller afterwards. */
int rawalign_dtw_destroy(rawalign_dtw_t *h);

/* Library counters for the last run of a batch or serving launch (timing
 * harness): device time of the DTW kernel in ms, kernels launched, in-band
 * cells.  Returns RA_EINVAL for an unknown batch. */
typedef struct {
    double dtw_ms;             /* CUDA-event time of the DTW kernel(s) */
    double total_ms;           /* CUDA-event time of the whole path */
    uint64_t cells;            /* in-band cells of the batch */
    uint64_t slots;            /* lane-cell slots the plan occupies (>= cells) */
    uint32_t launches;         /* kernels launched by one run */
    uint32_t split;            /* alignments run on a block of four warps (the longest ones) */
    double host_plan_ms;       /* host time of prepare spent planning (checks, bands, schedules,
                                  launch classes, staging of the records), on the library's threads */
    double host_upload_ms;     /* host time of prepare from issuing the uploads to their end
                                  (prepare returns once its inputs are copied) */
} rawalign_dtw_stats_t;
int rawalign_dtw_batch_stats(rawalign_dtw_t *h, uint64_t batch, rawalign_dtw_stats_t *out);

/* One alignment that allocates nothing (the paper has no counterpart to this
 * call; it exists for deployment).  Some callers may not allocate device
 * memory at all: a plug-in inside a host program that owns the whole device
 * memory budget, or a control loop that must never call cudaMalloc because it
 * can wait on the device and stall the process's other streams.  Such a
 * caller passes device pointers it already owns: d_events (n_events floats),
 * d_ref_signal (m expected values, i.e. the pore means of the region's
 * k-mers) and d_result (one rawalign_result_t, written on the stream).  The
 * band, end mode and score follow the batch call; is_best and decision are
 * not written (one alignment, no per-read decision).
 * Memory: the working rows live in one fixed array inside the library,
 * 3 * (65536 + 2) floats plus 256 bytes (about 0.8 MB) on every GPU that
 * loads the library, held until the process exits.  n_events above 65536, or
 * m of 2^30 or more, is rejected with RA_EINVAL.  No cudaMalloc, cudaFree or
 * allocating library routine is called, and nothing is copied from host
 * memory: the work record travels as a kernel parameter, so the call does
 * not wait for earlier work on the stream.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current; make that
 * first call before any stream capture.  Every call uses the same array and
 * leaves its contents behind: calls whose work overlaps on the GPU (other
 * streams, or other host threads) race and must be serialised by the caller.
 * Returns RA_OK once the work is queued on cuda_stream (a cudaStream_t). */
int rawalign_dtw_align_noalloc(const float *d_events, uint32_t n_events, const float *d_ref_signal,
                               uint32_t m, int32_t band_w, int64_t slope_num, int64_t slope_den,
                               int32_t end_mode, float b_match, rawalign_result_t *d_result,
                               void *cuda_stream);

/* Relative cost of one lane-cell slot for each striped variant (n must be the
 * number of variants, 10: same order as RA_KERNEL_VARIANT0 + v).  The planner
 * picks, per alignment, the variant with the fewest cost-weighted slots; the
 * autotuner measures these costs.  config.autotune_path may name a text file
 * of "G HR cost" lines with the same numbers, and the planner's bin edges:
 * "ring_bins S" (S = 2, the default: launch classes bin ring sizes by powers
 * of four; S = 1: by powers of two, or by powers of four for a batch that
 * would otherwise need more than 64 launches), "latency_split X" (an alignment
 * longer than X times the batch's estimated length moves to a 32-lane
 * variant; 0 = automatic) and "block_split X" (see RA_KERNEL_AUTO; 0, the
 * default, = never); create returns RA_EINVAL for other values.  None of
 * these change results, only the launch plan.  Returns RA_EINVAL for a
 * wrong count or a non-positive cost. */
int rawalign_dtw_set_variant_costs(rawalign_dtw_t *h, const double *costs, uint32_t n);

/* Anchor-guided batch (Sec. 2.4.2): as rawalign_dtw_prepare_batch, but each
 * candidate c is aligned through its chain anchors[anchor_offsets[c] ..
 * anchor_offsets[c+1]) (host arrays, copied before return; anchor_offsets
 * has n_cands+1 entries; anchors may be NULL when every chain is empty).
 * Only the gaps between anchors are aligned:
 *   - the path runs from (0,0) to (n-1,m-1) through gap 0, anchor 1, gap 1,
 *     ..., anchor K, gap K; gap k spans the rows and columns between the end
 *     of anchor k and the start of anchor k+1;
 *   - a gap with rows and columns is a global DTW of its own, banded around
 *     the line through its corners with the candidate's half-width band_w
 *     (< 0: no band; the candidate's slope is not used);
 *   - a gap with rows only aligns its events to the previous anchor's last
 *     value (the first anchor's first value for gap 0), a gap with columns
 *     only its values to the previous anchor's last event (the first
 *     anchor's first event); an anchor adds |e - r| along its diagonal;
 *   - C = the pieces' costs added in path order, N_Read = n, end = (n-1,m-1),
 *     w_eff = band_w (-1 without a band), cells = DP cells of the gaps plus
 *     the cells of anchors and one-sided gaps.  The end is GLOBAL whatever
 *     the handle's end_mode.
 * The arena needs, beyond rawalign_dtw_batch_bytes, about 200 bytes per gap
 * and 32 per anchor.  Errors: as rawalign_dtw_prepare_batch, and RA_EINVAL
 * for a chain that is unsorted, overlapping, of zero length or outside the
 * n x m table. */
int rawalign_dtw_prepare_anchored(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                  uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                  const rawalign_anchor_t *anchors, const uint64_t *anchor_offsets,
                                  uint64_t *batch);

/* Prepares, runs and releases an anchor-guided batch in one call (see
 * rawalign_dtw_prepare_anchored); the results come from rawalign_dtw_poll. */
int rawalign_dtw_submit_anchored(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                 uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                 const rawalign_anchor_t *anchors, const uint64_t *anchor_offsets,
                                 uint64_t *ticket);

/* The optimal warping path of one alignment (the paper maps with the score
 * alone and writes the path only on request, Sec. 2.4).  events: the read's
 * n_events events (host); cand: one candidate (its read_id is only copied to
 * the result); end_mode: RA_END_GLOBAL or RA_END_FREE.  The DP is the same as
 * the batch kernels' (bit-identical cost); the path steps back from the end
 * cell to the neighbour that held the minimum, NW first, then N, then W on
 * ties.  path_i / path_j (host, cap >= n_events + m - 1 entries) receive the
 * path from (0,0) to the end cell, *path_len its length (0 when no in-band
 * path reaches the end); result receives cost, score, end, w_eff and cells
 * (is_best = 0, decision = RA_UNMAPPED: one candidate decides nothing).  The
 * call runs on the handle's stream and returns when done.  It takes from the
 * arena, until it returns, about 1 byte per in-band cell plus 30 bytes per
 * event and 12 per column.  Errors: RA_EINVAL (bad arguments, cap too small,
 * non-finite events), RA_ENOMEM (arena too small), RA_EDEVICE. */
int rawalign_dtw_traceback(rawalign_dtw_t *h, const float *events, uint32_t n_events,
                           const rawalign_candidate_t *cand, int32_t end_mode, int32_t *path_i,
                           int32_t *path_j, uint32_t cap, uint32_t *path_len, rawalign_result_t *result);

/* Bytes of arena a batch of this shape needs (planning aid for callers).
 * Not included: ring scratch for alignments whose band is too wide for the
 * shared-memory ring (about 2w+1 > 2000 columns).  Those take it from the
 * arena's remaining free space, up to (blocks x groups per block x ring
 * entries x 4) bytes per launch class; with less free space their class runs
 * on fewer blocks (slower, same results), and RA_ENOMEM comes back only when
 * not even one block's ring fits. */
uint64_t rawalign_dtw_batch_bytes(uint64_t n_events, uint32_t n_reads, uint32_t n_cands,
                                  uint64_t total_ref_values);

#ifdef __cplusplus
}
#endif
#endif
