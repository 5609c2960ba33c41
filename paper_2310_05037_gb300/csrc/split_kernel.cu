// split_kernel.cu -- one long alignment on a whole block: the striped
// wavefront of dtw_stripe_kernel (Sec. 2.2 recurrence, Sec. 2.4.3 band, end
// cell and score of Sec. 2.3), with the stripes of the alignment dealt round
// robin to the block's warps.
//
// A 32-lane warp computes stripe k (H = 32 * HR rows; lane t owns HR rows and
// runs one column behind lane t-1, taking lane t-1's bottom row by
// __shfl_up_sync) while the next warp computes stripe k+1 a little behind it.
// The bottom row of stripe k goes from the warp that writes it to the warp
// that reads it through a buffer in global memory (L2) that holds the whole
// row, with a counter in shared memory: the stripe it belongs to and the
// values written so far.  The reader waits until the value it needs is
// written (a bounded wait: about a third of a second of polling, after which
// the alignment stops and its result carries RA_ETIMEDOUT).  The writer never
// waits: each warp has two buffers and alternates between them from one of
// its stripes to the next, and stripe k+2W cannot start before stripe k+1 has
// finished reading stripe k (stripe k+1 must finish before stripe k+W can,
// which must finish before its warp starts stripe k+2W).  All waits are on
// warps of the same block, which are resident together.
//
// Used for the few alignments so long that one warp alone would outlast the
// rest of the batch (long reads): the planner gives each such alignment to a
// block of four warps, which brings its time down about fourfold.
#include <climits>
#include <cstdint>

#include "device_util.cuh"
#include "internal.cuh"

namespace ra {

constexpr int kSplitWarps = 4;       // warps per block = stripes in flight
constexpr int kSplitPublish = 8;     // the writer publishes its count every 8 values
constexpr int kSplitAhead = 4;       // the reader fetches its row-above values 4 columns ahead
constexpr unsigned kSpinLimit = 1u << 20;  // polls of a bounded wait (x 256 ns)

struct SplitShared {
    // per warp and buffer: (stripe << 32) | values of its bottom row written
    volatile unsigned long long tag[kSplitWarps][2];
    volatile int abort;  // a bounded wait gave up
    unsigned long long cells;
    int item;
};

// Bounded wait of one lane until buffer tag *t says stripe `stripe` has more
// than `idx` values (or the block aborts); false when it gave up.
static __device__ __forceinline__ bool wait_written(volatile unsigned long long *t, int stripe, int idx,
                                                    volatile int *abort)
{
    const unsigned long long want = ((unsigned long long)(unsigned)stripe << 32) | (unsigned)(idx + 1);
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        const unsigned long long v = *t;
        if ((v >> 32) == (unsigned)stripe && v >= want) {
            __threadfence_block();  // the values behind the counter are visible
            return true;
        }
        if (*abort)
            return false;
        if (it >= 32)
            __nanosleep(256);  // poll without sleeping first: the writer is usually a few steps away
    }
    return false;
}

template <int HR, bool FREE_END>
__global__ void __launch_bounds__(128, 4) dtw_split_kernel(const StripeParams p)
{
    constexpr int G = 32;
    constexpr int H = G * HR;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitShared &sh = *reinterpret_cast<SplitShared *>(smem_raw);
    const int t = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int wprev = (w + kSplitWarps - 1) % kSplitWarps;
    // this block's bottom-row buffers: [warp][2][ring_cap] floats
    float *gbuf = p.gring + (size_t)blockIdx.x * kSplitWarps * 2 * p.ring_cap;
    pdl_allow_next();  // launch classes queue one after another in one stream

    while (true) {
        if (threadIdx.x == 0) {
            sh.item = atomicAdd(p.queue, 1);
            sh.abort = 0;
            sh.cells = 0;
        }
        if (threadIdx.x < 2 * kSplitWarps)
            sh.tag[threadIdx.x >> 1][threadIdx.x & 1] = ~0ull;  // no stripe yet
        __syncthreads();
        const int item = sh.item;
        if (item >= p.n_work) {
            if (blockIdx.x == 0)
                pdl_wait_prev();  // complete after the launch class queued before this one
            return;
        }
        const WorkDesc wd = p.work[item];
        const int nrows = wd.nrows, m = wd.m;
        const long long num = wd.num, dn = wd.den, wb = wd.w;
        const int K = (nrows + H - 1) / H;
        const float *ev = p.events + wd.ev_off;
        const float *rr = p.r_all + wd.r_off;
        // band of row i: columns [lo(i), hi(i)] (Sec. 2.4.3), in 64-bit integers
        auto lo_of = [&](long long i) {
            long long q, r;
            floordivmod(i * num - wb * dn + dn - 1, dn, q, r);
            return q;
        };
        auto hi_of = [&](long long i) {
            long long q, r;
            floordivmod(i * num + wb * dn, dn, q, r);
            return q;
        };
        // first column of stripe k: one before its first row's band (not
        // before column -1: columns left of the table hold no cell)
        auto first_col = [&](int k) -> long long {
            const long long l = lo_of((long long)k * H);
            return (l > 0 ? l : 0) - 1;
        };
        // values the writer of stripe k produces: its last lane's columns
        // from (first column of the stripe) - 31 to the band end of its last row
        auto run_len = [&](int k) -> int {
            const long long first = first_col(k) - (G - 1);
            long long last = hi_of((long long)k * H + H - 1);
            last = last < m - 1 ? last : m - 1;
            return (int)(last - first + 1);
        };
        unsigned long long cells = 0;
        float best = kInf;
        int bestj = -1;
        bool aborted = false;
        for (int k = w; k < K && !aborted; k += kSplitWarps) {
            // ---- lane set-up for stripe k
            const int i0 = k * H + t * HR;
            const int nvalid = min(max(nrows - i0, 0), HR);
            float e[HR], D[HR];
#pragma unroll
            for (int r = 0; r < HR; ++r) {
                e[r] = (r < nvalid) ? __ldg(ev + i0 + r) : kInf;
                D[r] = kInf;
            }
            const long long cs = first_col(k);  // stripe's first column, fully out of band
            int j = (int)cs - t - 1;                             // the loop pre-increments
            int b = -1;
            if (nvalid > 0) {
                const long long hb = hi_of(i0 + nvalid - 1);
                b = (int)(hb < m - 1 ? hb : m - 1);
            }
            // rows of this lane in band at column j: [lo_idx, hi_idx] from
            // floor/ceil of (j +- w) den / num relative to i0, stepped per column
            int Bq, Br, Aq, Ar, cq = 0, cr = 0, cnum = 1;
            if (num == 0) {
                Bq = 1 << 29;
                Aq = -(1 << 29);
                Br = Ar = 0;
            } else {
                long long Q, R;
                floordivmod(((long long)j + wb) * dn, num, Q, R);
                Bq = (int)(Q - i0);
                Br = (int)R;
                floordivmod(((long long)j - wb) * dn + num - 1, num, Q, R);
                Aq = (int)(Q - i0);
                Ar = (int)R;
                cq = (int)(dn / num);
                cr = (int)(dn % num);
                cnum = (int)num;
            }
            const int colmax = num == 0 ? (int)(wb < m - 1 ? wb : m - 1) : m - 1;
            // the row above the lane's first row: its in-band columns
            int loA = kBigCol;
            unsigned widA = 0;
            if (i0 > 0 && i0 <= nrows) {
                long long la = lo_of(i0 - 1);
                la = la < 0 ? 0 : la;
                long long ha = hi_of(i0 - 1);
                ha = ha < m - 1 ? ha : m - 1;
                if (ha >= la) {
                    loA = (int)la;
                    widA = (unsigned)(ha - la);
                }
            }
            const bool writer = (t == G - 1) && (k < K - 1);
            const int wp0 = (int)cs - (G - 1);  // writer's first column
            const int rp0 = k > 0 ? (int)first_col(k - 1) - (G - 1) : 0;  // previous writer's
            const int last_row = nrows - 1;
            const bool holds_last = (k == K - 1) && (i0 <= last_row) && (last_row < i0 + HR);
            const int r_last = last_row - i0;
            int need = b - j;  // steps until this lane is past its last column
            int S = need;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                S = max(S, __shfl_xor_sync(FULL, S, off));
            // the buffer this stripe writes, and the one the previous stripe wrote
            const int wb_ = (k / kSplitWarps) & 1, rb_ = ((k - 1) / kSplitWarps) & 1;
            float *wbuf = gbuf + ((size_t)w * 2 + wb_) * p.ring_cap;
            const float *rbuf = gbuf + ((size_t)wprev * 2 + rb_) * p.ring_cap;
            volatile unsigned long long *wtag = &sh.tag[w][wb_];
            volatile unsigned long long *rtag = &sh.tag[wprev][rb_];
            if (t == G - 1 && k < K - 1) {
                // starting a new row in this buffer (its last reader has finished)
                *wtag = (unsigned long long)(unsigned)k << 32;
            }
            __syncwarp();
            // lane 0's row above, fetched kSplitAhead columns ahead: q[x] holds
            // the value of column j + 1 + x (0 for the virtual start, +inf
            // outside the row above's band)
            bool ok = true;
            auto fetch = [&](int col) -> float {
                if (k == 0)
                    return col == -1 ? 0.f : kInf;
                if ((unsigned)(col - loA) > widA)
                    return kInf;
                const int idx = col - rp0;
                if (!wait_written(rtag, k - 1, idx, &sh.abort))
                    ok = false;
                return rbuf[idx];
            };
            float q0 = kInf, q1 = kInf, q2 = kInf, q3 = kInf;
            if (t == 0) {
                q0 = fetch(j + 1);
                q1 = fetch(j + 2);
                q2 = fetch(j + 3);
                q3 = fetch(j + 4);
            }
            if (__any_sync(FULL, !ok)) {
                if (t == 0)
                    sh.abort = 1;
                aborted = true;
                break;
            }
            float diag = kInf, bottom = kInf, vlast = kInf;
            unsigned ncells = 0;
            // ---- the stripe, one column per step
            for (int s = 0; s < S; ++s) {
                ++j;
                Bq += cq;
                Br += cr;
                if (Br >= cnum) {
                    Bq += 1;
                    Br -= cnum;
                }
                Aq += cq;
                Ar += cr;
                if (Ar >= cnum) {
                    Aq += 1;
                    Ar -= cnum;
                }
                // lane 0's row above: the virtual cell D(-1,-1) = 0 for the
                // first stripe, else the previous stripe's bottom row
                const float rc = q0;
                if (t == 0) {
                    q0 = q1;
                    q1 = q2;
                    q2 = q3;
                    q3 = fetch(j + kSplitAhead);
                }
                if (__any_sync(FULL, !ok)) {
                    aborted = true;
                    break;
                }
                const float shv = __shfl_up_sync(FULL, bottom, 1);
                const float src = (t == 0) ? rc : shv;
                const float upv = (k == 0 && t == 0) ? src : (((unsigned)(j - loA) <= widA) ? src : kInf);
                const float rj = __ldg(rr + min((unsigned)j, (unsigned)(m - 1)));
                const int loN = max(Aq - 0, 0);
                const int hiN = min(Bq + 1, nvalid);
                const int width = max(hiN - loN, 0);
                unsigned M;
                asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(M) : "r"(loN), "r"(width));
                M = ((unsigned)j <= (unsigned)colmax && j <= b) ? M : 0u;
                ncells += __popc(M);
                float nn = upv, nw = diag, fv = kInf;
#pragma unroll
                for (int r = 0; r < HR; ++r) {
                    const float eg = ((M >> r) & 1u) ? e[r] : kInf;
                    const float v = __fadd_rn(fabsf(__fsub_rn(eg, rj)), min3f(nw, nn, D[r]));
                    nw = D[r];
                    D[r] = v;
                    nn = v;
                    if (FREE_END && r == r_last)
                        fv = v;
                }
                diag = upv;
                bottom = D[HR - 1];
                if (FREE_END && holds_last && j <= b && fv < best) {
                    best = fv;
                    bestj = j;
                }
                if (!FREE_END && holds_last && j == b) {
                    // the last row at its last in-band column (the corner when b = m-1)
#pragma unroll
                    for (int r = 0; r < HR; ++r)
                        if (r == r_last)
                            vlast = D[r];
                }
                if (writer) {
                    const int idx = j - wp0;
                    wbuf[idx] = bottom;
                    if (((idx + 1) % kSplitPublish) == 0 && !p.stall_handoff) {
                        __threadfence_block();
                        *wtag = ((unsigned long long)(unsigned)k << 32) | (unsigned)(idx + 1);
                    }
                }
            }
            if (aborted) {
                if (t == 0)
                    sh.abort = 1;
                break;
            }
            cells += ncells;
            // end of the stripe: publish the whole bottom row
            __threadfence_block();
            if (t == G - 1 && k < K - 1 && !p.stall_handoff)
                *wtag = ((unsigned long long)(unsigned)k << 32) | (unsigned)run_len(k);
            if (holds_last) {
                const float v = vlast;
                float cost;
                int ei, ej;
                if (FREE_END) {
                    cost = best;
                    ej = bestj;
                    ei = bestj >= 0 ? last_row : -1;
                } else {
                    cost = (b == m - 1) ? v : kInf;
                    ei = last_row;
                    ej = m - 1;
                }
                const float sc = __fsub_rn(__fmul_rn(p.b_match, (float)wd.n_read), cost);
                rawalign_result_t *o = p.results + wd.cand;
                o->read_id = (uint64_t)wd.read;
                o->cand_idx = (uint32_t)wd.cand;
                o->cost = cost;
                o->score = sc;
                o->end_i = ei;
                o->end_j = ej;
                o->w_eff = wd.w_report;
                o->status = 0;
                atomicMax(p.best_keys + wd.read, best_key(sc, wd.cand));
            }
            __syncwarp();
        }
        atomicAdd(&sh.cells, (unsigned long long)cells);
        __syncthreads();
        if (threadIdx.x == 0) {
            rawalign_result_t *o = p.results + wd.cand;
            o->cells = sh.cells;
            if (sh.abort) {
                o->read_id = (uint64_t)wd.read;
                o->cand_idx = (uint32_t)wd.cand;
                o->cost = kInf;
                o->score = -kInf;
                o->end_i = -1;
                o->end_j = -1;
                o->w_eff = wd.w_report;
                o->status = RA_ETIMEDOUT;
            }
        }
        __syncthreads();
    }
}

static void *pick_split(int HR, bool free_end)
{
    if (HR == 24)
        return free_end ? (void *)dtw_split_kernel<24, true> : (void *)dtw_split_kernel<24, false>;
    return nullptr;
}

size_t split_smem_bytes() { return sizeof(SplitShared); }

int split_max_blocks_per_sm(int HR)
{
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (HR == 24 && dev >= 0 && dev < 64 && cached[dev] > 0)
        return cached[dev];
    void *fn = pick_split(HR, false), *fn2 = pick_split(HR, true);
    if (!fn || !fn2)
        return 0;
    const int smem = (int)sizeof(SplitShared);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(fn2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 128, smem) != cudaSuccess)
        return 0;
    if (HR == 24 && dev >= 0 && dev < 64)
        cached[dev] = nb;
    return nb;
}

cudaError_t launch_split(int HR, const StripeParams &p, int grid, cudaStream_t s, bool dependent)
{
    void *fn = pick_split(HR, p.end_free != 0);
    if (!fn)
        return cudaErrorInvalidValue;
    const int smem = (int)sizeof(SplitShared);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    void *args[] = {(void *)&p};
    return launch_maybe_dependent(fn, grid, 128, smem, s, args, dependent);
}

}  // namespace ra
