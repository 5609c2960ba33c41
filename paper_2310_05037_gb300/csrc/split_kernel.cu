// split_kernel.cu -- one long alignment on a whole block: the striped
// wavefront of dtw_stripe_kernel (Sec. 2.2 recurrence, Sec. 2.4.3 band, end
// cell and score of Sec. 2.3), with the stripes of the alignment dealt round
// robin to the block's warps.
//
// A 32-lane warp computes stripe k (H = 32 * HR rows; lane t owns HR rows and
// runs one column behind lane t-1, taking lane t-1's bottom row by
// __shfl_up_sync) while the next warp computes stripe k+1 a little behind it:
// the bottom row of stripe k goes through a ring in shared memory from the
// warp that writes it to the warp that reads it.  Each ring is a
// single-producer single-consumer queue with two counters in shared memory:
// the values written and the values read.  The reader waits until the value
// it needs is written, the writer until its slot has been read; both waits
// are bounded (about a third of a second of polling), and one that gives up
// stops the alignment, whose result then carries RA_ETIMEDOUT.  All warps
// wait only on warps of their own block, which are resident together, so
// nothing waits on work that cannot run.
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
constexpr int kSplitCap = 2048;      // ring entries (power of two) per warp pair
constexpr int kSplitPublish = 8;     // the writer publishes its count every 8 values
constexpr unsigned kSpinLimit = 1u << 20;  // polls of a bounded wait (x 256 ns)

struct SplitShared {
    float ring[kSplitWarps][kSplitCap];
    volatile int written[kSplitWarps];  // values the warp has written into its ring
    volatile int read[kSplitWarps];     // values the next warp has read from that ring
    volatile int abort;                 // a bounded wait gave up
    unsigned long long cells;
    int item;
};

// Bounded wait of one lane until *ctr >= target (or the block aborts);
// false when it gave up.
static __device__ __forceinline__ bool wait_at_least(volatile int *ctr, int target, volatile int *abort)
{
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        if (*ctr >= target) {
            __threadfence_block();  // the values behind the counter are visible
            return true;
        }
        if (*abort)
            return false;
        __nanosleep(256);
    }
    return false;
}

template <int HR, bool FREE_END>
__global__ void __launch_bounds__(128, 4) dtw_split_kernel(const StripeParams p)
{
    constexpr int G = 32;
    constexpr int H = G * HR;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int CM = kSplitCap - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitShared &sh = *reinterpret_cast<SplitShared *>(smem_raw);
    const int t = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int wprev = (w + kSplitWarps - 1) % kSplitWarps;

    while (true) {
        if (threadIdx.x == 0) {
            sh.item = atomicAdd(p.queue, 1);
            sh.abort = 0;
            sh.cells = 0;
        }
        if (threadIdx.x < kSplitWarps) {
            sh.written[threadIdx.x] = 0;
            sh.read[threadIdx.x] = 0;
        }
        __syncthreads();
        const int item = sh.item;
        if (item >= p.n_work)
            return;
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
        int wbase = 0, rbase = 0;  // sequence numbers: this warp's ring, the previous warp's ring
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
            int avail = 0, room = 0;  // reader: values known written; writer: sequence known free
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
                float rc = kInf;
                bool ok = true;
                if (t == 0 && (unsigned)(j - loA) <= widA) {
                    const int seq = rbase + (j - rp0);
                    if (seq >= avail) {
                        ok = wait_at_least(&sh.written[wprev], seq + 1, &sh.abort);
                        avail = sh.written[wprev];
                    }
                    rc = sh.ring[wprev][seq & CM];
                }
                if (t == 0 && k == 0)
                    rc = (j == -1) ? 0.f : kInf;
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
                    const int seq = wbase + (j - wp0);
                    if (seq >= room) {
                        ok = wait_at_least(&sh.read[w], seq + 1 - kSplitCap, &sh.abort);
                        room = sh.read[w] + kSplitCap;
                    }
                    sh.ring[w][seq & CM] = bottom;
                    if (((seq + 1) % kSplitPublish) == 0 && !p.stall_handoff) {
                        __threadfence_block();
                        sh.written[w] = seq + 1;
                    }
                }
                if (__any_sync(FULL, !ok)) {
                    aborted = true;
                    break;
                }
                if (t == 0 && k > 0 && (((j - rp0 + 1) % kSplitPublish) == 0)) {
                    // the values up to this column are read
                    __threadfence_block();
                    sh.read[wprev] = rbase + (j - rp0) + 1;
                }
            }
            if (aborted) {
                if (t == 0)
                    sh.abort = 1;
                break;
            }
            cells += ncells;
            // end of the stripe: publish everything written and read
            const int wrote = k < K - 1 ? run_len(k) : 0;
            const int readn = k > 0 ? run_len(k - 1) : 0;
            __threadfence_block();
            if (t == G - 1 && k < K - 1 && !p.stall_handoff)
                sh.written[w] = wbase + wrote;
            if (t == 0 && k > 0)
                sh.read[wprev] = rbase + readn;
            wbase += wrote;
            rbase += readn;
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

cudaError_t launch_split(int HR, const StripeParams &p, int grid, cudaStream_t s)
{
    void *fn = pick_split(HR, p.end_free != 0);
    if (!fn)
        return cudaErrorInvalidValue;
    const int smem = (int)sizeof(SplitShared);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    void *args[] = {(void *)&p};
    return cudaLaunchKernel(fn, dim3(grid), dim3(128), args, smem, s);
}

}  // namespace ra
