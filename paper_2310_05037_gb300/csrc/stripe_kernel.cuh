// stripe_kernel.cuh -- the hot loop of the path: banded DTW (Sec. 2.2, 2.4.3),
// end cell and score (Sec. 2.3) as a persistent striped wavefront.
//
// A group of G consecutive lanes owns one alignment at a time (32/G groups per
// warp, each on its own alignment; a group takes the next alignment from a
// global queue when it finishes).  Rows (read events) are cut into stripes of
// H = G*HR rows; lane t of stripe k owns rows i0..i0+HR-1 (i0 = k*H + t*HR)
// and keeps their events and previous-column DP values in registers.  Each
// step a lane computes one column j for its HR rows; lane t runs kLaneLag = 2
// columns behind lane t-1 and receives D(i0-1, j) from lane t-1's bottom row
// of two steps back by __shfl_up_sync, so that a lane's next two columns
// depend on nothing its neighbour computes meanwhile and can be computed as
// two interleaved dependency chains.  A lane does not wait for the stripe to finish: once it has
// passed the last in-band column of its rows it takes the same rows of the
// next stripe, dC steps later in its own schedule.  The first lane of a
// stripe reads its row above from a ring buffer that the last lane of the
// previous stripe wrote; the host chooses dC so that each value is written at
// least one step before it is read, a lane's windows never overlap, and the
// ring (>= dC + 2 entries) is never overwritten before it is read.
//
// Band (Sec. 2.4.3): out-of-band cells must act as +inf.  Instead of masking
// each result, the difference e - r of a row that is outside the band at the
// current column is replaced by +inf, so d = +inf and the cell is +inf
// whatever its neighbours are; this keeps the select off the dependent
// min -> add chain.  The rows in band at column j form an interval, found
// each step by a column-wise DDA (the last row whose band reaches j; the
// first row whose band has started is that one less a constant) and turned
// into a bit mask by one bmsk instruction.  Rows past the piece's last row
// hold event +inf, so the mask need not be clipped to them.  The host counts
// each piece's in-band cells exactly (a floor sum over its rows) and the
// kernel copies that count into the result; only the early-terminating
// instantiation, which may stop inside the band, counts the cells it computes
// (the population count of each step's mask).  The stripe change, which each
// lane makes alone while the rest of its warp waits, loads the lane's events
// and finds its last column in O(1).
// The cell itself is sub, min3 (one exact 3-input min), add, in that order;
// the subtractions of two rows issue as one packed f32x2 addition of -r.
#pragma once

#include <climits>
#include <cstdint>

#include "device_util.cuh"
#include "internal.cuh"

namespace ra {

// Per-group constants of the current alignment and per-lane band state that
// only stripe transitions read: kept in shared memory, not registers.
struct GroupCold {
    const float *ev;
    uint64_t fout_off;
    int nrows, row0, K, dC, den, q1, r1, qH, rH, qR, rR, t_last, r_last, cand, read, n_read, w_rep, fout_lo;
    int qdC, rdC, s_end, abort, written;  // abort/written: early termination
    float lb;                              // early termination: cost lower bound at the abort
};
struct LaneCold {
    unsigned long long cells;
    int loQ, loR, hiQ, hiR;
};

// Predicated store of one float to shared memory (no branch).
static __device__ __forceinline__ void st_shared_if(bool pred, float *addr, float v)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(addr);
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %0, 0;\n\t@p st.shared.f32 [%1], %2;\n\t}"
                 :: "r"((int)pred), "r"(a), "f"(v) : "memory");
}

template <int G, int HR, bool FREE_END, bool RING_SMEM, bool ET>
__global__ void __launch_bounds__(128) dtw_stripe_kernel(const StripeParams p)
{
    static_assert(HR < 32, "one bit of the band mask per row");
    constexpr int H = G * HR;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int BIGROW = 1 << 29;
    constexpr int GPB = 128 / G;  // groups per block
    extern __shared__ float smem[];
    __shared__ GroupCold gcs[GPB];
    __shared__ LaneCold lcs[128];
    const int lane = threadIdx.x & 31;
    const int t = lane & (G - 1);
    const int leader = lane & ~(G - 1);
    const int gw = (threadIdx.x >> 5) * (32 / G) + (lane / G);
    const int gglob = blockIdx.x * GPB + gw;
    // shared-memory rings start gw words apart modulo the bank count, so the
    // groups of a warp do not hit the same bank on the same step
    float *ring = RING_SMEM ? (smem + (size_t)gw * (p.ring_cap + 1)) : (p.gring + (size_t)gglob * p.ring_cap);
    const int rmask = p.ring_cap - 1;
    GroupCold *gc = gcs + gw;
    LaneCold *lc = lcs + threadIdx.x;
    pdl_allow_next();  // launch classes queue one after another in one stream

    // hot state
    const float *rr = p.r_all;
    int m = 1, s = 0, s_end = 0;
    int k = 0, j = 0, b = INT_MAX;
    // events in pairs: one packed subtraction (two f32 lanes, each rounded
    // as a scalar subtraction) gives two rows' e - r
    static_assert(HR % 2 == 0, "events are held in pairs");
    float2 ep[HR / 2];
    float D[HR];
#pragma unroll
    for (int r = 0; r < HR; ++r)
        D[r] = kInf;
#pragma unroll
    for (int q = 0; q < HR / 2; ++q)
        ep[q] = make_float2(0.f, 0.f);
    // column-wise DDA: rows in band at column j are [Aq, Bq] relative to
    // the lane's first row.  Only Bq (floor, remainder Br) is stepped: both
    // edges advance by the same (cq, cr) per column, so the lower edge is the
    // upper one less a constant (Dq, Dr), Aq = Bq - Dq - [Br < Dr]
    int Bq = -BIGROW, Br = 0, Dq = -2 * BIGROW, Dr = 0, cq = 0, cr = 0, cnum = 1;
    int nvalid = 0, colmax = -1;
    int loA = kBigCol;
    unsigned widA = 0;
    bool writer = false, holds_last = false;
    float diag = kInf, rnext = kInf, rnext2 = kInf, rjn = 0.f, rjn2 = 0.f;
    float b1 = kInf, b2 = kInf;  // this lane's bottom row one and two steps back
    float best = kInf;
    int bestj = -1;
    int lastLo = kBigCol, r_last = 0;
    float rowmin = kInf;  // early termination: smallest value of the stripe's last row so far
    unsigned ncells = 0;  // in-band cells since the last flush to lc->cells
    unsigned lastWid = 0;
    bool done = true, exhausted = false, have = false;

    // set-up of this lane's rows for stripe k: its events, and its last
    // column from the row-wise band DDA of its first row (kept in shared
    // memory), advanced to its last row in O(1).  The DP column and the
    // diagonal are not reset: a lane enters a stripe at least one column
    // before the first in-band column of its rows (the period dC guarantees
    // it), so its first step there has every row out of band, d = +inf, and
    // every value of the column becomes +inf whatever the old registers held.
    auto setup_stripe = [&]() {
        const int nrows = gc->nrows, K = gc->K, den = gc->den, q1 = gc->q1, r1 = gc->r1;
        const float *ev = gc->ev;
        const int i0 = k * H + t * HR;
        const int loQ = lc->loQ, loR = lc->loR, hiQ = lc->hiQ, hiR = lc->hiR;
        b = -1;
        nvalid = min(max(nrows - i0, 0), HR);
        // rows past the last one get event +inf, so they stay +inf whatever
        // the band mask says
        const float *evp = ev + i0;
        if (nvalid == HR) {
#pragma unroll
            for (int q = 0; q < HR / 2; ++q)
                ep[q] = make_float2(__ldg(evp + 2 * q), __ldg(evp + 2 * q + 1));
        } else {
#pragma unroll
            for (int q = 0; q < HR / 2; ++q)
                ep[q] = make_float2((2 * q < nvalid) ? __ldg(evp + 2 * q) : kInf,
                                    (2 * q + 1 < nvalid) ? __ldg(evp + 2 * q + 1) : kInf);
        }
        // the lane leaves the stripe after the band end of its last row
        // (clamped to the table); a full stripe's last row is HR - 1 rows
        // below the first, a step of (qR, rR) precomputed per alignment
        if (nvalid == HR) {
            int Qh = hiQ + gc->qR, Rh = hiR + gc->rR;
            if (Rh >= den)
                Qh += 1;
            b = Qh < m - 1 ? Qh : m - 1;
        } else if (nvalid > 0) {
            int Qh, Rh;
            row_dda(hiQ, hiR, q1, r1, den, nvalid - 1, Qh, Rh);
            b = Qh < m - 1 ? Qh : m - 1;
        }
        if (i0 != 0) {
            int Qa = loQ - q1, Ra = loR - r1;
            if (Ra < 0) {
                Qa -= 1;
                Ra += den;
            }
            int Qb = hiQ - q1, Rb = hiR - r1;
            if (Rb < 0) {
                Qb -= 1;
                Rb += den;
            }
            int la = Qa + (Ra > 0 ? 1 : 0);
            la = la < 0 ? 0 : la;
            const int ha = Qb < m - 1 ? Qb : m - 1;
            if (ha >= la) {
                loA = la;
                widA = (unsigned)(ha - la);
            } else {
                loA = kBigCol;
                widA = 0;
            }
        }
        writer = (t == G - 1) && (k < K - 1);
        holds_last = (k == K - 1) && (t == gc->t_last);
        if (ET)
            rowmin = kInf;
        if (FREE_END && holds_last) {
            r_last = gc->r_last;
            int Ql, Rl, Qh, Rh;
            row_dda(loQ, loR, q1, r1, den, r_last, Ql, Rl);
            row_dda(hiQ, hiR, q1, r1, den, r_last, Qh, Rh);
            int l = Ql + (Rl > 0 ? 1 : 0);
            l = l < 0 ? 0 : l;
            const int hh = Qh < m - 1 ? Qh : m - 1;
            lastLo = hh >= l ? l : kBigCol;
            lastWid = hh >= l ? (unsigned)(hh - l) : 0u;
        }
    };

    auto finish_lane = [&]() {
        b = INT_MAX;
        loA = kBigCol;
        writer = false;
        holds_last = false;
        nvalid = 0;
        colmax = -1;
    };

    // rows [loN, hiN) of the lane are in band at the current column: one
    // bit-field mask instruction (and the in-band cells of the step)
    auto band_mask = [&]() -> unsigned {
        const int Aq = Bq - Dq - (Br < Dr ? 1 : 0);
        const int loN = max(Aq, 0);
        // rows past the last one are +inf through their events; only the
        // early-terminating kernel, which counts the cells it computes,
        // clips the mask to them
        const int hiN = ET ? min(Bq + 1, nvalid) : Bq + 1;
        const int width = max(hiN - loN, 0);
        unsigned M;
        asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(M) : "r"(loN), "r"(width));
        M = ((unsigned)j <= (unsigned)colmax) ? M : 0u;
        if (ET)
            ncells += __popc(M);
        return M;
    };
    auto dda_step = [&]() {
        Bq += cq;
        Br += cr;
        if (Br >= cnum) {
            Bq += 1;
            Br -= cnum;
        }
    };
    auto last_row_value = [&](float v, int col) {
        // FREE end: running minimum of the last row (smallest column on
        // ties) and the frontier row kept for the next chunk (serving)
        if (v < best) {
            best = v;
            bestj = col;
        }
        if (p.fstore_out && (unsigned)(col - lastLo) <= lastWid)
            p.fstore_out[gc->fout_off + (unsigned)(col - gc->fout_lo)] = v;
    };
    auto wrap_if_needed = [&]() {
        if (j > b) {
            // this lane leaves stripe k
            if (holds_last) {
                float v = kInf;
                const int rl = gc->r_last;
#pragma unroll
                for (int r = 0; r < HR; ++r)
                    if (r == rl)
                        v = D[r];
                const int row_last = gc->row0 + gc->nrows - 1;
                float cost;
                int ei, ej;
                if (FREE_END) {
                    cost = best;
                    ej = bestj;
                    ei = bestj >= 0 ? row_last : -1;
                } else {
                    cost = (b == m - 1) ? v : kInf;
                    ei = row_last;
                    ej = m - 1;
                }
                const int cand = gc->cand, read = gc->read;
                const float sc = __fsub_rn(__fmul_rn(p.b_match, (float)gc->n_read), cost);
                rawalign_result_t *o = p.results + cand;
                o->read_id = (uint64_t)read;
                o->cand_idx = (uint32_t)cand;
                o->cost = cost;
                o->score = sc;
                o->end_i = ei;
                o->end_j = ej;
                o->w_eff = gc->w_rep;
                o->status = 0;
                atomicMax(p.best_keys + read, best_key(sc, cand));
                if (ET)
                    gc->written = 1;
            }
            if (ET && writer) {
                // branch and bound (Sec. 2.4.1): every path crosses the
                // stripe's last row and cells only add, so the final cost
                // is at least that row's smallest value; stop when even
                // that bound cannot beat the read's best score so far
                const unsigned long long key =
                    *(volatile const unsigned long long *)(p.best_keys + gc->read);
                const float best = key ? key_score(key) : -kInf;
                const float ub = __fsub_rn(__fmul_rn(p.b_match, (float)gc->n_read), rowmin);
                if (ub < best) {
                    gc->lb = rowmin;
                    gc->abort = 1;
                }
            }
            ++k;
            if (k < gc->K) {
                const int den = gc->den, qH = gc->qH, rH = gc->rH;
                int Q = lc->loQ + qH, R = lc->loR + rH;
                if (R >= den) {
                    Q += 1;
                    R -= den;
                }
                lc->loQ = Q;
                lc->loR = R;
                Q = lc->hiQ + qH;
                R = lc->hiR + rH;
                if (R >= den) {
                    Q += 1;
                    R -= den;
                }
                lc->hiQ = Q;
                lc->hiR = R;
                setup_stripe();
                j -= gc->dC;
                {
                    const int qdC = gc->qdC, rdC = gc->rdC;
                    Bq -= H + qdC;
                    Br -= rdC;
                    if (Br < 0) {
                        Bq -= 1;
                        Br += cnum;
                    }
                }
            } else {
                finish_lane();
            }
            // the lane's columns jumped: fetch the current and the next
            rnext = ring[j & rmask];
            rnext2 = ring[(j + 1) & rmask];
            rjn = __ldg(rr + min((unsigned)j, (unsigned)(m - 1)));
            rjn2 = __ldg(rr + min((unsigned)(j + 1), (unsigned)(m - 1)));
        }
    };
    // one column of the lane's rows
    auto single_step = [&](bool check) {
        ++j;
        dda_step();
        if (check)
            wrap_if_needed();
        const float rc = rnext;
        rnext = rnext2;
        rnext2 = ring[(j + 2) & rmask];
        const float sh = __shfl_up_sync(FULL, b2, 1, G);
        const float src = (t == 0) ? rc : sh;
        const float upv = ((unsigned)(j - loA) <= widA) ? src : kInf;
        const float rj = rjn;
        rjn = rjn2;
        rjn2 = __ldg(rr + min((unsigned)(j + 2), (unsigned)(m - 1)));
        const unsigned M = band_mask();
        float nn = upv, nw = diag, fv = kInf;
        const float2 nrj = make_float2(-rj, -rj);
        float2 t2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            // e - r (x + (-y) is x - y exactly), then +inf out of band
            if ((r & 1) == 0)
                t2 = __fadd2_rn(ep[r / 2], nrj);
            const float dt = ((M >> r) & 1u) ? ((r & 1) ? t2.y : t2.x) : kInf;
            const float v = __fadd_rn(fabsf(dt), min3f(nw, nn, D[r]));
            nw = D[r];
            D[r] = v;
            nn = v;
            if (FREE_END && r == r_last)
                fv = v;
        }
        diag = upv;
        const float bottom = D[HR - 1];
        b2 = b1;
        b1 = bottom;
        if (ET)
            rowmin = fminf(rowmin, bottom);
        if (FREE_END && holds_last)
            last_row_value(fv, j);
        if (RING_SMEM)
            st_shared_if(writer, ring + (j & rmask), bottom);
        else if (writer)
            ring[j & rmask] = bottom;
        __syncwarp();
    };
    // two columns of the lane's rows, as two interleaved chains
    auto pair_step = [&]() {
        ++j;
        dda_step();
        const int jA = j;
        const unsigned MA = band_mask();
        ++j;
        dda_step();
        const unsigned MB = band_mask();
        const float rcA = rnext, rcB = rnext2;
        rnext = ring[(j + 1) & rmask];
        rnext2 = ring[(j + 2) & rmask];
        const float shA = __shfl_up_sync(FULL, b2, 1, G);
        const float shB = __shfl_up_sync(FULL, b1, 1, G);
        const float upvA = ((unsigned)(jA - loA) <= widA) ? ((t == 0) ? rcA : shA) : kInf;
        const float upvB = ((unsigned)(j - loA) <= widA) ? ((t == 0) ? rcB : shB) : kInf;
        const float rjA = rjn, rjB = rjn2;
        rjn = __ldg(rr + min((unsigned)(j + 1), (unsigned)(m - 1)));
        rjn2 = __ldg(rr + min((unsigned)(j + 2), (unsigned)(m - 1)));
        float nnA = upvA, nwA = diag, nnB = upvB, nwB = upvA, fvA = kInf, fvB = kInf;
        const float2 nrjA = make_float2(-rjA, -rjA), nrjB = make_float2(-rjB, -rjB);
        float2 tA2 = make_float2(0.f, 0.f), tB2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            if ((r & 1) == 0) {
                tA2 = __fadd2_rn(ep[r / 2], nrjA);
                tB2 = __fadd2_rn(ep[r / 2], nrjB);
            }
            const float dA = ((MA >> r) & 1u) ? ((r & 1) ? tA2.y : tA2.x) : kInf;
            const float dB = ((MB >> r) & 1u) ? ((r & 1) ? tB2.y : tB2.x) : kInf;
            const float vA = __fadd_rn(fabsf(dA), min3f(nwA, nnA, D[r]));
            nwA = D[r];
            nnA = vA;
            const float vB = __fadd_rn(fabsf(dB), min3f(nwB, nnB, vA));
            nwB = vA;
            nnB = vB;
            D[r] = vB;
            if (FREE_END && r == r_last) {
                fvA = vA;
                fvB = vB;
            }
        }
        diag = upvB;
        b2 = nnA;
        b1 = nnB;
        if (ET)
            rowmin = fminf(rowmin, fminf(nnA, nnB));
        if (FREE_END && holds_last) {
            last_row_value(fvA, jA);
            last_row_value(fvB, j);
        }
        if (RING_SMEM) {
            st_shared_if(writer, ring + (jA & rmask), nnA);
            st_shared_if(writer, ring + (j & rmask), nnB);
        } else if (writer) {
            ring[jA & rmask] = nnA;
            ring[j & rmask] = nnB;
        }
        __syncwarp();
    };

    lc->cells = 0;
    while (true) {
        const bool need = done && !exhausted;
        if (__any_sync(FULL, need)) {
            if (ET) {
                // finished groups: add up the in-band cells their lanes
                // computed (a pruned alignment stops short of its band)
                unsigned long long c = lc->cells;
#pragma unroll
                for (int off = 1; off < G; off <<= 1)
                    c += __shfl_xor_sync(FULL, c, off);
                if (need && have && t == 0)
                    p.results[gc->cand].cells = c;
            }
            if (need)
                have = false;
            int tk = 0;
            if (need && t == 0)
                tk = atomicAdd(p.queue, 1);
            tk = __shfl_sync(FULL, tk, leader);
            __syncwarp();
            if (need) {
                if (tk >= p.n_work) {
                    exhausted = true;
                    rr = p.r_all;
                    m = 1;
                    k = 1;
                    finish_lane();
                } else {
                    const WorkDesc wd = p.work[tk];
                    bool skip_item = false;
#ifdef RAWALIGN_CHECKED
                    // checked build: every planned extent lies inside its
                    // array and the ring holds the item's period; a failing
                    // item is reported in err[0] (first one, + 1) and skipped
                    const bool bad =
                        wd.nrows <= 0 || wd.m <= 0 || wd.ev_off + (uint64_t)wd.nrows > p.n_events ||
                        wd.r_off + (uint64_t)wd.m > p.n_r || wd.cand < 0 || wd.cand >= p.n_results || wd.read < 0 ||
                        wd.read >= p.n_keys || (wd.s_end > 0 && wd.dC + 2 > p.ring_cap) ||
                        (wd.s_end > 0 && wd.fin_wid + kLaneLag * G + 4 > p.ring_cap) ||
                        (wd.fin_off != ~0ull && wd.fin_off + (uint64_t)wd.fin_wid + 1 > p.n_fstore) ||
                        (p.fstore_out && wd.fout_off > p.n_fstore);
                    if (bad) {
                        if (t == 0)
                            atomicCAS(p.err, 0, tk + 1);
                        have = false;
                        skip_item = true;
                    }
#endif
                    if (skip_item) {
                        // nothing runs for this item; the group takes the next
                    } else if (wd.s_end <= 0) {
                        // the band has no cell in the first row: nothing reaches the end
                        if (t == 0) {
                            rawalign_result_t *o = p.results + wd.cand;
                            o->read_id = (uint64_t)wd.read;
                            o->cand_idx = (uint32_t)wd.cand;
                            o->cost = kInf;
                            o->score = -kInf;
                            o->end_i = FREE_END ? -1 : wd.row0 + wd.nrows - 1;
                            o->end_j = FREE_END ? -1 : wd.m - 1;
                            o->w_eff = wd.w_report;
                            o->cells = 0;
                            o->status = 0;
                            atomicMax(p.best_keys + wd.read, best_key(-kInf, wd.cand));
                        }
                    } else {
                        have = true;
                        done = false;
                        const int K = (wd.nrows + H - 1) / H;
                        const long long num = wd.num, dn = wd.den, w = wd.w;
                        const long long Hn = (long long)H * num;
                        const int nl = wd.nrows - 1 - (K - 1) * H;
                        if (t == 0) {
                            gc->ev = p.events + wd.ev_off;
                            gc->fout_off = wd.fout_off;
                            gc->nrows = wd.nrows;
                            gc->row0 = wd.row0;
                            gc->K = K;
                            gc->dC = wd.dC;
                            gc->den = (int)dn;
                            gc->q1 = (int)(num / dn);
                            gc->r1 = (int)(num % dn);
                            gc->qH = (int)(Hn / dn);
                            gc->rH = (int)(Hn % dn);
                            gc->qR = (int)((HR - 1) * num / dn);
                            gc->rR = (int)((HR - 1) * num % dn);
                            if (!ET)
                                p.results[wd.cand].cells = wd.cells;
                            gc->t_last = nl / HR;
                            gc->r_last = nl % HR;
                            gc->cand = wd.cand;
                            gc->read = wd.read;
                            gc->n_read = wd.n_read;
                            gc->w_rep = wd.w_report;
                            gc->fout_lo = wd.fout_lo;
                            gc->s_end = wd.s_end;
                            gc->abort = 0;
                            gc->written = 0;
                        }
                        rr = p.r_all + wd.r_off;
                        m = wd.m;
                        s_end = wd.s_end;
                        const long long gi0 = (long long)wd.row0 + (long long)t * HR;
                        long long Q, R;
                        floordivmod(gi0 * num - w * dn, dn, Q, R);
                        lc->loQ = (int)Q;
                        lc->loR = (int)R;
                        floordivmod(gi0 * num + w * dn, dn, Q, R);
                        lc->hiQ = (int)Q;
                        lc->hiR = (int)R;
                        lc->cells = 0;
                        best = kInf;
                        bestj = -1;
                        k = 0;
                        j = wd.a0 - 1 - kLaneLag * t;  // first column of this lane
                        b1 = kInf;
                        b2 = kInf;
                        {
                            int Aq, Ar;
                            if (num == 0) {
                                Bq = BIGROW;
                                Aq = -BIGROW;
                                Br = Ar = cq = cr = 0;
                                cnum = 1;
                                colmax = (int)(w < wd.m - 1 ? w : wd.m - 1);
                                if (t == 0) {
                                    gc->qdC = 0;
                                    gc->rdC = 0;
                                }
                            } else {
                                // I_hi(j) = floor((j+w) den / num), I_lo(j) = ceil((j-w) den / num)
                                floordivmod(((long long)j + w) * dn, num, Q, R);
                                Bq = (int)(Q - gi0);
                                Br = (int)R;
                                floordivmod(((long long)j - w) * dn + num - 1, num, Q, R);
                                Aq = (int)(Q - gi0);
                                Ar = (int)R;
                                cq = (int)(dn / num);
                                cr = (int)(dn % num);
                                cnum = (int)num;
                                colmax = wd.m - 1;
                                if (t == 0) {
                                    const long long dd = (long long)wd.dC * dn;
                                    gc->qdC = (int)(dd / num);
                                    gc->rdC = (int)(dd % num);
                                }
                            }
                            // the loop pre-increments: step the column DDA back once
                            Bq -= cq;
                            Br -= cr;
                            if (Br < 0) {
                                Bq -= 1;
                                Br += cnum;
                            }
                            Aq -= cq;
                            Ar -= cr;
                            if (Ar < 0) {
                                Aq -= 1;
                                Ar += cnum;
                            }
                            Dq = Bq - Aq;
                            Dr = Br - Ar;
                            if (Dr < 0) {
                                Dr += cnum;
                                Dq -= 1;
                            }
                        }
                        --j;
                        s = 0;
                        // the row above row0 goes into the ring: a stored frontier,
                        // or the virtual cell D(-1,-1) = 0 that anchors the start
                        const bool virt = (wd.fin_off == ~0ull);
                        for (int x = t; x <= wd.fin_wid; x += G)
                            ring[(wd.fin_lo + x) & rmask] = virt ? 0.f : p.fstore[wd.fin_off + x];
                        __syncwarp(__activemask());
                        setup_stripe();
                        if (t == 0) {
                            loA = wd.fin_lo;
                            widA = (unsigned)wd.fin_wid;
                        }
                    }
                }
            }
            if (__all_sync(FULL, exhausted))
                break;
            __syncwarp();
            rnext = ring[(j + 1) & rmask];
            rnext2 = ring[(j + 2) & rmask];
            rjn = __ldg(rr + min((unsigned)(j + 1), (unsigned)(m - 1)));
            rjn2 = __ldg(rr + min((unsigned)(j + 2), (unsigned)(m - 1)));
            continue;
        }

        // steps until the first group of this warp finishes its alignment
        const int rem = done ? INT_MAX : s_end - s;
        // (early termination: at most 64 steps, then the group checks its
        // abort flag; otherwise at most 2^27 steps, so that the lane's cell
        // count, at most HR < 32 per step, fits in 32 bits until it is flushed)
        const int nstep = __reduce_min_sync(FULL, ET ? min(rem, 64) : min(rem, 1 << 27));
        // Runs of steps in which no lane of the warp changes stripe go two
        // columns at a time: the two columns are computed as two interleaved
        // chains (column j+1's row r needs column j's rows r-1 and r, and
        // the row above from the neighbour lane's bottom kLaneLag = 2 steps
        // back), so the schedulers see two independent dependency chains.
        // A step in which some lane changes stripe runs alone.
        int q = 0;
        while (q < nstep) {
            const int mine = (b == INT_MAX) ? INT_MAX : max(b - j, 0);
            const int run = __reduce_min_sync(FULL, min(mine, nstep - q));
            for (int x = 0; x + 1 < run; x += 2)
                pair_step();
            if (run & 1)
                single_step(false);
            q += run;
            if (q < nstep) {
                single_step(true);
                ++q;
            }
        }
        s += nstep;
        if (ET) {
            lc->cells += ncells;
            ncells = 0;
        }
        if (!done && s == s_end)
            done = true;
        if (ET) {
            __syncwarp();
            if (!done && gc->abort && !gc->written) {
                // pruned: the cost bound and the score bound take the result's
                // place, flagged; the cells computed so far are added at the
                // next acquisition
                done = true;
                if (t == 0) {
                    rawalign_result_t *o = p.results + gc->cand;
                    o->read_id = (uint64_t)gc->read;
                    o->cand_idx = (uint32_t)gc->cand;
                    o->cost = gc->lb;
                    o->score = __fsub_rn(__fmul_rn(p.b_match, (float)gc->n_read), gc->lb);
                    o->end_i = -1;
                    o->end_j = -1;
                    o->w_eff = gc->w_rep;
                    o->status = RA_RESULT_PRUNED;
                }
            }
        }
    }
    if (blockIdx.x == 0)
        pdl_wait_prev();  // complete after the launch class queued before this one
}

}  // namespace ra
