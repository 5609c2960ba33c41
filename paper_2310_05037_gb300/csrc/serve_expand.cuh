// serve_expand.cuh -- the work record of one serving piece (one chunk of one
// read against one candidate), computed from the candidate's carried state:
// the band (Sec. 2.4.3), the stripe schedule, the exact in-band cell count and
// the frontier rows (the DP row that the next chunk resumes from, Sec. 2.2).
//
// The same code runs on the host (the planner tests compare it with the batch
// planner's schedule and cell count) and on the device, where one thread per
// piece builds each flush's work records, so the host sends one record per
// chunk instead of one per piece.
#pragma once

#include <cstdint>

#include "internal.cuh"

namespace ra {

// A candidate of an admitted read: fixed at admission, except the frontier
// fields (cur, fr_lo, fr_wid, dead), which each chunk advances.
struct ServeCandDev {
    uint64_t r_off;       // floats from the arena base: expected signal (m values)
    uint64_t fr_off[2];   // floats from the arena base: the two frontier rows
    int64_t num, den;     // band slope (reference values per event)
    int64_t per;          // den / gcd(num, den): rows where row num / den is whole
    int64_t hi_row;       // first row whose band reaches the last column
    int32_t m, w, w_report;
    int32_t G, HR;        // lane layout of the candidate's striped variant
    int32_t dC;           // stripe period of that variant
    int32_t cls;          // launch bucket: variant * kServeCaps + ring size index
    int32_t cur;          // frontier row holding the last processed row
    int32_t fr_lo, fr_wid;  // its band: first column, width - 1
    int32_t dead;         // the band has left the table: no cell any more
    int32_t pad;
};
static_assert(sizeof(ServeCandDev) == 104, "ServeCandDev layout");

// One chunk of one read in a flush.
struct ServeChunkDev {
    uint64_t ev_off;      // index of the chunk's first event in the flush's events
    uint64_t cand_off;    // bytes from the arena base to the read's candidate records
    uint32_t n_cands;     // pieces of the chunk (0: a close-only chunk)
    uint32_t first_piece; // result slot of its first piece
    int32_t row0, nrows;  // rows (events) of the read the chunk covers
};
static_assert(sizeof(ServeChunkDev) == 32, "ServeChunkDev layout");

constexpr int kServeCaps = 24;  // ring size indices per variant (128 << i)

__host__ __device__ inline int64_t hd_fdiv(int64_t a, int64_t b)
{
    const int64_t q = a / b, r = a % b;
    return (r != 0 && ((r < 0) != (b < 0))) ? q - 1 : q;
}
__host__ __device__ inline int64_t hd_cdiv(int64_t a, int64_t b) { return -hd_fdiv(-a, b); }

// sum_{i=0}^{n-1} floor((a i + b) / c), a, b >= 0, c > 0, by the Euclidean
// reduction of the floor sum; every intermediate stays below 2^63 for the
// serving limits (rows < 2^31, slopes and widths < 2^30).
__host__ __device__ inline uint64_t hd_floor_sum(uint64_t n, uint64_t c, uint64_t a, uint64_t b)
{
    uint64_t acc = 0;
    while (n > 0) {
        if (a >= c) {
            acc += (n * (n - 1) / 2) * (a / c);
            a %= c;
        }
        if (b >= c) {
            acc += n * (b / c);
            b %= c;
        }
        const uint64_t y = a * n + b;
        if (y < c)
            break;
        n = y / c;
        b = y - n * c;
        const uint64_t t = a;
        a = c;
        c = t;
    }
    return acc;
}

// The band's first and last column in row i, clipped to the table.
__host__ __device__ inline int64_t hd_lo(const ServeCandDev &s, int64_t i)
{
    const int64_t v = hd_cdiv(i * s.num - (int64_t)s.w * s.den, s.den);
    return v > 0 ? v : 0;
}
__host__ __device__ inline int64_t hd_hi(const ServeCandDev &s, int64_t i)
{
    const int64_t v = hd_fdiv(i * s.num + (int64_t)s.w * s.den, s.den);
    return v < s.m - 1 ? v : s.m - 1;
}

// In-band cells of rows [r0, r1), exactly (the same sums as the batch
// planner's band_cells: 2w per row plus the whole-slope rows away from the
// table's edges, floor sums near them).
__host__ __device__ inline uint64_t hd_band_cells(const ServeCandDev &s, int64_t r0, int64_t r1)
{
    if (r1 <= r0)
        return 0;
    const int64_t num = s.num, den = s.den, w = s.w, m = s.m;
    if (num == 0) {
        const int64_t hi = w < m - 1 ? w : m - 1;
        return (uint64_t)(r1 - r0) * (uint64_t)(hi + 1);
    }
    if (w >= m - 1 && r0 >= 0 && (r1 - 1) * num <= w * den)
        return (uint64_t)(r1 - r0) * (uint64_t)m;
    const int64_t rmax = hd_fdiv((m - 1 + w) * den, num) + 1;
    if (r1 > rmax)
        r1 = rmax;
    if (r1 <= r0)
        return 0;
    if (s.per > 0 && r1 <= s.hi_row && r0 * num >= w * den - den + 1) {
        const uint64_t whole = (uint64_t)(hd_fdiv(r1 - 1, s.per) - hd_fdiv(r0 - 1, s.per));
        return (uint64_t)(r1 - r0) * (uint64_t)(2 * w) + whole;
    }
    const uint64_t wd = (uint64_t)(w * den);
    int64_t i_h = hd_cdiv((m - 1 - w) * den, num);
    if (i_h < 0)
        i_h = 0;
    uint64_t s_hi = 0;
    {
        const int64_t a = r0, e = r1 < (r0 > i_h ? r0 : i_h) ? r1 : (r0 > i_h ? r0 : i_h);
        if (e > a)
            s_hi += hd_floor_sum((uint64_t)e, (uint64_t)den, (uint64_t)num, wd) -
                    hd_floor_sum((uint64_t)a, (uint64_t)den, (uint64_t)num, wd);
        const int64_t a2 = r0 > i_h ? r0 : i_h;
        if (r1 > a2)
            s_hi += (uint64_t)(r1 - a2) * (uint64_t)(m - 1);
    }
    const int64_t i_l = hd_fdiv(w * den, num) + 1;
    uint64_t s_lo = 0;
    {
        const int64_t a = r0 > i_l ? r0 : i_l;
        if (r1 > a) {
            const uint64_t off = (uint64_t)(i_l * num - w * den + den - 1);
            s_lo = hd_floor_sum((uint64_t)(r1 - i_l), (uint64_t)den, (uint64_t)num, off) -
                   hd_floor_sum((uint64_t)(a - i_l), (uint64_t)den, (uint64_t)num, off);
        }
    }
    return s_hi - s_lo + (uint64_t)(r1 - r0);
}

// The work record of piece k of chunk c (result slot ch.first_piece + k, read
// slot c of the flush), and the candidate's state advanced past the chunk: a
// live candidate switches frontier rows; the last row's band becomes the
// stored frontier, or the candidate is dead once its band has no cell there.
__host__ __device__ inline void serve_piece(const ServeChunkDev &ch, uint32_t c, uint32_t k, ServeCandDev &s,
                                            WorkDesc &wd)
{
    const int64_t row0 = ch.row0, nrows = ch.nrows, last = row0 + nrows - 1;
    wd.ev_off = ch.ev_off;
    wd.r_off = s.r_off;
    wd.num = s.num;
    wd.den = s.den;
    wd.row0 = ch.row0;
    wd.nrows = ch.nrows;
    wd.m = s.m;
    wd.w = s.w;
    wd.cand = (int32_t)(ch.first_piece + k);
    wd.read = (int32_t)c;
    wd.n_read = (int32_t)(row0 + nrows);
    wd.w_report = s.w_report;
    if (row0 == 0) {
        wd.fin_off = ~0ull;
        wd.fin_lo = -1;
        wd.fin_wid = 0;
    } else {
        wd.fin_off = s.fr_off[s.cur];
        wd.fin_lo = s.fr_lo;
        wd.fin_wid = s.fr_wid;
    }
    wd.fout_off = s.fr_off[1 - s.cur];
    const int64_t lo_last = hd_lo(s, last), hi_last = hd_hi(s, last);
    wd.fout_lo = (int32_t)lo_last;
    // stripe schedule (the batch planner's closed form)
    wd.dC = 0;
    wd.a0 = 0;
    wd.s_end = 0;
    if (!s.dead) {
        const int64_t a0 = hd_lo(s, row0);
        wd.a0 = (int32_t)a0;
        if (a0 <= s.m - 1) {
            const int64_t H = (int64_t)s.G * s.HR, K = (nrows + H - 1) / H;
            const int64_t t_last = (nrows - 1 - (K - 1) * H) / s.HR;
            const int64_t se = hi_last - a0 + 3 + (int64_t)kLaneLag * t_last + (K - 1) * (int64_t)s.dC;
            wd.dC = s.dC;
            wd.s_end = (int32_t)(se > 1 ? se : 1);
        }
    }
    wd.cells = wd.s_end > 0 ? hd_band_cells(s, row0, row0 + nrows) : 0;
    // advance the candidate past this chunk
    if (!s.dead) {
        s.cur = 1 - s.cur;
        if (hi_last >= lo_last && wd.s_end > 0) {
            s.fr_lo = (int32_t)lo_last;
            s.fr_wid = (int32_t)(hi_last - lo_last);
        } else {
            s.dead = 1;
        }
    }
}

// Launchers (serve_kernels.cu): copy the records of newly admitted candidates
// to their places in the arena (byte offsets from its base); build every
// piece of a flush (one block per chunk), placing each work record in its
// launch class's range (class q = map[cls]: base[q] + the class's running
// count) and noting its chunk for the decision.
cudaError_t launch_serve_init(char *arena, const uint64_t *off, const ServeCandDev *recs, int n, cudaStream_t s);
cudaError_t launch_serve_expand(const ServeChunkDev *chunks, int n_chunks, char *arena, const int *cls_map,
                                const int *cls_base, int *cls_fill, WorkDesc *work, int *read_of, cudaStream_t s);

}  // namespace ra
