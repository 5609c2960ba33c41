// dtw_kernels.cu -- sm_103a kernels of the RawAlign alignment path.
//
//   expected_signal_kernel   Sup. A.1.1: r[j] = pore[k-mer index at j]
//   check_events_kernel      input validation (non-finite events)
//   dtw_stripe_kernel        Sec. 2.2 + 2.4.3 + 2.3: banded DTW, end cell, score
//                            (persistent, striped wavefront; the hot loop)
//   dtw_plain_kernel         the same alignment by one CTA per launch, one
//                            anti-diagonal per __syncthreads (reference point)
//   decide_kernel            Sec. 2.3 / 3.1: best candidate per read, threshold
//
// Arithmetic follows the definitions in a fixed order: d = |e - r| (one
// subtraction), the minimum of the three neighbours (exact), one addition;
// the score is a product then a difference, each rounded once.  No FMA can
// form (there is no multiply-add in the recurrence and the score uses _rn
// intrinsics), and the library is built without fast-math, so results are
// bit-identical to a sequential FP32 evaluation.
#include <cstdint>
#include <cstdio>

#include "internal.cuh"

namespace ra {

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Order-preserving key: larger score first, then smaller candidate index.
__device__ __forceinline__ unsigned long long best_key(float score, int cand)
{
    unsigned u = __float_as_uint(score);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)cand);
}

__device__ __forceinline__ float key_score(unsigned long long key)
{
    unsigned u = (unsigned)(key >> 32);
    u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
    return __uint_as_float(u);
}

__device__ __forceinline__ void floordivmod(long long x, long long d, long long &q, long long &r)
{
    q = x / d;
    r = x - q * d;
    if (r < 0) {
        q -= 1;
        r += d;
    }
}

// ---------------------------------------------------------------------------
// a1: expected signal.  One warp per candidate region; each lane forms the
// k-mer index of its own columns from the packed reference.
// ---------------------------------------------------------------------------
__global__ void expected_signal_kernel(const SigDesc *__restrict__ d, int n,
                                       const uint8_t *__restrict__ ref2bit,
                                       const float *__restrict__ pore, int k,
                                       float *__restrict__ r_all)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += nwarps) {
        const SigDesc sd = d[c];
        const int64_t m = (int64_t)sd.len - k + 1;
        float *out = r_all + sd.r_off;
        for (int64_t j = lane; j < m; j += 32) {
            unsigned idx = 0;
            for (int q = 0; q < k; ++q) {
                uint64_t pos = sd.strand ? sd.ref_off + sd.len - 1 - (uint64_t)(j + q)
                                         : sd.ref_off + (uint64_t)(j + q);
                unsigned code = (__ldg(ref2bit + (pos >> 2)) >> ((pos & 3) * 2)) & 3u;
                if (sd.strand)
                    code = 3u - code;
                idx = idx * 4u + code;
            }
            out[j] = __ldg(pore + idx);
        }
    }
}

__global__ void check_events_kernel(const float *__restrict__ ev, uint64_t n, int *err)
{
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        bad |= !isfinite(ev[x]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
        atomicOr(err + 1, 1);
}

// ---------------------------------------------------------------------------
// a2-a6: the striped wavefront.
//
// A group of G consecutive lanes owns one alignment at a time (32/G groups per
// warp, each running its own alignment; groups take new work from a global
// queue as they finish).  Rows are cut into stripes of H = G*HR rows; lane t
// of a stripe owns rows i0 .. i0+HR-1 (i0 = k*H + t*HR) and keeps their
// previous-column DP values, events and band limits in registers.  Each step
// the lane computes one column j for its HR rows; lane t runs one column
// behind lane t-1 and receives D(i0-1, j) from lane t-1's bottom row by
// __shfl_up_sync.  Lanes do not wait for the whole stripe: when lane t has
// passed the last in-band column of its rows it moves on to the same rows of
// the next stripe (k+1), dC steps later than lane t's schedule in stripe k.
// The first lane of a stripe reads the row above it from a ring buffer that
// the last lane of the previous stripe wrote; dC is chosen (host) so that the
// ring is written one step before it is read and a lane's windows never
// overlap.  Cells outside the band (Sec. 2.4.3) are forced to +inf by a
// per-row column interval; the minimum over three neighbours is one 3-input
// min.f32 (exact), so each cell is sub, min3, add in a fixed order.
// ---------------------------------------------------------------------------
template <int G, int HR, bool FREE_END>
__global__ void __launch_bounds__(128) dtw_stripe_kernel(const StripeParams p)
{
    constexpr int H = G * HR;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int t = lane & (G - 1);
    const int leader = lane & ~(G - 1);
    const int gw = (threadIdx.x >> 5) * (32 / G) + (lane / G);
    const int gglob = blockIdx.x * (blockDim.x / G) + gw;
    float *ring = p.ring_in_smem ? (smem + (size_t)gw * p.ring_cap)
                                 : (p.gring + (size_t)gglob * p.ring_cap);
    const int rmask = p.ring_cap - 1;

    // alignment state (the same in every lane of a group)
    const float *ev = p.r_all;
    const float *rr = p.r_all;
    int m = 1, nrows = 0, row0 = 0, K = 0, dC = 0, s = 0, s_end = -1, cand = -1, read = 0;
    int n_read = 0, w_rep = 0, fout_lo = 0;
    uint64_t fout_off = 0;
    int den = 1, q1 = 0, r1 = 0, qH = 0, rH = 0;
    int t_last = 0, r_last = 0;
    // lane state
    int k = 0, j = 0, b = 0x7FFFFFFF, aW = 0;
    int loQ = 0, loR = 0, hiQ = 0, hiR = 0;
    int lo[HR];
    unsigned wid[HR];
    float e[HR], D[HR];
#pragma unroll
    for (int r = 0; r < HR; ++r) {
        lo[r] = kBigCol;
        wid[r] = 0;
        e[r] = 0.f;
        D[r] = kInf;
    }
    int loA = kBigCol;
    unsigned widA = 0;
    float diag = kInf, bottom = kInf, rnext = kInf;
    float best = kInf;
    int bestj = -1;
    int lastLo = kBigCol;
    unsigned lastWid = 0;
    unsigned long long cells = 0;
    bool done = true, exhausted = false, have = false;

    // per-stripe set-up of this lane's rows (DDA from the lane's first row)
    auto setup_stripe = [&]() {
        const int i0 = k * H + t * HR;
        int Ql = loQ, Rl = loR, Qh = hiQ, Rh = hiR;
        b = -1;
        aW = kBigCol;
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const int li = i0 + r;
            if (li < nrows) {
                int l = Ql + (Rl > 0 ? 1 : 0);
                l = l < 0 ? 0 : l;
                int hh = Qh < m - 1 ? Qh : m - 1;
                if (hh >= l) {
                    lo[r] = l;
                    wid[r] = (unsigned)(hh - l);
                    cells += (unsigned long long)(hh - l + 1);
                    if (aW == kBigCol)
                        aW = l;
                } else {
                    lo[r] = kBigCol;
                    wid[r] = 0;
                }
                b = hh;
                e[r] = __ldg(ev + li);
            } else {
                lo[r] = kBigCol;
                wid[r] = 0;
            }
            D[r] = kInf;
            Ql += q1;
            Rl += r1;
            if (Rl >= den) {
                Ql += 1;
                Rl -= den;
            }
            Qh += q1;
            Rh += r1;
            if (Rh >= den) {
                Qh += 1;
                Rh -= den;
            }
        }
        if (i0 == 0) {
            loA = -1;  // replaced below by the caller for stripe 0 lane 0
            widA = 0;
        } else {
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
            int ha = Qb < m - 1 ? Qb : m - 1;
            if (ha >= la) {
                loA = la;
                widA = (unsigned)(ha - la);
            } else {
                loA = kBigCol;
                widA = 0;
            }
        }
        diag = kInf;
        if (k == K - 1 && t == t_last) {
            // rows of this lane: the last row is r_last
            lastLo = kBigCol;
            lastWid = 0;
#pragma unroll
            for (int r = 0; r < HR; ++r)
                if (r == r_last) {
                    lastLo = lo[r];
                    lastWid = wid[r];
                }
        }
    };

    while (true) {
        // groups that finished an alignment and may get another one
        const bool need = done && !exhausted;
        if (__any_sync(FULL, need)) {
            // finished groups: add up the in-band cells of their lanes
            unsigned long long c = cells;
#pragma unroll
            for (int off = 1; off < G; off <<= 1)
                c += __shfl_xor_sync(FULL, c, off);
            if (need && have && t == 0)
                p.results[cand].cells = c;
            if (need)
                have = false;
            int tk = 0;
            if (need && t == 0)
                tk = atomicAdd(p.queue, 1);
            tk = __shfl_sync(FULL, tk, leader);
            if (need) {
                if (tk >= p.n_work) {
                    exhausted = true;
                    ev = p.r_all;
                    rr = p.r_all;
                    m = 1;
                    nrows = 0;
                    K = 0;
                    k = 1;
                    b = 0x7FFFFFFF;
                    loA = kBigCol;
#pragma unroll
                    for (int r = 0; r < HR; ++r)
                        lo[r] = kBigCol;
                } else {
                    const WorkDesc wd = p.work[tk];
                    cand = wd.cand;
                    read = wd.read;
                    n_read = wd.n_read;
                    w_rep = wd.w_report;
                    if (wd.s_end <= 0) {
                        // no in-band cell in the first row: nothing reaches the end
                        if (t == 0) {
                            rawalign_result_t *o = p.results + cand;
                            o->read_id = (uint64_t)read;
                            o->cand_idx = (uint32_t)cand;
                            o->cost = kInf;
                            o->score = -kInf;
                            o->end_i = FREE_END ? -1 : wd.row0 + wd.nrows - 1;
                            o->end_j = FREE_END ? -1 : wd.m - 1;
                            o->w_eff = w_rep;
                            o->cells = 0;
                            o->status = 0;
                            atomicMax(p.best_keys + read, best_key(-kInf, cand));
                        }
                    } else {
                        have = true;
                        done = false;
                        ev = p.events + wd.ev_off;
                        rr = p.r_all + wd.r_off;
                        m = wd.m;
                        nrows = wd.nrows;
                        row0 = wd.row0;
                        dC = wd.dC;
                        s_end = wd.s_end;
                        fout_lo = wd.fout_lo;
                        fout_off = wd.fout_off;
                        K = (nrows + H - 1) / H;
                        const long long num = wd.num, dn = wd.den, w = wd.w;
                        den = (int)dn;
                        q1 = (int)(num / dn);
                        r1 = (int)(num % dn);
                        const long long Hn = (long long)H * num;
                        qH = (int)(Hn / dn);
                        rH = (int)(Hn % dn);
                        const long long gi0 = (long long)row0 + (long long)t * HR;
                        long long Q, R;
                        floordivmod(gi0 * num - w * dn, dn, Q, R);
                        loQ = (int)Q;
                        loR = (int)R;
                        floordivmod(gi0 * num + w * dn, dn, Q, R);
                        hiQ = (int)Q;
                        hiR = (int)R;
                        const int nl = nrows - 1 - (K - 1) * H;  // last row within the last stripe
                        t_last = nl / HR;
                        r_last = nl % HR;
                        k = 0;
                        cells = 0;
                        best = kInf;
                        bestj = -1;
                        setup_stripe();
                        if (t == 0) {
                            loA = wd.fin_lo;
                            widA = (unsigned)wd.fin_wid;
                        }
                        j = wd.a0 - 2 - t;
                        s = 0;
                        // the row above row0 goes into the ring (frontier, or the
                        // virtual cell D(-1,-1) = 0 that starts the alignment)
                        const bool virt = (wd.fin_off == ~0ull);
                        for (int x = t; x <= wd.fin_wid; x += G)
                            ring[(wd.fin_lo + x) & rmask] = virt ? 0.f : p.fstore[wd.fin_off + x];
                    }
                }
            }
            if (__all_sync(FULL, exhausted))
                break;
            __syncwarp();
            rnext = ring[(j + 1) & rmask];
            continue;
        }

        ++s;
        ++j;
        if (j > b) {
            // this lane leaves stripe k
            if (k == K - 1 && t == t_last && !FREE_END) {
                float v = kInf;
#pragma unroll
                for (int r = 0; r < HR; ++r)
                    if (r == r_last)
                        v = D[r];
                const float cost = (b == m - 1) ? v : kInf;
                const float sc = __fsub_rn(__fmul_rn(p.b_match, (float)n_read), cost);
                rawalign_result_t *o = p.results + cand;
                o->read_id = (uint64_t)read;
                o->cand_idx = (uint32_t)cand;
                o->cost = cost;
                o->score = sc;
                o->end_i = row0 + nrows - 1;
                o->end_j = m - 1;
                o->w_eff = w_rep;
                o->status = 0;
                atomicMax(p.best_keys + read, best_key(sc, cand));
            }
            if (FREE_END && k == K - 1 && t == t_last) {
                const float sc = __fsub_rn(__fmul_rn(p.b_match, (float)n_read), best);
                rawalign_result_t *o = p.results + cand;
                o->read_id = (uint64_t)read;
                o->cand_idx = (uint32_t)cand;
                o->cost = best;
                o->score = sc;
                o->end_i = bestj >= 0 ? row0 + nrows - 1 : -1;
                o->end_j = bestj;
                o->w_eff = w_rep;
                o->status = 0;
                atomicMax(p.best_keys + read, best_key(sc, cand));
            }
            ++k;
            if (k < K) {
                loQ += qH;
                loR += rH;
                if (loR >= den) {
                    loQ += 1;
                    loR -= den;
                }
                hiQ += qH;
                hiR += rH;
                if (hiR >= den) {
                    hiQ += 1;
                    hiR -= den;
                }
                setup_stripe();
                j -= dC;
            } else {
                b = 0x7FFFFFFF;
                loA = kBigCol;
#pragma unroll
                for (int r = 0; r < HR; ++r)
                    lo[r] = kBigCol;
            }
            rnext = ring[j & rmask];
        }

        const float rc = rnext;
        rnext = ring[(j + 1) & rmask];
        const float sh = __shfl_up_sync(FULL, bottom, 1, G);
        const float src = (t == 0) ? rc : sh;
        const float upv = ((unsigned)(j - loA) <= widA) ? src : kInf;
        int jc = j < 0 ? 0 : j;
        jc = jc > m - 1 ? m - 1 : jc;
        const float rj = __ldg(rr + jc);
        float nn = upv, nw = diag;
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const float dd = fabsf(__fsub_rn(e[r], rj));
            const float mn = min3f(nw, nn, D[r]);
            float v = __fadd_rn(dd, mn);
            v = ((unsigned)(j - lo[r]) <= wid[r]) ? v : kInf;
            nw = D[r];
            D[r] = v;
            nn = v;
        }
        diag = upv;
        bottom = D[HR - 1];
        if (FREE_END && k == K - 1 && t == t_last) {
            float fv = kInf;
#pragma unroll
            for (int r = 0; r < HR; ++r)
                if (r == r_last)
                    fv = D[r];
            if (fv < best) {
                best = fv;
                bestj = j;
            }
            if (p.fstore_out && (unsigned)(j - lastLo) <= lastWid)
                p.fstore_out[fout_off + (unsigned)(j - fout_lo)] = fv;
        }
        if (t == G - 1 && k < K - 1 && j >= aW && j <= b)
            ring[j & rmask] = bottom;
        __syncwarp();
        if (s == s_end)
            done = true;
    }
}

// ---------------------------------------------------------------------------
// The plain kernel: one alignment per launch, one CTA, one anti-diagonal per
// step with the in-band rows of that anti-diagonal computed in parallel.
// Three anti-diagonal buffers (indexed by row+1) live in global scratch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long ceil_div_ll(long long a, long long b)
{
    long long q, r;
    floordivmod(a, b, q, r);
    return q + (r > 0 ? 1 : 0);
}

__device__ __forceinline__ long long floor_div_ll(long long a, long long b)
{
    long long q, r;
    floordivmod(a, b, q, r);
    return q;
}

__global__ void __launch_bounds__(256) dtw_plain_kernel(const WorkDesc *__restrict__ wdp,
                                                        const float *__restrict__ events,
                                                        const float *__restrict__ r_all,
                                                        float *diag, rawalign_result_t *results,
                                                        unsigned long long *best_keys, float b_match,
                                                        int end_free)
{
    const WorkDesc wd = *wdp;
    const int n = wd.nrows, m = wd.m;
    const long long num = wd.num, den = wd.den, w = wd.w, nd = num + den;
    const float *e = events + wd.ev_off;
    const float *r = r_all + wd.r_off;
    float *B[3] = {diag, diag + (n + 2), diag + 2 * (n + 2)};
    __shared__ float s_best;
    __shared__ int s_bestj;
    __shared__ unsigned long long s_cells;
    for (int x = threadIdx.x; x < 3 * (n + 2); x += blockDim.x)
        diag[x] = kInf;
    if (threadIdx.x == 0) {
        s_best = kInf;
        s_bestj = -1;
        s_cells = 0;
    }
    __syncthreads();
    unsigned long long cells = 0;
    for (int d = 0; d <= n + m - 2; ++d) {
        float *cur = B[d % 3];
        const float *p1 = B[(d + 2) % 3];
        const float *p2 = B[(d + 1) % 3];
        long long ilo = ceil_div_ll(((long long)d - w) * den, nd);
        long long ihi = floor_div_ll(((long long)d + w) * den, nd);
        ilo = ilo > d - m + 1 ? ilo : d - m + 1;
        ilo = ilo > 0 ? ilo : 0;
        ihi = ihi < n - 1 ? ihi : n - 1;
        ihi = ihi < d ? ihi : d;
        for (long long i = ilo - 1 + threadIdx.x; i <= ihi + 1; i += blockDim.x) {
            if (i < ilo || i > ihi) {
                if (i >= -1 && i <= n)
                    cur[i + 1] = kInf;
                continue;
            }
            const long long jj = d - i;
            const float dd = fabsf(__fsub_rn(e[i], r[jj]));
            const float mn = (i == 0 && jj == 0) ? 0.f : min3f(p2[i], p1[i], p1[i + 1]);
            const float v = __fadd_rn(dd, mn);
            cur[i + 1] = v;
            cells++;
            if (i == n - 1 && v < s_best) {
                s_best = v;
                s_bestj = (int)jj;
            }
        }
        __syncthreads();
    }
    atomicAdd(&s_cells, cells);
    __syncthreads();
    if (threadIdx.x == 0) {
        const int dl = n + m - 2;
        long long dev = (long long)(m - 1) * den - (long long)(n - 1) * num;
        dev = dev < 0 ? -dev : dev;
        const bool corner_in = dev <= w * den;
        float cost;
        int ei, ej;
        if (end_free) {
            cost = s_best;
            ej = s_bestj;
            ei = ej >= 0 ? n - 1 : -1;
        } else {
            cost = corner_in ? B[dl % 3][n] : kInf;
            ei = n - 1;
            ej = m - 1;
        }
        const float sc = __fsub_rn(__fmul_rn(b_match, (float)wd.n_read), cost);
        rawalign_result_t *o = results + wd.cand;
        o->read_id = (uint64_t)wd.read;
        o->cand_idx = (uint32_t)wd.cand;
        o->cost = cost;
        o->score = sc;
        o->end_i = ei;
        o->end_j = ej;
        o->w_eff = wd.w_report;
        o->cells = s_cells;
        o->status = 0;
        atomicMax(best_keys + wd.read, best_key(sc, wd.cand));
    }
}

// ---------------------------------------------------------------------------
// a7: per-read decision from the per-read best keys.
// ---------------------------------------------------------------------------
__global__ void decide_kernel(rawalign_result_t *res, int n, const unsigned long long *keys,
                              const int *read_of, float thr, int final_decision)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int rd = read_of[c];
        const unsigned long long key = keys[rd];
        const unsigned bc = 0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull);
        const float bs = key_score(key);
        res[c].is_best = (bc == res[c].cand_idx) ? 1 : 0;
        res[c].decision = (bs >= thr) ? RA_MAPPED : (final_decision ? RA_UNMAPPED : RA_PENDING);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_expected_signal(const SigDesc *d, int n, const uint8_t *ref2bit, const float *pore,
                                   int k, float *r_all, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > 152 * 16)
        blocks = 152 * 16;
    expected_signal_kernel<<<blocks, 256, 0, s>>>(d, n, ref2bit, pore, k, r_all);
    return cudaGetLastError();
}

cudaError_t launch_check_events(const float *ev, uint64_t n, int *err, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8)
        blocks = 152 * 8;
    check_events_kernel<<<(unsigned)blocks, 256, 0, s>>>(ev, n, err);
    return cudaGetLastError();
}

template <int G, int HR, bool F>
static void *stripe_fn()
{
    return (void *)dtw_stripe_kernel<G, HR, F>;
}

static void *pick_stripe(int G, int HR, bool freeend)
{
#define RA_PICK(g, h)                                                          \
    if (G == g && HR == h)                                                     \
        return freeend ? stripe_fn<g, h, true>() : stripe_fn<g, h, false>();
    RA_PICK(32, 8)
    RA_PICK(16, 8)
    RA_PICK(8, 8)
    RA_PICK(4, 8)
#undef RA_PICK
    return nullptr;
}

int stripe_max_blocks_per_sm(int G, int HR, int block, size_t smem)
{
    void *fn = pick_stripe(G, HR, false);
    if (!fn)
        return 0;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(pick_stripe(G, HR, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_stripe(int G, int HR, const StripeParams &p, int grid, int block, size_t smem,
                          cudaStream_t s)
{
    void *fn = pick_stripe(G, HR, p.end_free != 0);
    if (!fn)
        return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    void *args[] = {(void *)&p};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t launch_plain(const WorkDesc *w, const float *events, const float *r_all, float *diag,
                         rawalign_result_t *results, unsigned long long *best_keys, float b_match,
                         int end_free, cudaStream_t s)
{
    dtw_plain_kernel<<<1, 256, 0, s>>>(w, events, r_all, diag, results, best_keys, b_match, end_free);
    return cudaGetLastError();
}

cudaError_t launch_decide(rawalign_result_t *results, int n, const unsigned long long *best_keys,
                          const int *read_of, float thr, int final_decision, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 8)
        blocks = 152 * 8;
    decide_kernel<<<blocks, 256, 0, s>>>(results, n, best_keys, read_of, thr, final_decision);
    return cudaGetLastError();
}

}  // namespace ra
