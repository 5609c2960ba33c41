// dtw_kernels.cu -- sm_103a kernels of the RawAlign alignment path.
//
//   expected_signal_kernel   Sup. A.1.1: r[j] = pore[k-mer index at j]
//   check_events_kernel      input validation (non-finite events)
//   (dtw_stripe_kernel, the hot loop, is in stripe_kernel.cu)
//   dtw_plain_kernel         the same alignment by one CTA per launch, one
//                            anti-diagonal per __syncthreads (reference point)
//   combine_kernel           Sec. 2.4.2: anchor-guided cost from its pieces
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
#include "device_util.cuh"

namespace ra {

// ---------------------------------------------------------------------------
// a1: expected signal.  One warp per candidate region, one column per lane
// (coalesced stores).  The reference is read as 32-bit words of 16 bases
// (base q of a word in bits 2q, 2q+1), so the k bases from position p are
// bits 2(p mod 16) .. 2(p mod 16)+2k-1 of the word pair at p/16: one funnel
// shift.  That window holds the bases with the first one in the LOWEST
// digit.  Forward strand: the k-mer index wants the first base in the
// highest digit, so the digits are reversed (bit reverse, then swap the two
// bits of each digit).  Reverse strand: the k-mer at column j of the reverse
// complement starts from the base at end-1-j and walks backwards, so its
// index is exactly the complemented window at end-k-j (first base lowest).
// The pore table is staged in shared memory when it has at most 4096 entries.
// ---------------------------------------------------------------------------
static __device__ __forceinline__ unsigned reverse_digits(unsigned w, int k)
{
    const unsigned y = __brev(w) >> (32 - 2 * k);
    return ((y & 0x55555555u) << 1) | ((y >> 1) & 0x55555555u);
}

template <bool SMEM_TABLE>
__global__ void __launch_bounds__(256) expected_signal_kernel(const SigDesc *__restrict__ d, int n,
                                                              const uint32_t *__restrict__ ref32,
                                                              const float *__restrict__ pore, int k,
                                                              float *__restrict__ r_all)
{
    extern __shared__ float table_s[];
    const float *table = pore;
    if (SMEM_TABLE) {
        const int nt = 1 << (2 * k);
        for (int x = threadIdx.x; x < nt; x += blockDim.x)
            table_s[x] = __ldg(pore + x);
        __syncthreads();
        table = table_s;
    }
    const unsigned kmask = (1u << (2 * k)) - 1u;  // k <= 8
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n; c += nwarps) {
        const SigDesc sd = d[c];
        const int64_t m = (int64_t)sd.len - k + 1;
        float *out = r_all + sd.r_off;
        const uint64_t last = sd.ref_off + sd.len - (uint64_t)k;  // window start of the reverse strand's column 0
        for (int64_t j = lane; j < m; j += 32) {
            const uint64_t p = sd.strand ? last - (uint64_t)j : sd.ref_off + (uint64_t)j;
            const uint64_t wi = p >> 4;
            const unsigned lo = __ldg(ref32 + wi), hi = __ldg(ref32 + wi + 1);
            const unsigned win = __funnelshift_r(lo, hi, 2u * (unsigned)(p & 15)) & kmask;
            const unsigned idx = sd.strand ? (win ^ kmask) : reverse_digits(win, k);
            out[j] = table[idx];
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

// The body of the plain kernel: one CTA, one alignment, one anti-diagonal
// per __syncthreads (three rotating diagonal buffers of n+2 floats in diag).
static __device__ __forceinline__ void plain_body(const WorkDesc &wd, const float *__restrict__ events,
                                                  const float *__restrict__ r_all, float *diag,
                                                  rawalign_result_t *results, unsigned long long *best_keys,
                                                  float b_match, int end_free)
{
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

__global__ void __launch_bounds__(256) dtw_plain_kernel(const WorkDesc *__restrict__ wdp,
                                                        const float *__restrict__ events,
                                                        const float *__restrict__ r_all,
                                                        float *diag, rawalign_result_t *results,
                                                        unsigned long long *best_keys, float b_match,
                                                        int end_free)
{
    plain_body(*wdp, events, r_all, diag, results, best_keys, b_match, end_free);
}

// The same kernel with its work record passed by value (as a kernel
// parameter), for callers that keep no work record in device memory.
__global__ void __launch_bounds__(256) dtw_plain_kernel_byval(const WorkDesc wd, const float *__restrict__ events,
                                                              const float *__restrict__ r_all, float *diag,
                                                              rawalign_result_t *results,
                                                              unsigned long long *best_keys, float b_match,
                                                              int end_free)
{
    plain_body(wd, events, r_all, diag, results, best_keys, b_match, end_free);
}

// ---------------------------------------------------------------------------
// Anchor-guided alignment (Sec. 2.4.2): a candidate's cost is its pieces'
// costs added in path order, starting from the first piece; a run of cells
// (an anchor's diagonal, or a gap with rows or columns only) is summed from
// its first cell.  One thread per candidate keeps the order fixed; then the
// score (Sec. 2.3) and the per-read best key as in the DTW kernels.
// ---------------------------------------------------------------------------
__global__ void combine_kernel(const CombineDesc *__restrict__ desc, int n, const PieceRef *__restrict__ plan,
                               const rawalign_result_t *__restrict__ pieces, const float *__restrict__ events,
                               const float *__restrict__ r_all, rawalign_result_t *__restrict__ results,
                               unsigned long long *best_keys, float b_match)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const CombineDesc cd = desc[c];
        float C = 0.f;
        unsigned long long cells = 0;
        for (uint32_t p = 0; p < cd.count; ++p) {
            const PieceRef pr = plan[cd.first + p];
            float piece;
            if (pr.kind == 0) {
                piece = pieces[pr.idx].cost;
                cells += pieces[pr.idx].cells;
            } else {
                const float *e = events + pr.ev;
                const float *r = r_all + pr.r;
                piece = 0.f;
                for (uint32_t x = 0; x < pr.len; ++x) {
                    const float d = fabsf(__fsub_rn(e[x * pr.ev_step], r[x * pr.r_step]));
                    piece = (x == 0) ? d : __fadd_rn(piece, d);
                }
                cells += pr.len;
            }
            C = (p == 0) ? piece : __fadd_rn(C, piece);
        }
        const float sc = __fsub_rn(__fmul_rn(b_match, (float)cd.n), C);
        rawalign_result_t *o = results + c;
        o->read_id = (uint64_t)cd.read;
        o->cand_idx = (uint32_t)c;
        o->cost = C;
        o->score = sc;
        o->end_i = cd.n - 1;
        o->end_j = cd.m - 1;
        o->w_eff = cd.w_report;
        o->cells = cells;
        o->status = 0;
        atomicMax(best_keys + cd.read, best_key(sc, c));
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

// SMs of the current device (queried once per device): grid-stride launches
// are capped at a few resident blocks per SM.
static int device_sms()
{
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return 152;
    if (sms[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return 152;
        sms[dev] = n;
    }
    return sms[dev];
}
cudaError_t launch_expected_signal(const SigDesc *d, int n, const uint8_t *ref2bit, const float *pore,
                                   int k, float *r_all, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > device_sms() * 8)
        blocks = device_sms() * 8;
    const uint32_t *ref32 = (const uint32_t *)ref2bit;  // 256-byte aligned, padded by 16 bytes
    if (k <= 6) {
        expected_signal_kernel<true><<<blocks, 256, sizeof(float) << (2 * k), s>>>(d, n, ref32, pore, k, r_all);
    } else {
        expected_signal_kernel<false><<<blocks, 256, 0, s>>>(d, n, ref32, pore, k, r_all);
    }
    return cudaGetLastError();
}

cudaError_t launch_combine(const CombineDesc *d, int n, const PieceRef *plan, const rawalign_result_t *pieces,
                           const float *events, const float *r_all, rawalign_result_t *results,
                           unsigned long long *best_keys, float b_match, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int blocks = (n + 127) / 128;
    if (blocks > device_sms() * 16)
        blocks = device_sms() * 16;
    combine_kernel<<<blocks, 128, 0, s>>>(d, n, plan, pieces, events, r_all, results, best_keys, b_match);
    return cudaGetLastError();
}

cudaError_t launch_check_events(const float *ev, uint64_t n, int *err, cudaStream_t s)
{
    if (n == 0)
        return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > (uint64_t)device_sms() * 8)
        blocks = device_sms() * 8;
    check_events_kernel<<<(unsigned)blocks, 256, 0, s>>>(ev, n, err);
    return cudaGetLastError();
}

cudaError_t launch_plain(const WorkDesc *w, const float *events, const float *r_all, float *diag,
                         rawalign_result_t *results, unsigned long long *best_keys, float b_match,
                         int end_free, cudaStream_t s)
{
    dtw_plain_kernel<<<1, 256, 0, s>>>(w, events, r_all, diag, results, best_keys, b_match, end_free);
    return cudaGetLastError();
}

cudaError_t launch_plain_byval(const WorkDesc &w, const float *events, const float *r_all, float *diag,
                               rawalign_result_t *results, unsigned long long *best_keys, float b_match,
                               int end_free, cudaStream_t s)
{
    dtw_plain_kernel_byval<<<1, 256, 0, s>>>(w, events, r_all, diag, results, best_keys, b_match, end_free);
    return cudaGetLastError();
}

cudaError_t launch_decide(rawalign_result_t *results, int n, const unsigned long long *best_keys,
                          const int *read_of, float thr, int final_decision, cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    int blocks = (n + 255) / 256;
    if (blocks > device_sms() * 8)
        blocks = device_sms() * 8;
    decide_kernel<<<blocks, 256, 0, s>>>(results, n, best_keys, read_of, thr, final_decision);
    return cudaGetLastError();
}

}  // namespace ra
