// traceback.cu -- the optimal warping path of one alignment.  RawAlign maps
// with the score alone and writes the path only when asked (Sec. 2.4); this
// entry point is that option.  One CTA runs the DP one anti-diagonal at a time
// (the same cell arithmetic as every kernel of the library: d = |e - r|, the
// exact 3-way min, one addition) and records for each in-band cell which
// neighbour held the minimum: NW first, then N, then W on ties.  Thread 0 then
// walks back from the end cell to (0,0).
#include "engine.h"
#include "device_util.cuh"

namespace ra {

enum : uint8_t { kDirStart = 0, kDirNW = 1, kDirN = 2, kDirW = 3 };

static __device__ __forceinline__ long long floor_div_tb(long long a, long long b)
{
    long long q, r;
    floordivmod(a, b, q, r);
    return q;
}

// Directions are stored row by row over each row's band: cell (i, j) at
// row_off[i] + j - row_lo[i].  diag: 3 anti-diagonal buffers of n + 2 floats.
__global__ void __launch_bounds__(256) dtw_trace_kernel(const WorkDesc wd, const float *__restrict__ e,
                                                        const float *__restrict__ r, float *diag,
                                                        const int32_t *__restrict__ row_lo,
                                                        const uint64_t *__restrict__ row_off, uint8_t *dir,
                                                        int end_free, float b_match, int32_t *path_i,
                                                        int32_t *path_j, uint32_t *path_len,
                                                        rawalign_result_t *result)
{
    const int n = wd.nrows, m = wd.m;
    const long long num = wd.num, den = wd.den, w = wd.w, nd = num + den;
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
        const float *p1 = B[(d + 2) % 3];  // anti-diagonal d-1
        const float *p2 = B[(d + 1) % 3];  // anti-diagonal d-2
        // rows of anti-diagonal d inside the band |j*den - i*num| <= w*den, j = d - i
        long long ilo = -floor_div_tb(-(((long long)d - w) * den), nd);
        long long ihi = floor_div_tb(((long long)d + w) * den, nd);
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
            const long long j = d - i;
            const float nw = p2[i], nn = p1[i], ww = p1[i + 1];
            const float dd = fabsf(__fsub_rn(e[i], r[j]));
            const bool start = (i == 0 && j == 0);
            const float mn = start ? 0.f : min3f(nw, nn, ww);
            const float v = __fadd_rn(dd, mn);
            cur[i + 1] = v;
            dir[row_off[i] + (uint64_t)(j - row_lo[i])] =
                start ? kDirStart : (nw == mn ? kDirNW : (nn == mn ? kDirN : kDirW));
            cells++;
            if (i == n - 1 && v < s_best) {
                s_best = v;
                s_bestj = (int)j;
            }
        }
        __syncthreads();
    }
    atomicAdd(&s_cells, cells);
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    long long dev = (long long)(m - 1) * den - (long long)(n - 1) * num;
    dev = dev < 0 ? -dev : dev;
    float cost;
    int ei, ej;
    if (end_free) {
        cost = s_best;
        ej = s_bestj;
        ei = ej >= 0 ? n - 1 : -1;
    } else {
        cost = dev <= w * den ? B[(n + m - 2) % 3][n] : kInf;
        ei = n - 1;
        ej = m - 1;
    }
    uint32_t len = 0;
    if (cost < kInf && ei >= 0) {
        // walk back; a path has at most n + m - 1 cells, which also bounds the loop
        int i = ei, j = ej;
        while (len < (uint32_t)(n + m - 1)) {
            path_i[len] = i;
            path_j[len] = j;
            ++len;
            const uint8_t t = dir[row_off[i] + (uint64_t)(j - row_lo[i])];
            if (t == kDirStart)
                break;
            if (t != kDirW)
                --i;
            if (t != kDirN)
                --j;
        }
    }
    *path_len = len;
    result->read_id = (uint64_t)wd.read;
    result->cand_idx = (uint32_t)wd.cand;
    result->cost = cost;
    result->score = __fsub_rn(__fmul_rn(b_match, (float)wd.n_read), cost);
    result->end_i = ei;
    result->end_j = ej;
    result->w_eff = wd.w_report;
    result->cells = s_cells;
    result->status = 0;
    result->is_best = 0;
    result->decision = RA_UNMAPPED;
}

}  // namespace ra

using namespace ra_host;

extern "C" int rawalign_dtw_traceback(rawalign_dtw_t *h, const float *events, uint32_t n_events,
                                      const rawalign_candidate_t *cand, int32_t end_mode, int32_t *path_i,
                                      int32_t *path_j, uint32_t cap, uint32_t *path_len, rawalign_result_t *result)
{
    NvtxRange nvtx_range("rawalign_dtw_traceback");
    if (!h || !events || !cand || !path_i || !path_j || !path_len || !result || n_events == 0)
        return RA_EINVAL;
    if (end_mode != RA_END_GLOBAL && end_mode != RA_END_FREE)
        return RA_EINVAL;
    const int k = h->cfg.k;
    if (cand->strand > 1 || cand->ref_offset > h->ref_len || cand->ref_len_bases > h->ref_len - cand->ref_offset ||
        (int64_t)cand->ref_len_bases < k)
        return RA_EINVAL;
    const int64_t n = n_events, m = (int64_t)cand->ref_len_bases - k + 1;
    if (n >= (1 << 30) || m >= (1 << 30) || (uint64_t)cap < (uint64_t)(n + m - 1))
        return RA_EINVAL;
    for (int64_t x = 0; x < n; ++x)
        if (!std::isfinite(events[x]))
            return RA_EINVAL;
    BandDef band;
    int32_t wrep;
    if (band_for(n, m, cand->band_w, cand->slope_num, cand->slope_den, band, wrep) != 0)
        return RA_EINVAL;
    // each row's band: first column and the offset of its directions
    std::vector<int32_t> lo(n);
    std::vector<uint64_t> off(n + 1);
    off[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t a = band.lo(i), b = band.hi(i);
        lo[i] = (int32_t)std::min<int64_t>(a, m);
        off[i + 1] = off[i] + (uint64_t)std::max<int64_t>(b - a + 1, 0);
    }
    WorkDesc wd{};
    wd.num = band.num;
    wd.den = band.den;
    wd.nrows = (int32_t)n;
    wd.m = (int32_t)m;
    wd.w = (int32_t)band.w;
    wd.cand = 0;
    wd.read = (int32_t)cand->read_id;
    wd.n_read = (int32_t)n;
    wd.w_report = wrep;
    SigDesc sd{};
    sd.ref_off = cand->ref_offset;
    sd.r_off = 0;
    sd.len = cand->ref_len_bases;
    sd.strand = cand->strand;

    cudaSetDevice(h->device);
    std::vector<void *> blocks;
    auto take = [&](uint64_t bytes) {
        void *p = h->arena.alloc(std::max<uint64_t>(bytes, 1));
        if (p)
            blocks.push_back(p);
        return p;
    };
    auto release = [&]() {
        for (void *p : blocks)
            h->arena.release(p);
    };
    float *d_e = (float *)take(4ull * n);
    float *d_r = (float *)take(4ull * m);
    SigDesc *d_sd = (SigDesc *)take(sizeof(SigDesc));
    uint8_t *d_dir = (uint8_t *)take(off[n]);
    int32_t *d_lo = (int32_t *)take(4ull * n);
    uint64_t *d_off = (uint64_t *)take(8ull * (n + 1));
    float *d_diag = (float *)take(4ull * 3 * (n + 2));
    int32_t *d_pi = (int32_t *)take(4ull * (n + m));
    int32_t *d_pj = (int32_t *)take(4ull * (n + m));
    uint32_t *d_len = (uint32_t *)take(4);
    rawalign_result_t *d_res = (rawalign_result_t *)take(sizeof(rawalign_result_t));
    if (!d_e || !d_r || !d_sd || !d_dir || !d_lo || !d_off || !d_diag || !d_pi || !d_pj || !d_len || !d_res) {
        release();
        return RA_ENOMEM;
    }
    cudaStream_t s = h->stream;
    uint32_t len = 0;
    int rc = RA_OK;
    do {
        if (cudaMemcpyAsync(d_e, events, 4ull * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_sd, &sd, sizeof(sd), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_lo, lo.data(), 4ull * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_off, off.data(), 8ull * (n + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            launch_expected_signal(d_sd, 1, h->d_ref, h->d_pore, k, d_r, s) != cudaSuccess) {
            rc = RA_EDEVICE;
            break;
        }
        dtw_trace_kernel<<<1, 256, 0, s>>>(wd, d_e, d_r, d_diag, d_lo, d_off, d_dir, end_mode == RA_END_FREE,
                                           h->cfg.b_match, d_pi, d_pj, d_len, d_res);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&len, d_len, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(result, d_res, sizeof(*result), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = RA_EDEVICE;
            break;
        }
        if (len > (uint32_t)(n + m - 1)) {
            rc = RA_EDEVICE;
            break;
        }
        if (len && (cudaMemcpy(path_i, d_pi, 4ull * len, cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(path_j, d_pj, 4ull * len, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            rc = RA_EDEVICE;
            break;
        }
    } while (0);
    cudaStreamSynchronize(s);
    release();
    if (rc != RA_OK)
        return rc;
    std::reverse(path_i, path_i + len);
    std::reverse(path_j, path_j + len);
    *path_len = len;
    return RA_OK;
}
