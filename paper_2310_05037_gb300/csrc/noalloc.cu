// noalloc.cu -- one alignment with no device allocation at all.
//
// For callers that are not allowed to allocate device memory: for example a
// plug-in that runs inside a host program which owns the whole device memory
// budget, or a sequencing control loop that must never call cudaMalloc,
// because cudaMalloc can wait for the device and stall the other streams of
// the process.  Such a caller passes its own input and output buffers; the
// working rows the DP needs live in a fixed array that is part of the loaded
// library itself (a static __device__ array, so every GPU that loads the
// library holds it until the process exits).
//
// The work is the plain one-CTA kernel of dtw_kernels.cu (its variant that
// takes the work record by value, as a kernel parameter, so nothing is copied
// from host memory), with its scratch (three anti-diagonal buffers and the
// per-read best key) placed in that array.
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr uint32_t kMaxRows = 1u << 16;  // events (DP rows) per alignment at most
constexpr uint32_t kMaxCols = 1u << 30;  // expected values per alignment: below this (as the batch path)
constexpr size_t kKeyOff = 128;          // per-read best key (8 bytes)
constexpr size_t kDiagOff = 256;         // 3 * (kMaxRows + 2) floats
constexpr size_t kScratchBytes = kDiagOff + sizeof(float) * 3 * ((size_t)kMaxRows + 2);

// The scratch array: host code sees only a stand-in for this name, so the
// device address is looked up with cudaGetSymbolAddress on each device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up on the first
// call for that device.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return RA_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
            return RA_EDEVICE;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RA_OK;
}

}  // namespace

extern "C" int rawalign_dtw_align_noalloc(const float *d_events, uint32_t n_events, const float *d_ref_signal,
                                          uint32_t m, int32_t band_w, int64_t slope_num, int64_t slope_den,
                                          int32_t end_mode, float b_match, rawalign_result_t *d_result,
                                          void *cuda_stream)
{
    if (!d_events || !d_ref_signal || !d_result || n_events == 0 || m == 0)
        return RA_EINVAL;
    if (n_events > kMaxRows)
        return RA_EINVAL;  // more rows than the fixed scratch holds
    if (m >= kMaxCols)
        return RA_EINVAL;  // the kernel's diagonal index n + m - 2 must stay a small int
    if (end_mode != RA_END_GLOBAL && end_mode != RA_END_FREE)
        return RA_EINVAL;
    ra::WorkDesc wd;
    memset(&wd, 0, sizeof wd);
    int64_t num = 0, den = 1, w = 0;
    int32_t wrep = 0;
    if (ra::host_band(n_events, m, band_w, slope_num, slope_den, &num, &den, &w, &wrep) != RA_OK)
        return RA_EINVAL;
    wd.ev_off = 0;
    wd.r_off = 0;
    wd.fin_off = ~0ull;
    wd.num = num;
    wd.den = den;
    wd.row0 = 0;
    wd.nrows = (int32_t)n_events;
    wd.m = (int32_t)m;
    wd.w = (int32_t)w;
    wd.cand = 0;
    wd.read = 0;
    wd.n_read = (int32_t)n_events;
    wd.fin_lo = -1;
    wd.fin_wid = 0;
    wd.w_report = wrep;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != RA_OK)
        return rc;
    char *b = (char *)base;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the best key starts fresh on every call (a device-side memset on the
    // stream); the diagonal buffers are reset by the kernel itself
    if (cudaMemsetAsync(b + kKeyOff, 0, sizeof(unsigned long long), s) != cudaSuccess)
        return RA_EDEVICE;
    cudaError_t e = ra::launch_plain_byval(wd, d_events, d_ref_signal, (float *)(b + kDiagOff), d_result,
                                           (unsigned long long *)(b + kKeyOff), b_match, end_mode == RA_END_FREE, s);
    return e == cudaSuccess ? RA_OK : RA_EDEVICE;
}
