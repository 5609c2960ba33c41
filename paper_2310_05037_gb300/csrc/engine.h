// engine.h -- host-side planning types shared by engine.cu (batches) and
// serve.cu (Read-Until serving): band rule, stripe schedule, arena, records,
// and the handle itself.  Internal to librawalign_dtw.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

using namespace ra;

namespace ra_host {

// An NVTX range around one entry point (submit, plan, launch, poll), so that
// a profiler's timeline shows where the host time goes; without a profiler
// attached the calls do nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kBlock = 128;
constexpr int kLag = ra::kLaneLag;  // columns between neighbouring lanes (the kernel's)
// (lanes per alignment, rows per lane); the cost factor is the relative issue
// cost of one lane-cell slot (more rows per lane amortise the per-step work).
// Relative cost of one lane-cell slot per variant: the autotuner's
// measurement on a GB300 (each variant on a batch shaped for its steady
// state; 8 rows per lane pay the per-step overhead over fewer cells, 24 rows
// amortise it further).  rawalign_dtw_set_variant_costs replaces them.
constexpr int kVariants[][2] = {{32, 16}, {16, 16}, {32, 8}, {16, 8}, {8, 8}, {4, 8}, {16, 24}, {8, 24}, {32, 24},
                               {4, 24}};
const double kSlotCost[] = {1.2107, 1.2336, 1.8882, 1.9132, 1.9968, 2.1240, 1.0095, 1.0287, 1.0, 1.0656};
constexpr int kNumVariants = 10;
constexpr int kSplitVariant = 8;  // (32, 24): the lane layout of the block-split kernel
constexpr int kMaxClasses = 64;              // launches per run (variant x ring size)
constexpr size_t kSmemRingLimit = 96 * 1024; // larger rings go to global memory

// Host worker threads for the planner's parallel loops, created once per
// process.  One loop runs on the pool at a time; a loop started while the
// pool is busy (another handle planning on another thread, or a loop inside
// a pool task) runs on threads of its own instead.  The calling thread takes
// tasks too, so a loop also completes if the workers are gone (a forked child).
class WorkerPool {
public:
    explicit WorkerPool(unsigned workers)
    {
        for (unsigned w = 0; w < workers; ++w)
            th_.emplace_back([this] { work(); });
    }
    ~WorkerPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_)
            t.join();
    }
    // Runs fn(t) for t in [0, T); false (nothing run) if the pool is busy.
    bool try_run(unsigned T, const std::function<void(unsigned)> &fn)
    {
        std::unique_lock<std::mutex> rl(run_mu_, std::try_to_lock);
        if (!rl.owns_lock())
            return false;
        std::unique_lock<std::mutex> lk(mu_);
        job_ = &fn;
        tasks_ = T;
        next_ = 0;
        pending_ = T;
        ++gen_;
        cv_.notify_all();
        take(lk);
        done_cv_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
        return true;
    }

private:
    void take(std::unique_lock<std::mutex> &lk)
    {
        while (job_ && next_ < tasks_) {
            const unsigned t = next_++;
            const std::function<void(unsigned)> *job = job_;
            lk.unlock();
            (*job)(t);
            lk.lock();
            if (--pending_ == 0)
                done_cv_.notify_all();
        }
    }
    void work()
    {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        while (true) {
            cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_)
                return;
            seen = gen_;
            take(lk);
        }
    }
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    std::vector<std::thread> th_;
    const std::function<void(unsigned)> *job_ = nullptr;
    unsigned tasks_ = 0, next_ = 0, pending_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

inline unsigned host_threads()
{
    return std::min(std::max(1u, std::thread::hardware_concurrency()), 16u);
}

inline WorkerPool &worker_pool()
{
    static WorkerPool pool(host_threads() - 1);
    return pool;
}

// Runs task(t) for t in [0, T) on the worker pool (or on threads of its own
// when the pool is busy).
inline void run_tasks(unsigned T, const std::function<void(unsigned)> &task)
{
    if (T <= 1) {
        if (T == 1)
            task(0);
        return;
    }
    if (worker_pool().try_run(T, task))
        return;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < T; ++t)
        th.emplace_back(task, t);
    for (auto &x : th)
        x.join();
}

// Runs fn(lo, hi) over [0, n) in up to 16 ranges (one when n is small).
template <typename F>
inline void parallel_for(uint64_t n, F fn, uint64_t min_per_thread = 1 << 15)
{
    const uint64_t T = std::max<uint64_t>(1, std::min<uint64_t>(host_threads(), n / min_per_thread));
    if (T == 1) {
        fn((uint64_t)0, n);
        return;
    }
    run_tasks((unsigned)T, [&](unsigned t) { fn(n * t / T, n * (t + 1) / T); });
}

// ---------------------------------------------------------------- band math
inline int64_t fdiv(int64_t a, int64_t b)
{
    int64_t q = a / b, r = a % b;
    return (r != 0 && ((r < 0) != (b < 0))) ? q - 1 : q;
}
inline int64_t cdiv(int64_t a, int64_t b) { return -fdiv(-a, b); }

struct BandDef {
    int64_t num = 0, den = 1, w = 0, m = 1;
    int64_t per = 0;    // den / gcd(num, den) when known (0: not computed), see band_cells
    int64_t hi_row = 0; // with per: the first row whose band reaches the last column
    int64_t lo(int64_t i) const { return std::max<int64_t>(0, cdiv(i * num - w * den, den)); }
    int64_t hi(int64_t i) const { return std::min<int64_t>(m - 1, fdiv(i * num + w * den, den)); }
};

// sum_{i=0}^{n-1} floor((a i + b) / c) for n, a, b >= 0 and c > 0, in
// O(log c) steps: whole multiples of c in a and b are summed directly, and
// with a, b < c the sum counts the lattice points under the line, which is
// the same kind of sum with the roles of a and c exchanged (the Euclidean
// reduction of the floor sum).
inline uint64_t floor_sum(uint64_t n, uint64_t c, uint64_t a, uint64_t b)
{
    unsigned __int128 acc = 0;
    while (n > 0) {
        if (a >= c) {
            acc += (unsigned __int128)(n * (n - 1) / 2) * (a / c);
            a %= c;
        }
        if (b >= c) {
            acc += (unsigned __int128)n * (b / c);
            b %= c;
        }
        // points (i, k) with k >= 1 and k c <= a i + b: per k, the rows
        // i >= (k c - b) / a; rewritten as a floor sum over k of (c k' + y % c) / a
        uint64_t an;
        if (!__builtin_mul_overflow(a, n, &an) && an <= UINT64_MAX - b) {
            const uint64_t y = an + b;
            if (y < c)
                break;
            n = y / c;
            b = y - n * c;
        } else {
            const unsigned __int128 y = (unsigned __int128)a * n + b;
            n = (uint64_t)(y / c);
            b = (uint64_t)(y % c);
        }
        std::swap(a, c);
    }
    return (uint64_t)acc;
}

// Fills a band's per and hi_row, which let band_cells count rows away from
// the table's edges in O(1) (for bands counted many times, as in serving).
inline void prepare_cell_count(BandDef &b)
{
    if (b.num <= 0)
        return;
    int64_t x = b.num, y = b.den;
    while (y) {
        const int64_t t = x % y;
        x = y;
        y = t;
    }
    b.per = b.den / x;
    b.hi_row = std::max<int64_t>(0, cdiv((b.m - 1 - b.w) * b.den, b.num));
}

// In-band cells of rows [r0, r1) of a band (the table's cells (i, j) with
// lo(i) <= j <= hi(i)), exactly, in O(log den): the sums of hi and of lo over
// the rows are floor sums between the rows where the band meets the table's
// edges.  Rows whose band starts past the last column hold no cell.
inline uint64_t band_cells(const BandDef &b, int64_t r0, int64_t r1)
{
    if (r1 <= r0)
        return 0;
    if (b.num == 0)
        return (uint64_t)(r1 - r0) * (uint64_t)(b.hi(0) - b.lo(0) + 1);
    // a band that covers every row of the range whole (short pieces with a
    // wide band, as most gaps of anchor-guided alignment): m cells per row
    if (b.w >= b.m - 1 && r0 >= 0 && (r1 - 1) * b.num <= b.w * b.den)
        return (uint64_t)(r1 - r0) * (uint64_t)b.m;
    // rows with lo(i) <= m - 1: i num - w den <= (m - 1) den
    r1 = std::min<int64_t>(r1, fdiv((b.m - 1 + b.w) * b.den, b.num) + 1);
    if (r1 <= r0)
        return 0;
    const uint64_t num = (uint64_t)b.num, den = (uint64_t)b.den, wd = (uint64_t)(b.w * b.den);
    if (b.per > 0 && r1 <= b.hi_row && r0 * b.num >= b.w * b.den - b.den + 1) {
        // no row of the range meets an edge of the table: with x = i num / den,
        // hi - lo + 1 = floor(x + w) - ceil(x - w) + 1 = 2w + [x is whole],
        // and x is whole exactly on the multiples of den / gcd(num, den)
        const uint64_t whole = (uint64_t)(fdiv(r1 - 1, b.per) - fdiv(r0 - 1, b.per));
        return (uint64_t)(r1 - r0) * (uint64_t)(2 * b.w) + whole;
    }
    // sum of hi: floor((i num + w den) / den) below i_h, m - 1 from i_h on
    const int64_t i_h = std::max<int64_t>(0, cdiv((b.m - 1 - b.w) * b.den, b.num));
    uint64_t s_hi = 0;
    {
        const int64_t a = r0, e = std::min(r1, std::max(r0, i_h));
        if (e > a)
            s_hi += floor_sum((uint64_t)e, den, num, wd) - floor_sum((uint64_t)a, den, num, wd);
        const int64_t a2 = std::max(r0, i_h);
        if (r1 > a2)
            s_hi += (uint64_t)(r1 - a2) * (uint64_t)(b.m - 1);
    }
    // sum of lo: 0 up to i_l, from i_l on ceil((i num - w den) / den) >= 1,
    // a floor sum over t = i - i_l with offset i_l num - w den + den - 1 >= den
    const int64_t i_l = fdiv(b.w * b.den, b.num) + 1;
    uint64_t s_lo = 0;
    {
        const int64_t a = std::max(r0, i_l);
        if (r1 > a) {
            const uint64_t off = (uint64_t)(i_l * b.num - b.w * b.den + b.den - 1);
            s_lo = floor_sum((uint64_t)(r1 - i_l), den, num, off) - floor_sum((uint64_t)(a - i_l), den, num, off);
        }
    }
    return s_hi - s_lo + (uint64_t)(r1 - r0);
}

// Band of one candidate (Sec. 2.4.3): derived slope (m-1)/(n-1) unless given;
// w_eff = max(w, ceil(num/(2 den)), 1); no band -> num 0, den 1, w = m.
inline int band_for(int64_t n, int64_t m, int32_t band_w, int64_t num_in, int64_t den_in, BandDef &b,
             int32_t &w_report)
{
    b.m = m;
    if (band_w < 0 || n == 1 || m == 1) {
        b.num = 0;
        b.den = 1;
        b.w = m;
        w_report = -1;
        return 0;
    }
    int64_t num = num_in, den = den_in;
    if (num == 0 && den == 0) {
        num = m - 1;
        den = n - 1;
    }
    if (num < 0 || den <= 0 || num > (1ll << 30) || den > (1ll << 30))
        return -1;
    int64_t half = (num + 2 * den - 1) / (2 * den);
    int64_t w = std::max<int64_t>(std::max<int64_t>(band_w, half), 1);
    if (w > (1ll << 30))
        return -1;
    b.num = num;
    b.den = den;
    b.w = w;
    w_report = (int32_t)w;
    return 0;
}

// Schedule of one piece (rows row0..row0+nrows-1) for a (G, HR) variant, in
// O(1): dC bounds b(k,t) - a(k+1,t) + 2 for every lane and stripe, where b is
// the last in-band column of a lane's rows in stripe k and a the first of its
// rows in stripe k+1.  With hi(x) <= x*s + w and lo(y) >= y*s - w
// (s = num/den, y - x = H - HR + 1): b - a <= 2w - (H - HR + 1) s, and
// b - a <= m - 1 from the table's edges.  Lane t runs kLag columns behind lane
// t-1 (it takes lane t-1's bottom row from kLag steps back, so the kernel can
// compute two consecutive columns of a lane as two interleaved chains); the
// last lane of a stripe writes a ring entry kLag * (G-1) steps after lane 0
// passed its column, and lane 0 of the next stripe may read it two steps
// before it uses it, two steps after it is written: dC >= kLag * G + 3.
struct Sched {
    int32_t dC = 0, a0 = 0, s_end = 0;
    double cells_est = 0;
    double eff = 0;  // in-band cells / lane-cell slots (estimate)
};

// The part of schedule() that depends on the variant, given the band edges
// every variant shares (a0 = lo(row0), b_last = hi(last row)); with G and HR
// fixed at compile time the divisions by H and HR become multiplications.
// Same operations in the same order as schedule(), so the same results.
template <int G, int HR>
inline Sched schedule_from_edges(const BandDef &b, int64_t nrows, int64_t a0, int64_t b_last)
{
    Sched s;
    constexpr int64_t H = (int64_t)G * HR;
    const int64_t K = (nrows + H - 1) / H;
    s.a0 = (int32_t)a0;
    if (s.a0 > b.m - 1) {
        s.s_end = 0;
        return s;
    }
    int64_t span = fdiv(2 * b.w * b.den - (H - HR + 1) * b.num, b.den);
    span = std::min<int64_t>(span, b.m - 1);
    const int64_t dC = std::max<int64_t>((int64_t)kLag * G + 3, span + 2);
    const int64_t nl = nrows - 1 - (K - 1) * H;
    const int64_t t_last = nl / HR;
    s.dC = (int32_t)dC;
    const int64_t se = b_last - s.a0 + 3 + (int64_t)kLag * t_last + (K - 1) * dC;
    s.s_end = (int32_t)std::max<int64_t>(se, 1);
    s.cells_est = (double)nrows * (double)std::min<int64_t>(2 * b.w + 1, b.m);
    const double slots = (double)s.s_end * G * HR;
    s.eff = slots > 0 ? s.cells_est / slots : 0;
    return s;
}

inline Sched schedule(const BandDef &b, int64_t row0, int64_t nrows, int G, int HR)
{
    Sched s;
    const int64_t H = (int64_t)G * HR;
    const int64_t K = (nrows + H - 1) / H;
    const int64_t last = row0 + nrows - 1;
    s.a0 = (int32_t)b.lo(row0);
    if (s.a0 > b.m - 1) {
        s.s_end = 0;
        return s;
    }
    int64_t span = fdiv(2 * b.w * b.den - (H - HR + 1) * b.num, b.den);
    span = std::min<int64_t>(span, b.m - 1);
    const int64_t dC = std::max<int64_t>((int64_t)kLag * G + 3, span + 2);
    const int64_t nl = nrows - 1 - (K - 1) * H;
    const int64_t t_last = nl / HR;
    const int64_t b_last = b.hi(last);
    s.dC = (int32_t)dC;
    const int64_t se = b_last - s.a0 + 3 + (int64_t)kLag * t_last + (K - 1) * dC;
    s.s_end = (int32_t)std::max<int64_t>(se, 1);
    s.cells_est = (double)nrows * (double)std::min<int64_t>(2 * b.w + 1, b.m);
    const double slots = (double)s.s_end * G * HR;
    s.eff = slots > 0 ? s.cells_est / slots : 0;
    return s;
}

// ---------------------------------------------------------------- flat map
// Hash map from 64-bit keys (tickets, read ids) to small values, for the
// serving path's per-chunk bookkeeping: open addressing with linear probing
// in one array (no allocation per entry), at most half full, and deletion by
// backward shift (no tombstones, so lookups stay short however many entries
// come and go).  Every key value is allowed; occupancy is kept apart.
template <class V>
class FlatMap64 {
  public:
    explicit FlatMap64(size_t cap = 16) { rehash(cap); }
    size_t size() const { return n_; }
    void reserve(size_t n)
    {
        if (2 * n > keys_.size())
            rehash(2 * n);
    }
    void clear()
    {
        if (n_)
            std::fill(used_.begin(), used_.end(), (uint8_t)0);
        n_ = 0;
    }
    V *find(uint64_t k)
    {
        for (size_t i = slot(k);; i = (i + 1) & mask_) {
            if (!used_[i])
                return nullptr;
            if (keys_[i] == k)
                return &vals_[i];
        }
    }
    bool contains(uint64_t k) { return find(k) != nullptr; }
    // the value of k, inserted value-initialised when absent
    V &operator[](uint64_t k)
    {
        if (V *v = find(k))
            return *v;
        if (2 * (n_ + 1) > keys_.size())
            rehash(2 * keys_.size());
        size_t i = slot(k);
        while (used_[i])
            i = (i + 1) & mask_;
        used_[i] = 1;
        keys_[i] = k;
        vals_[i] = V();
        ++n_;
        return vals_[i];
    }
    bool erase(uint64_t k)
    {
        size_t i = slot(k);
        while (true) {
            if (!used_[i])
                return false;
            if (keys_[i] == k)
                break;
            i = (i + 1) & mask_;
        }
        // backward shift: move later entries of the probe run into the hole
        // unless their home slot lies cyclically in (hole, entry]
        size_t j = i;
        while (true) {
            j = (j + 1) & mask_;
            if (!used_[j])
                break;
            const size_t h = slot(keys_[j]);
            const bool stays = (i <= j) ? (i < h && h <= j) : (i < h || h <= j);
            if (stays)
                continue;
            keys_[i] = keys_[j];
            vals_[i] = vals_[j];
            i = j;
        }
        used_[i] = 0;
        --n_;
        return true;
    }

  private:
    // the finaliser of MurmurHash3 (a bijective 64-bit mix)
    size_t slot(uint64_t k) const
    {
        k ^= k >> 33;
        k *= 0xff51afd7ed558ccdull;
        k ^= k >> 33;
        k *= 0xc4ceb9fe1a85ec53ull;
        k ^= k >> 33;
        return (size_t)k & mask_;
    }
    void rehash(size_t cap)
    {
        size_t c = 16;
        while (c < cap)
            c <<= 1;
        std::vector<uint64_t> ok;
        std::vector<V> ov;
        std::vector<uint8_t> ou;
        ok.swap(keys_);
        ov.swap(vals_);
        ou.swap(used_);
        keys_.assign(c, 0);
        vals_.assign(c, V());
        used_.assign(c, 0);
        mask_ = c - 1;
        n_ = 0;
        for (size_t x = 0; x < ou.size(); ++x)
            if (ou[x])
                (*this)[ok[x]] = ov[x];
    }
    std::vector<uint64_t> keys_;
    std::vector<V> vals_;
    std::vector<uint8_t> used_;
    size_t mask_ = 0, n_ = 0;
};

// ---------------------------------------------------------------- arena
// Best-fit allocator over the caller's arena: free ranges indexed by offset
// (to merge a released range with its neighbours) and by size (to find the
// smallest range that fits in O(log n)); 256-byte granules.
struct Arena {
    char *base = nullptr;
    uint64_t size = 0;
    void init(void *p, uint64_t n)
    {
        base = (char *)p;
        size = n;
        free_.clear();
        by_size_.clear();
        used_.clear();
        if (n)
            add_free(0, n);
    }
    void *alloc(uint64_t n)
    {
        n = (n + 255) & ~255ull;
        if (n == 0)
            n = 256;
        auto bs = by_size_.lower_bound(std::make_pair(n, (uint64_t)0));
        if (bs == by_size_.end())
            return nullptr;
        const uint64_t off = bs->second, sz = bs->first;
        by_size_.erase(bs);
        free_.erase(off);
        if (sz > n)
            add_free(off + n, sz - n);
        used_[off] = n;
        return base + off;
    }
    void release(void *p)
    {
        if (!p)
            return;
        uint64_t off = (uint64_t)((char *)p - base);
        auto u = used_.find(off);
        if (u == used_.end())
            return;
        uint64_t n = u->second;
        used_.erase(u);
        // merge with the free neighbours on both sides
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {
            n += nx->second;
            by_size_.erase(std::make_pair(nx->second, nx->first));
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                off = pv->first;
                n += pv->second;
                by_size_.erase(std::make_pair(pv->second, pv->first));
                free_.erase(pv);
            }
        }
        add_free(off, n);
    }

private:
    void add_free(uint64_t off, uint64_t n)
    {
        free_[off] = n;
        by_size_.insert(std::make_pair(n, off));
    }
    std::map<uint64_t, uint64_t> free_;                 // offset -> size
    std::set<std::pair<uint64_t, uint64_t>> by_size_;   // (size, offset)
    std::map<uint64_t, uint64_t> used_;                 // offset -> size
};

struct ClassLaunch {
    bool split = false;  // the block-split kernel: one alignment per block of four warps
    int G = 0, HR = 0;
    double max_cost = 0;       // lane-steps of the class's largest alignment (steps x lanes, empty as 0)
    int first = 0, count = 0;  // range in the sorted work array
    int ring_cap = 0;
    int ring_in_smem = 1;
    int grid = 0;
    size_t smem = 0;
    float *gring = nullptr;
};

struct Batch {
    uint64_t slots = 0;          // planned lane-cell slots (sum of steps x G x HR)
    uint32_t n_reads = 0, n_cands = 0;
    uint64_t n_events = 0;
    uint64_t n_r = 0;            // expected values in d_r
    uint32_t n_split = 0;        // work items on the block-split kernel
    double host_plan_ms = 0, host_upload_ms = 0;  // host time of prepare: planning, uploads
    std::vector<void *> blocks;  // arena allocations
    float *d_events = nullptr;
    SigDesc *d_sig = nullptr;
    float *d_r = nullptr;
    WorkDesc *d_work = nullptr;
    rawalign_result_t *d_results = nullptr;
    unsigned long long *d_keys = nullptr;
    int *d_read_of = nullptr;
    int *d_queue = nullptr;  // [kNumVariants]
    int *d_err = nullptr;    // [2]
    float *d_plain_diag = nullptr;
    int max_rows = 0;
    uint32_t n_work = 0;                    // DTW work items (candidates, or gaps when anchored)
    bool anchored = false;                  // anchor-guided batch (Sec. 2.4.2)
    bool et = false;                        // early termination (Sec. 2.4.1)
    rawalign_result_t *d_pres = nullptr;    // anchored: per-gap DTW results
    unsigned long long *d_pkeys = nullptr;  // anchored: per-gap keys (unused by the decision)
    PieceRef *d_plan = nullptr;             // anchored: pieces of every candidate in path order
    CombineDesc *d_cdesc = nullptr;         // anchored: per-candidate piece range and table size
    std::vector<ClassLaunch> classes;
    uint64_t cells = 0;
    bool auto_release = false;
    bool plain = false;
    cudaGraphExec_t graph_part[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t launches = 0;
    bool ran = false;
};

struct Ticket {
    uint64_t batch = 0;  // batch id (0 = serving)
    cudaEvent_t done = nullptr;
    rawalign_result_t *d_results = nullptr;
    uint32_t n = 0;
    int *d_err = nullptr;
    std::vector<rawalign_result_t> host;  // serving: filled at flush completion
    std::vector<uint64_t> read_ids;       // serving: caller read ids per result
    bool serving = false;
};

// One piece of work as planned on the host.
struct PlanItem {
    WorkDesc wd;
    int wave = 0;       // early termination: 0 = first candidate of its read (queued first), 1 = the others
    int variant = 0;
    int cap = 0;        // ring entries the piece needs (power of two)
    double cost = 0;    // lane-steps: longest first
    bool split = false; // runs on a whole block of four warps (split kernel)
};

// Scratch of the launch-order sort, kept by a handle across batches.
struct SortScratch {
    std::vector<uint64_t> key, key2;
    std::vector<int> tmp;
};

struct ServeState;

// Planner knobs the autotuner may set (tuning file lines "ring_bins S" and
// "latency_split X"): launch classes bin ring sizes by powers of 2^S, and
// an alignment longer than X times the estimated batch length moves to a
// 32-lane variant (X <= 0: 0.5 for batches with few alignments per resident
// group, else 1.0).
struct PlanParams {
    int ring_bin_shift = 2;     // 2: ring sizes in powers of four; 1: powers of two (falling back to
                                // four for a batch that would need more than kMaxClasses launches)
    double latency_split = 0;
    bool split = true;          // the block-split kernel may be used (not with early termination)
    double split_factor = 0.0;  // "block_split X": an alignment whose time on one warp exceeds X times
                                // the batch's balanced length (its work over all resident lanes)
                                // goes to a block of four warps; 0 = never (the default: on the
                                // long-read workload it measured slower than 32-lane groups)
};

}  // namespace ra_host

using namespace ra_host;

struct rawalign_dtw {
    rawalign_dtw_config_t cfg{};
    cudaStream_t stream = nullptr;
    cudaStream_t aux[kMaxClasses] = {};   // launch classes as parallel branches (see classes_as_chain)
    cudaEvent_t fork = nullptr, join[kMaxClasses] = {};
    cudaStream_t upload = nullptr;         // batch uploads: overlap the previous batch's kernels
    cudaEvent_t uploaded = nullptr;
    char *stage = nullptr;                 // pinned host staging for planned records (grown on demand)
    size_t stage_bytes = 0;
    std::vector<ra_host::PlanItem> plan_items;  // planning scratch, reused across batches
    std::vector<int> plan_order;
    ra_host::SortScratch plan_sort;
    int device = 0;
    int sm_count = 152;
    Arena arena;
    float *d_pore = nullptr;
    uint8_t *d_ref = nullptr;
    uint64_t ref_len = 0;
    uint64_t next_id = 1;
    std::map<uint64_t, Batch> batches;
    std::map<uint64_t, Ticket> tickets;
    int max_blocks[kNumVariants][2] = {};
    ServeState *serve = nullptr;       // Read-Until serving state (serve.cu)
    double slot_cost[kNumVariants] = {};  // relative cost of a lane-cell slot per variant
    ra_host::PlanParams plan;             // planner knobs from the tuning file
};


namespace ra_host {

inline int cuda_ok(cudaError_t e)
{
    if (e == cudaSuccess)
        return RA_OK;
    fprintf(stderr, "rawalign_dtw: CUDA error %s\n", cudaGetErrorString(e));
    return RA_EDEVICE;
}

#define RA_CUDA(x)                      \
    do {                                \
        int rc__ = ra_host::cuda_ok(x); \
        if (rc__ != RA_OK)              \
            return rc__;                \
    } while (0)

inline int next_pow2(int64_t x)
{
    int64_t p = 1;
    while (p < x)
        p <<= 1;
    return (int)p;
}

// Chooses the striped variant for one piece of an alignment: most in-band
// cells per unit of issue cost, ties to the earlier (wider) variant.
// f(std::integral_constant<int, v>) for v = 0, 1, ... in order
template <class F, size_t... V>
inline void for_each_variant(F &&f, std::index_sequence<V...>)
{
    (f(std::integral_constant<int, (int)V>{}), ...);
}

inline int choose_variant(const BandDef &band, int64_t row0, int64_t n, Sched &out, const double *cost = kSlotCost)
{
    // the band edges of the first and last rows are the same for every
    // variant: computed once, then each variant's schedule from them
    const int64_t a0 = band.lo(row0), b_last = band.hi(row0 + n - 1);
    if (a0 > band.m - 1) {
        // no cell in the first row: nothing to schedule (every variant agrees)
        out = schedule_from_edges<kVariants[0][0], kVariants[0][1]>(band, n, a0, b_last);
        return 0;
    }
    int best = -1;
    double best_score = -1;
    auto consider = [&](auto vt) {
        constexpr int v = decltype(vt)::value;
        const Sched s = schedule_from_edges<kVariants[v][0], kVariants[v][1]>(band, n, a0, b_last);
        const double score = s.eff / cost[v] * (1.0 + 0.02 * (kNumVariants - v));
        if (score > best_score) {
            best_score = score;
            best = v;
            out = s;
        }
    };
    for_each_variant(consider, std::make_index_sequence<kNumVariants>{});
    return best;
}

inline int ring_need(const WorkDesc &wd, int G, int bin_shift = 2);

// Floats of one bottom-row buffer of the block-split kernel (a power of two):
// a stripe's last lane writes its columns from the stripe's first column - 32
// to the band end of its last row, at most (H-1) num/den + 2w + 36 and at
// most m + 33 values (H = 32 x 24 rows).
inline int split_row_cap(const WorkDesc &wd)
{
    const int64_t H = 32 * 24;
    int64_t need = (int64_t)wd.m + 33;
    if (wd.den > 0) {
        const int64_t banded = ((H - 1) * wd.num + wd.den - 1) / wd.den + 2 * (int64_t)wd.w + 36;
        need = std::min(need, banded);
    }
    int64_t cap = 128;
    while (cap < need)
        cap <<= 1;
    return (int)cap;
}

inline void set_schedule(PlanItem &it, const Sched &s, int bin_shift = 2)
{
    it.wd.dC = s.dC;
    it.wd.a0 = s.a0;
    it.wd.s_end = s.s_end;
    it.cost = (double)s.s_end * kVariants[it.variant][0];
    it.cap = ring_need(it.wd, kVariants[it.variant][0], bin_shift);
}

// A batch lasts at least as long as its longest alignment on one group.  The
// batch's length is estimated as its cost-weighted lane-cell slots spread
// over the resident lanes (about 512 per SM).  Alignments start longest
// first.  With many alignments per resident group (about 32 groups per SM)
// the queue balances the load and only an alignment longer than the whole
// estimate sets the batch's length; with few (long reads: under 4 per
// group) each group runs one or two alignments, so any alignment above half
// the estimate is on the critical path.  Those move to the 32-lane variant
// with the best cost-weighted efficiency when that is shorter, so one group
// of 32 lanes finishes them in about half the time.  (Measured on a GB300:
// the half-estimate rule gives +15 % on 4,000 long reads and -10 % on 90,000
// uneven alignments, hence the switch.)
// Lane-cell slots (steps x lanes x rows, empty items as 0) per variant:
// integers, so the sums do not depend on how the items are split over threads.
inline void variant_slots(const PlanItem *items, size_t n, uint64_t out[kNumVariants])
{
    std::mutex mu;
    for (int v = 0; v < kNumVariants; ++v)
        out[v] = 0;
    parallel_for(n, [&](uint64_t lo, uint64_t hi) {
        uint64_t acc[kNumVariants] = {};
        for (uint64_t x = lo; x < hi; ++x)
            acc[items[x].variant] += (uint64_t)std::max(items[x].wd.s_end, 0) * kVariants[items[x].variant][0] *
                                     kVariants[items[x].variant][1];
        std::lock_guard<std::mutex> g(mu);
        for (int v = 0; v < kNumVariants; ++v)
            out[v] += acc[v];
    });
}

// slots: receives the lane-cell slots per variant after the pass.
inline void shorten_longest(PlanItem *items, size_t n, int sm_count, const double *cost, uint64_t slots[kNumVariants],
                            const PlanParams &pp = PlanParams())
{
    variant_slots(items, n, slots);
    double total = 0;
    for (int v = 0; v < kNumVariants; ++v)
        total += (double)slots[v] * cost[v];
    const double groups = 32.0 * std::max(sm_count, 1);
    const double theta = pp.latency_split > 0 ? pp.latency_split : ((double)n < 4.0 * groups ? 0.5 : 1.0);
    const double batch_len = theta * total / (512.0 * std::max(sm_count, 1));
    std::mutex mu;
    parallel_for(n, [&](uint64_t lo, uint64_t hi) {
        int64_t moved[kNumVariants] = {};
        bool any = false;
        for (uint64_t x = lo; x < hi; ++x) {
            PlanItem &it = items[x];
            const int v0 = it.variant;
            double dur = (double)it.wd.s_end * kVariants[v0][1] * cost[v0];
            const double split_len = pp.split_factor * total / (512.0 * std::max(sm_count, 1));
            if (it.wd.s_end <= 0 || dur <= std::min(batch_len, pp.split && pp.split_factor > 0 ? split_len : batch_len))
                continue;
            BandDef band;
            band.num = it.wd.num;
            band.den = it.wd.den;
            band.w = it.wd.w;
            band.m = it.wd.m;
            int best = -1;
            Sched best_s;
            if (kVariants[v0][0] != 32) {
                double best_score = -1;
                for (int v = 0; v < kNumVariants; ++v) {
                    if (kVariants[v][0] != 32)
                        continue;
                    Sched s = schedule(band, it.wd.row0, it.wd.nrows, 32, kVariants[v][1]);
                    const double score = s.eff / cost[v];
                    if (s.s_end > 0 && score > best_score) {
                        best_score = score;
                        best = v;
                        best_s = s;
                    }
                }
                if (best >= 0 && (double)best_s.s_end * kVariants[best][1] * cost[best] >= dur)
                    best = -1;
                if (best >= 0)
                    dur = (double)best_s.s_end * kVariants[best][1] * cost[best];
            }
            // the balanced length: the batch's work spread over every resident lane
            if (pp.split && pp.split_factor > 0 && dur > split_len) {
                // still longer than the batch on one warp: a block of four
                // warps takes it (the split kernel's lanes hold 24 rows)
                Sched s24 = schedule(band, it.wd.row0, it.wd.nrows, 32, 24);
                if (s24.s_end > 0) {
                    best = kSplitVariant;
                    best_s = s24;
                    it.split = true;
                }
            }
            if (best < 0)
                continue;
            moved[v0] -= (int64_t)it.wd.s_end * kVariants[v0][0] * kVariants[v0][1];
            it.variant = best;
            set_schedule(it, best_s, pp.ring_bin_shift);
            if (it.split)
                it.cap = split_row_cap(it.wd);
            moved[best] += (int64_t)std::max(it.wd.s_end, 0) * kVariants[best][0] * kVariants[best][1];
            any = true;
        }
        if (any) {
            std::lock_guard<std::mutex> g(mu);
            for (int v = 0; v < kNumVariants; ++v)
                slots[v] = (uint64_t)((int64_t)slots[v] + moved[v]);
        }
    });
}

// Sorts the items into launch order (variant, ring size, longest first) and
// cuts them into launch classes of one variant and one ring size, so that a
// few alignments with very wide bands do not force a large ring (and fewer
// resident blocks, or a ring in global memory) on everything else.  Classes
// are returned longest-alignment first.  Returns false if more than
// kMaxClasses would be needed.
inline bool make_classes(const PlanItem *items, size_t n, std::vector<int> &order, std::vector<ClassLaunch> &classes,
                         SortScratch &scr, bool longest_first = true)
{
    // Launch order: a stable LSD radix sort (16-bit digits) on one 64-bit key
    // per item, the bucket (variant, ring size, wave) above the complemented
    // step count, so ascending keys are longest first within a bucket and
    // equal keys keep item order.  Exact order by length matters: the groups
    // of a warp run in lockstep until the first of them finishes, so
    // neighbours in the queue should finish together.  With early termination
    // each bucket holds the reads' first candidates before the others.
    // Linear in the number of items and deterministic.
    constexpr int kCaps = 24;  // ring sizes 128 << i
    auto cap_index = [](int cap) {
        int i = 0;
        while (i < kCaps - 1 && (128ll << i) < cap)
            ++i;
        return i;
    };
    if (scr.key.size() < n) {
        scr.key.resize(n);
        scr.key2.resize(n);
        scr.tmp.resize(n);
    }
    if (order.size() < n)
        order.resize(n);
    uint64_t *key = scr.key.data(), *key2 = scr.key2.data();
    int *ord = order.data(), *tmp = scr.tmp.data();
    parallel_for(n, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t x = lo; x < hi; ++x) {
            const PlanItem &it = items[x];
            const uint64_t bucket = (uint64_t)(((it.split ? 512 : 0) + it.variant * kCaps + cap_index(it.cap)) * 2 +
                                               it.wave);
            // without longest_first (serving flushes of similar pieces) the
            // step counts do not take part in the order, only in max_cost
            key[x] = bucket << 32 | (longest_first ? (uint64_t)~(uint32_t)std::max(it.wd.s_end, 0) : 0u);
            ord[x] = (int)x;
        }
    });
    if (n <= 16384) {
        // small batches (serving flushes): the same stable LSD radix sort with
        // 8-bit digits on one thread, skipping the digits every key shares
        uint64_t diff = 0;
        for (size_t x = 1; x < n; ++x)
            diff |= key[x] ^ key[0];
        for (int shift = 0; shift < 64; shift += 8) {
            if (((diff >> shift) & 0xFF) == 0)
                continue;
            uint32_t c8[257] = {};
            for (size_t x = 0; x < n; ++x)
                ++c8[((key[x] >> shift) & 0xFF) + 1];
            for (int d = 0; d < 256; ++d)
                c8[d + 1] += c8[d];
            for (size_t x = 0; x < n; ++x) {
                const uint32_t y = c8[(key[x] >> shift) & 0xFF]++;
                key2[y] = key[x];
                tmp[y] = ord[x];
            }
            std::swap(key, key2);
            std::swap(ord, tmp);
        }
    }
    // each pass: per-chunk digit counts, offsets in (digit, chunk) order,
    // then every chunk scatters its items in order (stable)
    const size_t T = std::max<size_t>(1, std::min<size_t>(host_threads(), n / (1 << 16)));
    std::vector<uint32_t> cnt(n > 16384 ? (T << 16) : 0), tot(n > 16384 ? (1 << 16) : 0);
    auto chunks = [&](auto fn) { run_tasks((unsigned)T, [&](unsigned t) { fn((size_t)t); }); };
    for (int shift = 0; shift < 48 && n > 16384; shift += 16) {
        chunks([&](size_t t) {
            uint32_t *c = cnt.data() + (t << 16);
            std::fill(c, c + (1 << 16), 0u);
            for (size_t x = n * t / T; x < n * (t + 1) / T; ++x)
                ++c[(key[x] >> shift) & 0xFFFF];
        });
        uint64_t first_digit = 0;
        for (size_t t = 0; t < T; ++t)
            first_digit += cnt[(t << 16) + ((key[0] >> shift) & 0xFFFF)];
        if (first_digit == n)
            continue;  // one value of this digit: the pass would move nothing
        // offsets in (digit, chunk) order: each digit's total over the
        // chunks, an exclusive scan of the totals, then each digit's chunks
        chunks([&](size_t t) {
            for (size_t d = (t << 16) / T; d < ((t + 1) << 16) / T; ++d) {
                uint32_t sum = 0;
                for (size_t c = 0; c < T; ++c)
                    sum += cnt[(c << 16) + d];
                tot[d] = sum;
            }
        });
        uint32_t acc = 0;
        for (size_t d = 0; d < (1 << 16); ++d) {
            const uint32_t c = tot[d];
            tot[d] = acc;
            acc += c;
        }
        chunks([&](size_t t) {
            for (size_t d = (t << 16) / T; d < ((t + 1) << 16) / T; ++d) {
                uint32_t at = tot[d];
                for (size_t c = 0; c < T; ++c) {
                    const uint32_t v = cnt[(c << 16) + d];
                    cnt[(c << 16) + d] = at;
                    at += v;
                }
            }
        });
        chunks([&](size_t t) {
            uint32_t *c = cnt.data() + (t << 16);
            for (size_t x = n * t / T; x < n * (t + 1) / T; ++x) {
                const uint32_t y = c[(key[x] >> shift) & 0xFFFF]++;
                key2[y] = key[x];
                tmp[y] = ord[x];
            }
        });
        std::swap(key, key2);
        std::swap(ord, tmp);
    }
    if (ord != order.data())
        std::copy(ord, ord + n, order.data());
    // classes: runs of one (variant, ring size); a class's longest item heads
    // one of its two wave runs
    classes.clear();
    size_t pos = 0;
    while (pos < n) {
        const PlanItem &f = items[ord[pos]];
        ClassLaunch cl;
        cl.split = f.split;
        cl.G = kVariants[f.variant][0];
        cl.HR = kVariants[f.variant][1];
        cl.first = (int)pos;
        cl.ring_cap = f.cap;
        cl.max_cost = 0;
        const uint64_t id = key[pos] >> 33;
        for (; pos < n && (key[pos] >> 33) == id; ++pos) {
            if (!longest_first)
                cl.max_cost = std::max(cl.max_cost, (double)std::max(items[ord[pos]].wd.s_end, 0) * cl.G);
            else if ((int)pos == cl.first || (key[pos] >> 32) != (key[pos - 1] >> 32))
                cl.max_cost = std::max(cl.max_cost, (double)(uint32_t)~(uint32_t)key[pos] * cl.G);
        }
        cl.count = (int)pos - cl.first;
        classes.push_back(cl);
    }
    if (classes.size() > (size_t)kMaxClasses)
        return false;
    std::stable_sort(classes.begin(), classes.end(),
                     [](const ClassLaunch &x, const ClassLaunch &y) { return x.max_cost > y.max_cost; });
    return true;
}

inline bool make_classes(const std::vector<PlanItem> &items, std::vector<int> &order, std::vector<ClassLaunch> &classes,
                         bool longest_first = true)
{
    SortScratch scr;
    const bool ok = make_classes(items.data(), items.size(), order, classes, scr, longest_first);
    order.resize(items.size());
    return ok;
}

// make_classes, and when the ring sizes binned by powers of two would need
// more than kMaxClasses launches, the same with ring sizes binned by powers of
// four (the items' ring sizes are recomputed; the block-split ones keep theirs).
inline bool make_classes_binned(PlanItem *items, size_t n, std::vector<int> &order, std::vector<ClassLaunch> &classes,
                                SortScratch &scr, int bin_shift, bool longest_first = true)
{
    if (make_classes(items, n, order, classes, scr, longest_first))
        return true;
    if (bin_shift >= 2)
        return false;
    parallel_for(n, [&](uint64_t lo, uint64_t hi) {
        for (uint64_t x = lo; x < hi; ++x)
            if (!items[x].split)
                items[x].cap = ring_need(items[x].wd, kVariants[items[x].variant][0], 2);
    });
    return make_classes(items, n, order, classes, scr, longest_first);
}

// How a run's launch classes share the GPU.  With many alignments per
// resident group they queue as a programmatic dependent-launch chain on the
// stream, in the plan's order (longest class first): each class's blocks
// start as SM slots free up, and the order in which classes take the SMs is
// the planned one (measured on GB300: anchor-guided batches 21 -> 16.6 ms and
// steady, batched uneven 1.4 % faster).  With few alignments per group (long
// reads) every class should start at once, so they run as parallel branches
// on streams of their own (the chain measured 8-10 % slower on 4,000 long
// reads).
inline bool classes_as_chain(uint64_t n_work, int sm_count)
{
    return n_work >= 4ull * 32 * (uint64_t)std::max(sm_count, 1);
}

// Ring entries one piece needs: the stripe period plus two (written one step
// before read) and room for the stored row above (serving).
inline int ring_need(const WorkDesc &wd, int G, int bin_shift)
{
    int64_t need = std::max<int64_t>((int64_t)wd.dC + 2, (int64_t)wd.fin_wid + (int64_t)kLag * G + 4);
    // sizes in powers of 2^bin_shift (default four: 128, 512, 2048, ...):
    // coarser bins give fewer launch classes, finer ones smaller rings
    int64_t cap = 128;
    while (cap < need)
        cap <<= bin_shift;
    return (int)cap;
}

// Launch geometry of each class: ring in shared memory when it fits, grid of
// as many resident blocks as the SMs hold (capped by the work), and a global
// ring (from alloc(bytes)) otherwise.  Returns RA_OK, RA_ENOMEM or RA_EDEVICE.
template <typename Alloc>
int finalize_classes(int sm_count, std::vector<ClassLaunch> &classes, Alloc alloc)
{
    for (auto &cl : classes) {
        if (cl.split) {
            // one alignment per block; each block's warps hand their bottom
            // rows on through 2 buffers each of ring_cap floats in the arena
            const int nb = split_max_blocks_per_sm(cl.HR);
            if (nb <= 0)
                return RA_EDEVICE;
            cl.ring_in_smem = 0;
            cl.smem = split_smem_bytes();
            cl.grid = std::max(1, std::min(sm_count * nb, cl.count));
            while (!(cl.gring = (float *)alloc(sizeof(float) * (uint64_t)cl.grid * 4 * 2 * cl.ring_cap))) {
                if (cl.grid == 1)
                    return RA_ENOMEM;
                cl.grid = (cl.grid + 1) / 2;
            }
            continue;
        }
        const int gpb = kBlock / cl.G;
        const size_t smem = (size_t)gpb * (cl.ring_cap + 1) * sizeof(float);
        cl.ring_in_smem = smem <= kSmemRingLimit;
        cl.smem = cl.ring_in_smem ? smem : 0;
        const int nb = stripe_max_blocks_per_sm(cl.G, cl.HR, kBlock, cl.smem);
        if (nb <= 0)
            return RA_EDEVICE;
        cl.grid = std::max(1, std::min(sm_count * nb, (cl.count + gpb - 1) / gpb));
        if (!cl.ring_in_smem) {
            // ring scratch comes from the arena's free space: with less room,
            // fewer blocks (the persistent groups share the same queue)
            while (!(cl.gring = (float *)alloc(sizeof(float) * (uint64_t)cl.grid * gpb * cl.ring_cap))) {
                if (cl.grid == 1)
                    return RA_ENOMEM;
                cl.grid = (cl.grid + 1) / 2;
            }
        }
    }
    return RA_OK;
}

// serving entry points' helpers (serve.cu)
void serve_destroy(rawalign_dtw *h);
int serve_poll(rawalign_dtw *h, uint64_t ticket, rawalign_result_t *out, uint32_t cap, uint32_t *n_out,
               int64_t timeout_us, bool *handled);

}  // namespace ra_host
