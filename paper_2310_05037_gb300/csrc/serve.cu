// serve.cu -- Read-Until serving (Sec. 1, Sec. 3.1: decisions per chunk of
// signal while the read is still in the pore).
//
// A read is admitted on its first chunk, with its candidate regions, if a read
// slot is free and the arena can hold the read's device state: the expected
// signal of every candidate (Sup. A.1.1) and two frontier rows per candidate.
// The frontier is the band of the DTW row of the last event aligned so far;
// the next chunk resumes the DP from it (Sec. 2.2), so a chunked read gives the
// same DP as aligning its whole prefix at once.  Each chunk's cost is the
// minimum over its last row (FREE end: the read prefix against a longer
// reference window) and its score is B_Match * events so far - cost.
//
// submit_chunk only queues.  flush launches every queued chunk of every read
// as one batch (continuous batching): chunks that arrive while a flush is on
// the GPU go into the next flush, and the stream orders the flushes, so a
// read's chunk k+1 always sees the frontier chunk k wrote.  A read's memory
// and slot are returned when the flush carrying its last chunk completes.
#include <numeric>
#include <tuple>
#include <unordered_map>
#include <unordered_set>

#include "engine.h"
#include "serve_expand.cuh"

namespace ra_host {

struct ServeCand {
    BandDef band;
    int32_t w_report = 0;
    uint32_t m = 0;
    uint64_t r_off = 0;           // floats from the arena base: expected signal (m values)
    uint64_t fr_off[2] = {0, 0};  // floats from the arena base: frontier rows
    uint32_t fr_cap = 0;          // floats per frontier row
    SigDesc sig{};
    int cls = -1;                 // launch bucket (variant, ring size), set when the first chunk is planned
};

struct ServeRead {
    uint64_t read_id = 0;
    void *block = nullptr;  // arena block: candidate records, expected signals, frontiers
    uint64_t rec_off = 0;   // bytes from the arena base to the candidate records (the block's start)
    uint32_t rows_done = 0;
    std::vector<ServeCand> cands;
    bool signal_done = false;
    bool closed = false;
};

struct PendingChunk {
    uint64_t read_id = 0;
    std::vector<float> ev;
    std::vector<uint64_t> tickets;
    int last = 0;
};

// Pinned host staging buffers, reused across flushes (copies to and from
// pageable memory would make the host wait for the device).
struct PinnedPool {
    std::multimap<size_t, void *> free_;
    void *get(size_t bytes)
    {
        auto it = free_.lower_bound(bytes);
        if (it != free_.end()) {
            void *p = it->second;
            free_.erase(it);
            return p;
        }
        size_t cap = 1 << 16;
        while (cap < bytes)
            cap <<= 1;
        void *p = nullptr;
        if (cudaHostAlloc(&p, cap, cudaHostAllocDefault) != cudaSuccess)
            return nullptr;
        sizes_[p] = cap;
        return p;
    }
    void put(void *p)
    {
        if (p)
            free_.emplace(sizes_[p], p);
    }
    ~PinnedPool()
    {
        for (auto &kv : sizes_)
            cudaFreeHost(kv.first);
    }
    std::map<void *, size_t> sizes_;
};

struct FlushRec {
    cudaEvent_t done = nullptr;
    cudaEvent_t t_ev[3] = {nullptr, nullptr, nullptr};  // timing: start, inputs copied, kernels done
    std::vector<void *> blocks;
    rawalign_result_t *d_res = nullptr;
    rawalign_result_t *h_res = nullptr;  // pinned
    void *h_in = nullptr;                 // pinned inputs of this flush
    struct T {
        uint64_t ticket, read_id;
        uint32_t first, count;
        int last;
    };
    std::vector<T> tickets;
    std::vector<uint64_t> closing;  // reads whose memory is returned on completion
    uint32_t n_items = 0;           // per-candidate results in h_res
    bool reaped = false;
};

// Shape of a serving piece for the variant cache: rows, band slope and
// half-width, table width.
struct ShapeKey {
    int64_t rows, num, den, w, m;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(rows, num, den, w, m) < std::tie(o.rows, o.num, o.den, o.w, o.m);
    }
};

struct ServeState {
    int slots = 0;
    uint32_t max_events = 0;
    int max_cands = 0;
    int active = 0;
    std::unordered_map<uint64_t, ServeRead> reads;
    std::vector<PendingChunk> pending;  // [0, n_pending) are queued; later entries keep their buffers for reuse
    size_t n_pending = 0;
    std::map<uint64_t, FlushRec *> flushes;       // by flush id
    FlatMap64<uint64_t> ticket_flush;  // ticket -> flush id
    // reaped results: one block per flush, and per ticket its place in the block
    struct ReadyBlock {
        std::vector<rawalign_result_t> res;
        uint32_t left = 0;  // tickets not polled yet
    };
    struct ReadyRef {
        uint64_t fid;
        uint32_t first, count;
    };
    std::unordered_map<uint64_t, ReadyBlock> ready_blocks;  // by flush id
    FlatMap64<ReadyRef> ready;                              // by ticket
    std::vector<std::vector<rawalign_result_t>> res_pool;   // result buffers of polled blocks, for reuse
    void drop_block(std::unordered_map<uint64_t, ReadyBlock>::iterator b)
    {
        if (res_pool.size() < 8)
            res_pool.push_back(std::move(b->second.res));
        ready_blocks.erase(b);
    }
    // a flush's planning arrays, kept across flushes (no allocation, no
    // first-touch page faults once they have grown)
    struct FlushScratch {
        std::vector<ServeRead *> rds;
        std::vector<uint64_t> ev_first, item_first;
        std::vector<SigDesc> sig;
        std::vector<uint64_t> init_off;
        std::vector<ServeCandDev> init_rec;
        std::vector<ServeChunkDev> chunks;
        std::vector<int> cls_count, cls_map, cls_base;
        std::vector<ClassLaunch> classes;
    } scratch;
    FlatMap64<size_t> pending_at;                              // read id -> index in pending
    uint64_t next_flush = 1;
    PinnedPool pinned;
    std::vector<cudaEvent_t> timing_events;  // reusable timing events
    std::map<ShapeKey, int> shape_variant;   // variant chosen per piece shape
    rawalign_dtw_serve_stats_t stats{};
};

namespace {

ServeState *state(rawalign_dtw *h)
{
    if (!h->serve && h->cfg.serve_slots > 0) {
        h->serve = new (std::nothrow) ServeState();
        if (h->serve) {
            h->serve->slots = h->cfg.serve_slots;
            h->serve->max_events = h->cfg.serve_max_events > 0 ? (uint32_t)h->cfg.serve_max_events : 0;
            h->serve->max_cands = h->cfg.max_candidates > 0 ? h->cfg.max_candidates : 64;
            h->serve->reads.reserve(2 * (size_t)h->serve->slots);
            h->serve->ready.reserve(4 * (size_t)h->serve->slots);
            h->serve->ticket_flush.reserve(4 * (size_t)h->serve->slots);
            h->serve->pending_at.reserve(2 * (size_t)h->serve->slots);
        }
    }
    return h->serve;
}

void release_read(rawalign_dtw *h, ServeState *st, uint64_t read_id)
{
    auto it = st->reads.find(read_id);
    if (it == st->reads.end())
        return;
    h->arena.release(it->second.block);
    st->reads.erase(it);
    st->active--;
}

// Copies a completed flush's results to its tickets and returns its memory.
// Early reject (config.serve_early_reject): true when no candidate of the
// chunk can reach the threshold within max_events events.  Each candidate's
// best possible score is fl(fl(B * max_events) - cost): the cost of a FREE end
// never decreases as rows are added, and both roundings are monotone.
bool unreachable(const rawalign_result_t *r, uint32_t n, float b_match, uint32_t max_events, float thr)
{
    volatile float xb = b_match * (float)max_events;  // rounded once, never contracted with the subtraction
    for (uint32_t c = 0; c < n; ++c) {
        volatile float best = xb - r[c].cost;
        if (best >= thr)
            return false;
    }
    return true;
}

double ms_since(std::chrono::steady_clock::time_point t0);

void reap(rawalign_dtw *h, ServeState *st, uint64_t fid, FlushRec *f)
{
    if (f->reaped)
        return;
    const auto t_reap = std::chrono::steady_clock::now();
    const bool reject = h->cfg.serve_early_reject && st->max_events > 0;
#ifdef RAWALIGN_CHECKED
    // checked build: a work item of this flush failed its device-side checks
    const bool failed = f->n_items && ((const int *)(f->h_res + f->n_items))[0] != 0;
#else
    const bool failed = false;
#endif
    {
        // the flush's results in one block; each ticket refers to its part
        ServeState::ReadyBlock &blk = st->ready_blocks[fid];
        if (!st->res_pool.empty()) {
            blk.res = std::move(st->res_pool.back());
            st->res_pool.pop_back();
        }
        blk.res.assign(f->h_res, f->h_res + f->n_items);
        blk.left = (uint32_t)f->tickets.size();
        rawalign_result_t *res = blk.res.data();
        for (auto &t : f->tickets) {
            rawalign_result_t *v = res + t.first;
            const bool dead = reject && !t.last && t.count && v[0].decision == RA_PENDING &&
                              unreachable(v, t.count, h->cfg.b_match, st->max_events, h->cfg.score_threshold);
            for (uint32_t c = 0; c < t.count; ++c) {
                v[c].read_id = t.read_id;
                v[c].cand_idx = c;
                if ((t.last || dead) && v[c].decision == RA_PENDING)
                    v[c].decision = RA_UNMAPPED;
                if (failed)
                    v[c].status = RA_EDEVICE;
            }
            st->ready[t.ticket] = ServeState::ReadyRef{fid, t.first, t.count};
            st->ticket_flush.erase(t.ticket);
        }
        if (blk.left == 0)
            st->drop_block(st->ready_blocks.find(fid));
    }
    if (f->t_ev[0]) {
        float a = 0, b = 0, c = 0;
        if (cudaEventElapsedTime(&a, f->t_ev[0], f->t_ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, f->t_ev[1], f->t_ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&c, f->t_ev[2], f->done) == cudaSuccess) {
            st->stats.h2d_ms += a;
            st->stats.device_ms += b;
            st->stats.d2h_ms += c;
        }
        for (cudaEvent_t e : f->t_ev)
            st->timing_events.push_back(e);
    }
    for (uint32_t x = 0; x < f->n_items; ++x)
        st->stats.cells += f->h_res[x].cells;
    for (void *p : f->blocks)
        h->arena.release(p);
    f->blocks.clear();
    st->pinned.put(f->h_res);
    st->pinned.put(f->h_in);
    for (uint64_t r : f->closing)
        release_read(h, st, r);
    if (f->t_ev[0])
        st->timing_events.push_back(f->done);  // a timing event too
    else
        cudaEventDestroy(f->done);
    f->reaped = true;
    st->flushes.erase(fid);
    delete f;
    st->stats.host_reap_ms += ms_since(t_reap);
}

void reap_done(rawalign_dtw *h, ServeState *st)
{
    std::vector<uint64_t> ids;
    for (auto &kv : st->flushes)
        if (cudaEventQuery(kv.second->done) == cudaSuccess)
            ids.push_back(kv.first);
    for (uint64_t id : ids)
        reap(h, st, id, st->flushes[id]);
}

}  // namespace

void serve_destroy(rawalign_dtw *h)
{
    ServeState *st = h->serve;
    if (!st)
        return;
    cudaStreamSynchronize(h->stream);
    std::vector<uint64_t> ids;
    for (auto &kv : st->flushes)
        ids.push_back(kv.first);
    for (uint64_t id : ids)
        reap(h, st, id, st->flushes[id]);
    std::vector<uint64_t> rs;
    for (auto &kv : st->reads)
        rs.push_back(kv.first);
    for (uint64_t r : rs)
        release_read(h, st, r);
    for (cudaEvent_t e : st->timing_events)
        cudaEventDestroy(e);
    delete st;
    h->serve = nullptr;
}

// Copies up to cap results of a reaped ticket into out and forgets the
// ticket (and its flush's block once every ticket of the flush is taken).
uint32_t take_ready(ServeState *st, uint64_t ticket, rawalign_result_t *out, uint32_t cap)
{
    const ServeState::ReadyRef *r = st->ready.find(ticket);
    if (!r)
        return 0;
    const ServeState::ReadyRef ref = *r;
    st->ready.erase(ticket);
    auto b = st->ready_blocks.find(ref.fid);
    if (b == st->ready_blocks.end())
        return 0;
    const uint32_t n = std::min(cap, ref.count);
    if (n)
        memcpy(out, b->second.res.data() + ref.first, sizeof(rawalign_result_t) * n);
    if (--b->second.left == 0)
        st->drop_block(b);
    return n;
}

int serve_poll(rawalign_dtw *h, uint64_t ticket, rawalign_result_t *out, uint32_t cap, uint32_t *n_out,
               int64_t timeout_us, bool *handled)
{
    *handled = false;
    ServeState *st = h->serve;
    if (!st)
        return RA_OK;
    if (!st->ready.contains(ticket)) {
        const uint64_t *tf = st->ticket_flush.find(ticket);
        if (!tf) {
            // queued but not flushed yet?
            for (size_t ci = 0; ci < st->n_pending; ++ci)
                for (uint64_t t : st->pending[ci].tickets)
                    if (t == ticket) {
                        *handled = true;
                        return RA_ENOTREADY;
                    }
            return RA_OK;  // not a serving ticket
        }
        *handled = true;
        const uint64_t fid = *tf;
        FlushRec *f = st->flushes[fid];
        auto t0 = std::chrono::steady_clock::now();
        while (true) {
            cudaError_t e = cudaEventQuery(f->done);
            if (e == cudaSuccess)
                break;
            if (e != cudaErrorNotReady)
                return cuda_ok(e);
            if (timeout_us == 0)
                return RA_ENOTREADY;
            if (timeout_us > 0) {
                auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0);
                if (el.count() >= timeout_us)
                    return RA_ENOTREADY;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(10));
        }
        reap(h, st, fid, f);
        if (!st->ready.contains(ticket))
            return RA_EDEVICE;
    }
    *handled = true;
    *n_out = take_ready(st, ticket, out, cap);
    return RA_OK;
}

}  // namespace ra_host

namespace ra_host {
namespace {

// Queues one chunk (the body of rawalign_dtw_submit_chunk); nothing changes
// when it returns an error.
// No NaN or infinity among x[0, n): an exponent field of all ones, tested
// without an early exit so that the host compiler vectorises the loop.
bool all_finite(const float *x, uint32_t n)
{
    uint32_t bad = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, x + i, sizeof u);
        bad |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);
    }
    return bad == 0;
}

int submit_one(rawalign_dtw *h, ServeState *st, uint64_t read_id, const float *events, uint32_t n_events,
               const rawalign_candidate_t *cands, uint32_t n_cands, int last, uint64_t *ticket)
{
    if (!all_finite(events, n_events))
        return RA_EINVAL;
    auto it = st->reads.find(read_id);
    if (it == st->reads.end()) {
        // admission: a read slot and arena memory for the read's device state
        if (!cands || n_cands == 0 || (int)n_cands > st->max_cands)
            return RA_EINVAL;
        const int k = h->cfg.k;
        ServeRead rd;
        rd.read_id = read_id;
        rd.cands.reserve(n_cands);
        uint64_t floats = 0;
        for (uint32_t c = 0; c < n_cands; ++c) {
            const rawalign_candidate_t &cd = cands[c];
            if (cd.strand > 1 || cd.slope_den <= 0 || cd.slope_num < 0)
                return RA_EINVAL;
            if (cd.ref_offset > h->ref_len || cd.ref_len_bases > h->ref_len - cd.ref_offset ||
                (int64_t)cd.ref_len_bases < k || cd.ref_len_bases >= (1u << 30))
                return RA_EINVAL;
            ServeCand sc;
            sc.m = cd.ref_len_bases - k + 1;
            // rows are unknown until the read ends: the slope must be given;
            // n = 2 keeps the band rule from treating the piece as one row
            if (band_for(2, sc.m, cd.band_w, cd.slope_num, cd.slope_den, sc.band, sc.w_report) != 0)
                return RA_EINVAL;
            prepare_cell_count(sc.band);  // band_cells counts a chunk in O(1) away from the table's edges
            sc.fr_cap = (uint32_t)std::min<int64_t>(2 * sc.band.w + 2, (int64_t)sc.m + 1);
            sc.sig.ref_off = cd.ref_offset;
            sc.sig.len = cd.ref_len_bases;
            sc.sig.strand = cd.strand;
            floats += ((sc.m + 63) & ~63u) + 2ull * ((sc.fr_cap + 63) & ~63u);
            rd.cands.push_back(sc);
        }
        if (st->active >= st->slots)
            return RA_EAGAIN;
        // the block starts with the candidates' device records (the state
        // each chunk advances), then per candidate its expected signal and
        // its two frontier rows
        const uint64_t rec_floats = ((uint64_t)n_cands * sizeof(ServeCandDev) + 255) / 256 * 64;
        floats += rec_floats;
        rd.block = h->arena.alloc(floats * sizeof(float));
        if (!rd.block) {
            reap_done(h, st);
            rd.block = h->arena.alloc(floats * sizeof(float));
            if (!rd.block)
                return RA_EAGAIN;  // admission refused by free HBM in the arena
        }
        rd.rec_off = (uint64_t)((char *)rd.block - h->arena.base);
        uint64_t off = rd.rec_off / sizeof(float) + rec_floats;
        for (auto &sc : rd.cands) {
            sc.r_off = off;
            sc.sig.r_off = off;
            off += (sc.m + 63) & ~63u;
            sc.fr_off[0] = off;
            off += (sc.fr_cap + 63) & ~63u;
            sc.fr_off[1] = off;
            off += (sc.fr_cap + 63) & ~63u;
        }
        st->active++;
        it = st->reads.emplace(read_id, std::move(rd)).first;
    } else if (cands) {
        return RA_EINVAL;  // candidates come with the first chunk only
    }
    ServeRead &rd = it->second;
    if (rd.closed)
        return RA_EINVAL;
    // one pending chunk per read per flush: later chunks join it
    PendingChunk *pc = nullptr;
    if (const size_t *pa = st->pending_at.find(read_id))
        pc = &st->pending[*pa];
    uint64_t queued = pc ? pc->ev.size() : 0;
    if (st->max_events && rd.rows_done + queued + n_events > st->max_events)
        return RA_EINVAL;
    if (!pc) {
        if (st->n_pending == st->pending.size())
            st->pending.push_back(PendingChunk());
        pc = &st->pending[st->n_pending];
        st->pending_at[read_id] = st->n_pending++;
        pc->ev.clear();
        pc->tickets.clear();
        pc->last = 0;
        pc->read_id = read_id;
    }
    pc->ev.insert(pc->ev.end(), events, events + n_events);
    pc->last = pc->last || last;
    if (last)
        rd.closed = true;
    uint64_t t = h->next_id++;
    pc->tickets.push_back(t);
    *ticket = t;
    return RA_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace ra_host

extern "C" int rawalign_dtw_submit_chunk(rawalign_dtw_t *h, uint64_t read_id, const float *events, uint32_t n_events,
                                         const rawalign_candidate_t *cands, uint32_t n_cands, int last,
                                         uint64_t *ticket)
{
    NvtxRange nvtx_range("rawalign_dtw_submit_chunk");
    if (!h || !ticket || (n_events && !events))
        return RA_EINVAL;
    ServeState *st = state(h);
    if (!st)
        return RA_EINVAL;  // serving not configured (serve_slots == 0)
    const auto t0 = std::chrono::steady_clock::now();
    cudaSetDevice(h->device);
    const int rc = submit_one(h, st, read_id, events, n_events, cands, n_cands, last, ticket);
    st->stats.host_submit_ms += ms_since(t0);
    return rc;
}

extern "C" int rawalign_dtw_submit_chunks(rawalign_dtw_t *h, const rawalign_chunk_t *chunks, uint32_t n_chunks,
                                          const float *events, const rawalign_candidate_t *cands, uint64_t *tickets,
                                          int32_t *status)
{
    NvtxRange nvtx_range("rawalign_dtw_submit_chunks");
    if (!h || (n_chunks && (!chunks || !tickets || !status)))
        return RA_EINVAL;
    ServeState *st = state(h);
    if (!st)
        return RA_EINVAL;
    for (uint32_t c = 0; c < n_chunks; ++c)
        if ((chunks[c].n_events && !events) || (chunks[c].n_cands && !cands))
            return RA_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    cudaSetDevice(h->device);
    for (uint32_t c = 0; c < n_chunks; ++c) {
        const rawalign_chunk_t &ch = chunks[c];
        tickets[c] = 0;
        status[c] = submit_one(h, st, ch.read_id, ch.n_events ? events + ch.ev_offset : nullptr, ch.n_events,
                               ch.n_cands ? cands + ch.cand_offset : nullptr, ch.n_cands, ch.last, &tickets[c]);
        if (status[c] != RA_OK)
            tickets[c] = 0;
    }
    st->stats.host_submit_ms += ms_since(t0);
    return RA_OK;
}

namespace {
int flush_impl(rawalign_dtw *h, ServeState *st);
}

extern "C" int rawalign_dtw_flush(rawalign_dtw_t *h)
{
    NvtxRange nvtx_range("rawalign_dtw_flush");
    if (!h)
        return RA_EINVAL;
    ServeState *st = h->serve;
    if (!st)
        return RA_OK;
    const auto t0 = std::chrono::steady_clock::now();
    cudaSetDevice(h->device);
    const int rc = flush_impl(h, st);
    st->stats.host_flush_ms += ms_since(t0);
    return rc;
}

namespace {
int flush_impl(rawalign_dtw *h, ServeState *st)
{
    reap_done(h, st);
    if (st->n_pending == 0)
        return RA_OK;
    const auto t_plan = std::chrono::steady_clock::now();
    // plan: the host places every chunk's events and pieces (prefix sums),
    // registers its tickets, gives each new candidate its variant and launch
    // bucket and counts the pieces per bucket; the device then builds each
    // piece's work record from the chunk record and the candidate's carried
    // state (serve_piece), so nothing here is done per piece
    FlushRec *f = new FlushRec();
    ServeState::FlushScratch &sc_ = st->scratch;
    const size_t n_pend = st->n_pending;
    const int n_keys_cls = kNumVariants * kServeCaps;
    std::vector<ServeRead *> &rds = sc_.rds;
    std::vector<uint64_t> &ev_first = sc_.ev_first, &item_first = sc_.item_first;
    std::vector<SigDesc> &sig = sc_.sig;
    std::vector<uint64_t> &init_off = sc_.init_off;
    std::vector<ServeCandDev> &init_rec = sc_.init_rec;
    std::vector<ServeChunkDev> &chunks = sc_.chunks;
    std::vector<int> &cls_count = sc_.cls_count, &cls_map = sc_.cls_map, &cls_base = sc_.cls_base;
    rds.resize(n_pend);
    ev_first.assign(n_pend + 1, 0);
    item_first.assign(n_pend + 1, 0);
    sig.clear();
    init_off.clear();
    init_rec.clear();
    chunks.resize(n_pend);
    cls_count.assign(n_keys_cls, 0);
    // ring sizes of serving buckets: powers of four at least, so that the
    // buckets of ten variants stay few
    const int bin_shift = std::max(2, h->plan.ring_bin_shift);
    for (size_t ci = 0; ci < n_pend; ++ci) {
        const PendingChunk &pc = st->pending[ci];
        ServeRead &rd = st->reads.at(pc.read_id);
        rds[ci] = &rd;
        const uint64_t nrows = pc.ev.size();
        const uint32_t count = nrows ? (uint32_t)rd.cands.size() : 0;  // a close-only chunk returns nothing
        ev_first[ci + 1] = ev_first[ci] + nrows;
        item_first[ci + 1] = item_first[ci] + count;
        for (uint64_t t : pc.tickets)
            f->tickets.push_back({t, pc.read_id, (uint32_t)item_first[ci], count, pc.last});
        if (pc.last)
            f->closing.push_back(pc.read_id);
        ServeChunkDev &ch = chunks[ci];
        ch.ev_off = ev_first[ci];
        ch.cand_off = rd.rec_off;
        ch.n_cands = count;
        ch.first_piece = (uint32_t)item_first[ci];
        ch.row0 = (int32_t)rd.rows_done;
        ch.nrows = (int32_t)nrows;
        for (uint32_t c = 0; c < count; ++c) {
            ServeCand &sc = rd.cands[c];
            if (sc.cls < 0) {
                // first chunk of the candidate: its variant (cached per shape
                // across reads) and its launch bucket, then its device record
                const ShapeKey key{(int64_t)nrows, sc.band.num, sc.band.den, sc.band.w, sc.band.m};
                int v;
                auto hit = st->shape_variant.find(key);
                if (hit != st->shape_variant.end()) {
                    v = hit->second;
                } else {
                    Sched sch;
                    v = choose_variant(sc.band, rd.rows_done, (int64_t)nrows, sch, h->slot_cost);
                    if (st->shape_variant.size() < 4096)
                        st->shape_variant[key] = v;
                }
                const int G = kVariants[v][0], HR = kVariants[v][1];
                const int64_t H = (int64_t)G * HR;
                int64_t span = fdiv(2 * sc.band.w * sc.band.den - (H - HR + 1) * sc.band.num, sc.band.den);
                span = std::min<int64_t>(span, sc.band.m - 1);
                const int64_t dC = std::max<int64_t>((int64_t)kLag * G + 3, span + 2);
                // ring: the stripe period and the widest stored row above
                const int64_t need =
                    std::max<int64_t>(dC + 2, std::min<int64_t>(2 * sc.band.w, sc.band.m - 1) + (int64_t)kLag * G + 4);
                // (admission keeps m below 2^30, so 2^30 entries always suffice)
                int cap_i = 0;
                while ((128ll << cap_i) < need && cap_i < kServeCaps - 1)
                    cap_i = std::min(cap_i + bin_shift, kServeCaps - 1);
                sc.cls = v * kServeCaps + cap_i;
                ServeCandDev d{};
                d.r_off = sc.r_off;
                d.fr_off[0] = sc.fr_off[0];
                d.fr_off[1] = sc.fr_off[1];
                d.num = sc.band.num;
                d.den = sc.band.den;
                d.per = sc.band.per;
                d.hi_row = sc.band.hi_row;
                d.m = (int32_t)sc.m;
                d.w = (int32_t)sc.band.w;
                d.w_report = sc.w_report;
                d.G = G;
                d.HR = HR;
                d.dC = (int32_t)dC;
                d.cls = sc.cls;
                d.cur = 0;
                d.fr_lo = -1;
                d.fr_wid = 0;
                d.dead = 0;
                init_off.push_back(rd.rec_off + (uint64_t)c * sizeof(ServeCandDev));
                init_rec.push_back(d);
            }
            if (!rd.signal_done)
                sig.push_back(sc.sig);
            cls_count[sc.cls]++;
        }
    }
    const uint32_t chunk_idx = (uint32_t)n_pend;
    const uint64_t n_ev = ev_first[n_pend];
    const uint32_t n_items = (uint32_t)item_first[n_pend];
    if (n_items == 0) {
        // only close-only chunks: nothing to run
        f->h_res = nullptr;
        RA_CUDA(cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming));
        RA_CUDA(cudaEventRecord(f->done, h->stream));
        const uint64_t fid = st->next_flush++;
        st->flushes[fid] = f;
        for (auto &t : f->tickets)
            st->ticket_flush[t.ticket] = fid;
        st->n_pending = 0;
        st->pending_at.clear();
        return RA_OK;
    }
    // launch classes: one per bucket in use, its pieces contiguous in the
    // work array; with more buckets than launches, one class per variant with
    // the variant's largest ring
    std::vector<ClassLaunch> &classes = sc_.classes;
    classes.clear();
    cls_map.assign(n_keys_cls, 0);
    cls_base.clear();
    int n_used = 0;
    for (int key = 0; key < n_keys_cls; ++key)
        n_used += cls_count[key] > 0;
    const bool per_variant = n_used > kMaxClasses;
    {
        for (int v = 0; v < kNumVariants; ++v) {
            int merged = -1;
            for (int ci = 0; ci < kServeCaps; ++ci) {
                const int key = v * kServeCaps + ci;
                if (!cls_count[key])
                    continue;
                if (per_variant && merged >= 0) {
                    ClassLaunch &cl = classes[merged];
                    cl.count += cls_count[key];
                    cl.ring_cap = 128 << ci;  // keys ascend: the largest ring so far
                    cl.max_cost = cl.count;
                    cls_map[key] = merged;
                    continue;
                }
                ClassLaunch cl;
                cl.G = kVariants[v][0];
                cl.HR = kVariants[v][1];
                cl.ring_cap = 128 << ci;
                cl.count = cls_count[key];
                cl.max_cost = cl.count;
                cls_map[key] = (int)classes.size();
                if (per_variant)
                    merged = (int)classes.size();
                classes.push_back(cl);
            }
        }
        int base = 0;
        for (auto &cl : classes) {
            cl.first = base;
            cls_base.push_back(base);
            base += cl.count;
        }
    }
    const int n_classes = (int)classes.size();
    // device memory for this flush
    auto take = [&](uint64_t bytes) -> void * {
        void *p = h->arena.alloc(std::max<uint64_t>(bytes, 256));
        if (p)
            f->blocks.push_back(p);
        return p;
    };
    // the flush's inputs live in one arena block and travel in one copy:
    // events, signal descriptors, new candidates, chunk records, the bucket
    // map and bases, and the zeroed bucket counters, per-chunk best keys and
    // queue counters; the work records and read slots that the device builds
    // follow in the same block
    auto al256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t n_init = init_off.size();
    const size_t b_ev = sizeof(float) * n_ev, b_sig = sizeof(SigDesc) * sig.size();
    const size_t b_iidx = sizeof(uint64_t) * n_init, b_irec = sizeof(ServeCandDev) * n_init;
    const size_t b_ch = sizeof(ServeChunkDev) * n_pend, b_map = sizeof(int) * n_keys_cls;
    const size_t b_base = sizeof(int) * (size_t)std::max(n_classes, 1), b_fill = b_base;
    const size_t b_keys = sizeof(unsigned long long) * chunk_idx, b_q = sizeof(int) * (kMaxClasses + 2);
    const size_t b_work = sizeof(WorkDesc) * n_items, b_rd = sizeof(int) * n_items;
    const size_t o_sig = al256(b_ev), o_iidx = o_sig + al256(b_sig), o_irec = o_iidx + al256(b_iidx);
    const size_t o_ch = o_irec + al256(b_irec), o_map = o_ch + al256(b_ch), o_base = o_map + al256(b_map);
    const size_t o_fill = o_base + al256(b_base), o_keys = o_fill + al256(b_fill), o_q = o_keys + al256(b_keys);
    const size_t in_bytes = o_q + al256(b_q);  // copied from the host
    const size_t o_work = in_bytes, o_rd = o_work + al256(b_work), all_bytes = o_rd + al256(b_rd);
    char *d_in = (char *)take(all_bytes);
    f->d_res = (rawalign_result_t *)take(sizeof(rawalign_result_t) * n_items);
    bool ok = d_in && f->d_res;
    if (ok)
        ok = finalize_classes(h->sm_count, classes, take) == RA_OK;
    if (ok) {
        f->h_in = st->pinned.get(in_bytes);
        f->h_res = (rawalign_result_t *)st->pinned.get(sizeof(rawalign_result_t) * (n_items + 1));
        ok = f->h_in && f->h_res;
    }
    if (!ok) {
        // nothing was launched and no host state advanced
        for (void *p : f->blocks)
            h->arena.release(p);
        st->pinned.put(f->h_in);
        st->pinned.put(f->h_res);
        // the new candidates are planned again with the next flush
        for (size_t ci = 0; ci < n_pend; ++ci)
            if (!rds[ci]->signal_done)
                for (auto &sc : rds[ci]->cands)
                    sc.cls = -1;
        delete f;
        return RA_ENOMEM;
    }
    char *hin = (char *)f->h_in;
    for (size_t ci = 0; ci < n_pend; ++ci) {
        const PendingChunk &pc = st->pending[ci];
        if (!pc.ev.empty())
            memcpy(hin + sizeof(float) * ev_first[ci], pc.ev.data(), sizeof(float) * pc.ev.size());
    }
    if (b_sig)
        memcpy(hin + o_sig, sig.data(), b_sig);
    if (n_init) {
        memcpy(hin + o_iidx, init_off.data(), b_iidx);
        memcpy(hin + o_irec, init_rec.data(), b_irec);
    }
    memcpy(hin + o_ch, chunks.data(), b_ch);
    memcpy(hin + o_map, cls_map.data(), b_map);
    memcpy(hin + o_base, cls_base.data(), sizeof(int) * n_classes);
    memset(hin + o_fill, 0, in_bytes - o_fill);
    float *d_ev = (float *)d_in;
    SigDesc *d_sig = (SigDesc *)(d_in + o_sig);
    WorkDesc *d_work = (WorkDesc *)(d_in + o_work);
    int *d_read_of = (int *)(d_in + o_rd);
    unsigned long long *d_keys = (unsigned long long *)(d_in + o_keys);
    int *d_queue = (int *)(d_in + o_q);
    cudaStream_t s = h->stream;
    const auto t_launch = std::chrono::steady_clock::now();
    st->stats.host_plan_ms += std::chrono::duration<double, std::milli>(t_launch - t_plan).count();
    // timing events (start, inputs copied, kernels done, done), reused
    while (st->timing_events.size() < 4) {
        cudaEvent_t e = nullptr;
        RA_CUDA(cudaEventCreate(&e));
        st->timing_events.push_back(e);
    }
    for (int q = 0; q < 3; ++q) {
        f->t_ev[q] = st->timing_events.back();
        st->timing_events.pop_back();
    }
    f->done = st->timing_events.back();
    st->timing_events.pop_back();
    RA_CUDA(cudaEventRecord(f->t_ev[0], s));
    RA_CUDA(cudaMemcpyAsync(d_in, hin, in_bytes, cudaMemcpyHostToDevice, s));
    RA_CUDA(cudaEventRecord(f->t_ev[1], s));
    float *abase = (float *)h->arena.base;
    RA_CUDA(launch_serve_init(h->arena.base, (const uint64_t *)(d_in + o_iidx), (const ServeCandDev *)(d_in + o_irec),
                              (int)n_init, s));
    if (!sig.empty())
        RA_CUDA(launch_expected_signal(d_sig, (int)sig.size(), h->d_ref, h->d_pore, h->cfg.k, abase, s));
    RA_CUDA(launch_serve_expand((const ServeChunkDev *)(d_in + o_ch), (int)n_pend, h->arena.base,
                                (const int *)(d_in + o_map), (const int *)(d_in + o_base), (int *)(d_in + o_fill),
                                d_work, d_read_of, s));
    // launch classes: a dependent-launch chain on the stream, or parallel
    // branches (classes_as_chain)
    const bool chain = classes_as_chain(n_items, h->sm_count);
    if (!chain)
        RA_CUDA(cudaEventRecord(h->fork, s));
    for (int ci = 0; ci < n_classes; ++ci) {
        auto &cl = classes[ci];
        cudaStream_t cs = chain ? s : h->aux[ci];
        if (!chain)
            RA_CUDA(cudaStreamWaitEvent(cs, h->fork, 0));
        StripeParams p{};
        p.work = d_work + cl.first;
        p.n_work = cl.count;
        p.queue = d_queue + ci;
        p.events = d_ev;
        p.r_all = abase;
        p.fstore = abase;
        p.fstore_out = abase;
        p.results = f->d_res;
        p.best_keys = d_keys;
        p.gring = cl.gring;
        p.ring_cap = cl.ring_cap;
        p.ring_in_smem = cl.ring_in_smem;
        p.b_match = h->cfg.b_match;
        p.end_free = 1;
        p.err = d_queue + kMaxClasses;
        p.n_events = n_ev;
        p.n_r = h->arena.size / sizeof(float);
        p.n_fstore = h->arena.size / sizeof(float);
        p.n_results = (int)n_items;
        p.n_keys = (int)chunk_idx;
        RA_CUDA(launch_stripe(cl.G, cl.HR, p, cl.grid, kBlock, cl.smem, cs, chain && ci > 0));
        if (!chain) {
            RA_CUDA(cudaEventRecord(h->join[ci], cs));
            RA_CUDA(cudaStreamWaitEvent(s, h->join[ci], 0));
        }
    }
    RA_CUDA(launch_decide(f->d_res, (int)n_items, d_keys, d_read_of, h->cfg.score_threshold, 0, s));
    RA_CUDA(cudaEventRecord(f->t_ev[2], s));
    f->n_items = n_items;
    RA_CUDA(cudaMemcpyAsync(f->h_res, f->d_res, sizeof(rawalign_result_t) * n_items, cudaMemcpyDeviceToHost, s));
#ifdef RAWALIGN_CHECKED
    // the kernels' error word travels back behind the results
    RA_CUDA(cudaMemcpyAsync(f->h_res + n_items, d_queue + kMaxClasses, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
#endif
    RA_CUDA(cudaEventRecord(f->done, s));
    // launched: advance the host-side read state (the candidates' frontier
    // state advances on the device)
    for (size_t ci = 0; ci < n_pend; ++ci) {
        ServeRead &rd = *rds[ci];
        rd.signal_done = true;
        rd.rows_done += (uint32_t)st->pending[ci].ev.size();
    }
    st->stats.host_launch_ms += ms_since(t_launch);
    st->stats.flushes++;
    st->stats.chunks += chunk_idx;
    st->stats.pieces += n_items;
    const uint64_t fid = st->next_flush++;
    st->flushes[fid] = f;
    for (auto &t : f->tickets)
        st->ticket_flush[t.ticket] = fid;
    st->n_pending = 0;
    st->pending_at.clear();
    return RA_OK;
}
}  // namespace

extern "C" int rawalign_dtw_poll_chunks(rawalign_dtw_t *h, const uint64_t *tickets, uint32_t n_tickets,
                                        rawalign_result_t *out, uint32_t cap, uint32_t *counts, int64_t timeout_us)
{
    NvtxRange nvtx_range("rawalign_dtw_poll_chunks");
    if (!h || (n_tickets && (!tickets || !counts)) || (cap && !out))
        return RA_EINVAL;
    ServeState *st = h->serve;
    if (!st)
        return RA_EINVAL;
    cudaSetDevice(h->device);
    // every ticket known and named once; the flushes still to wait for
    {
        std::vector<uint64_t> sorted(tickets, tickets + n_tickets);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return RA_EINVAL;
    }
    std::vector<uint64_t> wait_for;
    for (uint32_t x = 0; x < n_tickets; ++x) {
        const uint64_t t = tickets[x];
        if (st->ready.contains(t))
            continue;
        if (const uint64_t *tf = st->ticket_flush.find(t)) {
            wait_for.push_back(*tf);
            continue;
        }
        for (size_t ci = 0; ci < st->n_pending; ++ci)
            for (uint64_t q : st->pending[ci].tickets)
                if (q == t)
                    return RA_ENOTREADY;  // queued, not flushed: waiting would not help
        return RA_EINVAL;
    }
    std::sort(wait_for.begin(), wait_for.end());
    wait_for.erase(std::unique(wait_for.begin(), wait_for.end()), wait_for.end());
    const auto t0 = std::chrono::steady_clock::now();
    for (uint64_t fid : wait_for) {
        FlushRec *f = st->flushes[fid];
        while (true) {
            cudaError_t e = cudaEventQuery(f->done);
            if (e == cudaSuccess)
                break;
            if (e != cudaErrorNotReady)
                return cuda_ok(e);
            if (timeout_us == 0)
                return RA_ENOTREADY;
            if (timeout_us < 0) {
                RA_CUDA(cudaEventSynchronize(f->done));
                break;
            }
            if (ms_since(t0) * 1e3 >= (double)timeout_us)
                return RA_ENOTREADY;
            std::this_thread::yield();
        }
    }
    for (uint64_t fid : wait_for) {
        auto it = st->flushes.find(fid);
        if (it != st->flushes.end())
            reap(h, st, fid, it->second);
    }
    uint64_t total = 0;
    for (uint32_t x = 0; x < n_tickets; ++x) {
        const ServeState::ReadyRef *r = st->ready.find(tickets[x]);
        if (!r)
            return RA_EDEVICE;
        total += r->count;
    }
    if (total > cap)
        return RA_EINVAL;
    uint64_t pos = 0;
    for (uint32_t x = 0; x < n_tickets; ++x) {
        const uint32_t n = take_ready(st, tickets[x], out + pos, UINT32_MAX);
        counts[x] = n;
        pos += n;
    }
    return RA_OK;
}

extern "C" int rawalign_dtw_serve_stats(rawalign_dtw_t *h, rawalign_dtw_serve_stats_t *out, int reset)
{
    if (!h || !out)
        return RA_EINVAL;
    ServeState *st = h->serve;
    if (!st) {
        memset(out, 0, sizeof *out);
        return RA_OK;
    }
    *out = st->stats;
    if (reset)
        memset(&st->stats, 0, sizeof st->stats);
    return RA_OK;
}
