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

namespace ra_host {

struct ServeCand {
    BandDef band;
    int32_t w_report = 0;
    uint64_t r_off = 0;     // floats from the arena base: expected signal (m values)
    uint64_t fr_off[2] = {0, 0};  // floats from the arena base: frontier rows
    uint32_t fr_cap = 0;    // floats per frontier row
    int cur = 0;            // frontier holding the last processed row
    int32_t fr_lo = -1, fr_wid = 0;  // its band (first column, width - 1)
    uint32_t m = 0;
    bool dead = false;      // the band has left the table: no cell any more
    SigDesc sig{};
    int64_t plan_rows = -1; // chunk height of the cached variant choice
    int plan_variant = 0;   // variant chosen for chunks of plan_rows rows
    ChunkSched csched;      // schedule of the next chunk of plan_rows rows, stepped without divisions
};

struct ServeRead {
    uint64_t read_id = 0;
    void *block = nullptr;  // arena block: expected signals + frontiers
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
    std::unordered_map<uint64_t, uint64_t> ticket_flush;  // ticket -> flush id
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
    std::unordered_map<uint64_t, ReadyRef> ready;           // by ticket
    std::vector<std::vector<rawalign_result_t>> res_pool;   // result buffers of polled blocks, for reuse
    void drop_block(std::unordered_map<uint64_t, ReadyBlock>::iterator b)
    {
        if (res_pool.size() < 8)
            res_pool.push_back(std::move(b->second.res));
        ready_blocks.erase(b);
    }
    // a flush's planning arrays, kept across flushes (no allocation, no
    // first-touch page faults once they have grown)
    struct Update {  // host state advanced only once the flush is launched
        ServeCand *sc;
        int32_t fr_lo, fr_wid;
        bool dead;
    };
    struct FlushScratch {
        std::vector<ServeRead *> rds;
        std::vector<uint64_t> ev_first, item_first, sig_first;
        std::vector<SigDesc> sig;
        std::vector<PlanItem> items;
        std::vector<int> read_of;
        std::vector<Update> updates;
        std::vector<int> order;
        std::vector<ClassLaunch> classes;
        SortScratch sort;
    } scratch;
    std::unordered_map<uint64_t, size_t> pending_at;           // read id -> index in pending
    uint64_t next_flush = 1;
    PinnedPool pinned;
    std::vector<cudaEvent_t> timing_events;  // reusable timing events
    std::map<ShapeKey, int> shape_variant;   // variant chosen per piece shape
    std::mutex shape_mu;                     // guards shape_variant while a flush plans in parallel
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
uint32_t take_ready(ServeState *st, std::unordered_map<uint64_t, ServeState::ReadyRef>::iterator r,
                    rawalign_result_t *out, uint32_t cap)
{
    const ServeState::ReadyRef ref = r->second;
    st->ready.erase(r);
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
    auto r = st->ready.find(ticket);
    if (r == st->ready.end()) {
        auto tf = st->ticket_flush.find(ticket);
        if (tf == st->ticket_flush.end()) {
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
        FlushRec *f = st->flushes[tf->second];
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
        reap(h, st, tf->second, f);
        r = st->ready.find(ticket);
        if (r == st->ready.end())
            return RA_EDEVICE;
    }
    *handled = true;
    *n_out = take_ready(st, r, out, cap);
    return RA_OK;
}

}  // namespace ra_host

namespace ra_host {
namespace {

// Queues one chunk (the body of rawalign_dtw_submit_chunk); nothing changes
// when it returns an error.
int submit_one(rawalign_dtw *h, ServeState *st, uint64_t read_id, const float *events, uint32_t n_events,
               const rawalign_candidate_t *cands, uint32_t n_cands, int last, uint64_t *ticket)
{
    for (uint32_t x = 0; x < n_events; ++x)
        if (!std::isfinite(events[x]))
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
        rd.block = h->arena.alloc(floats * sizeof(float));
        if (!rd.block) {
            reap_done(h, st);
            rd.block = h->arena.alloc(floats * sizeof(float));
            if (!rd.block)
                return RA_EAGAIN;  // admission refused by free HBM in the arena
        }
        uint64_t off = (uint64_t)((char *)rd.block - h->arena.base) / sizeof(float);
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
    auto pa = st->pending_at.find(read_id);
    if (pa != st->pending_at.end())
        pc = &st->pending[pa->second];
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
    // plan: one piece of work per (chunk, candidate).  A first pass places
    // every chunk's events, pieces and signal descriptors (prefix sums) and
    // registers its tickets; the second fills the records (on the host
    // worker threads when the flush is large).  Each read has at most one
    // pending chunk, so the chunks touch disjoint read state; only the
    // handle-wide shape cache is shared (under a lock).
    FlushRec *f = new FlushRec();
    using Update = ServeState::Update;
    ServeState::FlushScratch &sc_ = st->scratch;
    const size_t n_pend = st->n_pending;
    std::vector<ServeRead *> &rds = sc_.rds;
    std::vector<uint64_t> &ev_first = sc_.ev_first, &item_first = sc_.item_first, &sig_first = sc_.sig_first;
    rds.resize(n_pend);
    ev_first.assign(n_pend + 1, 0);
    item_first.assign(n_pend + 1, 0);
    sig_first.assign(n_pend + 1, 0);
    for (size_t ci = 0; ci < n_pend; ++ci) {
        const PendingChunk &pc = st->pending[ci];
        ServeRead &rd = st->reads.at(pc.read_id);
        rds[ci] = &rd;
        const uint64_t nrows = pc.ev.size();
        const uint64_t count = nrows ? rd.cands.size() : 0;  // a close-only chunk returns nothing
        ev_first[ci + 1] = ev_first[ci] + nrows;
        item_first[ci + 1] = item_first[ci] + count;
        sig_first[ci + 1] = sig_first[ci] + (rd.signal_done ? 0 : count);
        for (uint64_t t : pc.tickets)
            f->tickets.push_back({t, pc.read_id, (uint32_t)item_first[ci], (uint32_t)count, pc.last});
        if (pc.last)
            f->closing.push_back(pc.read_id);
    }
    const uint32_t chunk_idx = (uint32_t)n_pend;
    const uint64_t n_ev = ev_first[n_pend];
    std::vector<SigDesc> &sig = sc_.sig;
    std::vector<PlanItem> &items = sc_.items;
    std::vector<int> &read_of = sc_.read_of;
    std::vector<Update> &updates = sc_.updates;
    sig.resize(sig_first[n_pend]);
    items.resize(item_first[n_pend]);
    read_of.resize(item_first[n_pend]);
    updates.resize(item_first[n_pend]);
    auto plan_chunk = [&](size_t ci) {
        const PendingChunk &pc = st->pending[ci];
        ServeRead &rd = *rds[ci];
        const uint32_t row0 = rd.rows_done, nrows = (uint32_t)pc.ev.size();
        const uint64_t ev_off = ev_first[ci];
        const uint32_t first = (uint32_t)item_first[ci];
        const uint32_t count = (uint32_t)(item_first[ci + 1] - first);
        for (uint32_t c = 0; c < count; ++c) {
            ServeCand &sc = rd.cands[c];
            if (!rd.signal_done)
                sig[sig_first[ci] + c] = sc.sig;
            PlanItem &it = items[first + c];
            memset(&it.wd, 0, sizeof(WorkDesc));
            it.wave = 0;
            it.split = false;
            WorkDesc &wd = it.wd;
            wd.ev_off = ev_off;
            wd.r_off = sc.r_off;
            wd.num = sc.band.num;
            wd.den = sc.band.den;
            wd.row0 = (int32_t)row0;
            wd.nrows = (int32_t)nrows;
            wd.m = (int32_t)sc.m;
            wd.w = (int32_t)sc.band.w;
            wd.cand = (int32_t)(first + c);
            wd.read = (int32_t)ci;
            wd.n_read = (int32_t)(row0 + nrows);
            wd.w_report = sc.w_report;
            if (row0 == 0) {
                wd.fin_off = ~0ull;
                wd.fin_lo = -1;
                wd.fin_wid = 0;
            } else {
                wd.fin_off = sc.fr_off[sc.cur];
                wd.fin_lo = sc.fr_lo;
                wd.fin_wid = sc.fr_wid;
            }
            wd.fout_off = sc.fr_off[1 - sc.cur];
            const int64_t last_row = (int64_t)row0 + nrows - 1;
            int64_t lo_last = -1, hi_last = -1;  // band of the last row (computed below)
            uint64_t cells = UINT64_MAX;          // in-band cells (computed below)
            Sched sch;
            if (sc.dead) {
                it.variant = 0;
                sch.s_end = 0;
            } else if (sc.plan_rows == (int64_t)nrows) {
                // chunks of one height get one variant: the choice hardly
                // depends on where the rows start (the results never do);
                // their schedules follow from the previous chunk's
                it.variant = sc.plan_variant;
                const int G = kVariants[it.variant][0], HR = kVariants[it.variant][1];
                if (sc.csched.row0 != (int64_t)row0 || sc.csched.rows != (int64_t)nrows || sc.csched.G != G ||
                    sc.csched.HR != HR)
                    sc.csched.init(sc.band, row0, nrows, G, HR);
                sc.csched.next(sc.band, sch, lo_last, hi_last, cells);
                if (sch.s_end <= 0)
                    it.variant = 0;
            } else {
                // candidates of one shape (chunk height, band, table width)
                // share one choice across reads: a small handle-wide cache
                const ShapeKey key{(int64_t)nrows, sc.band.num, sc.band.den, sc.band.w, sc.band.m};
                int cached = -1;
                {
                    std::lock_guard<std::mutex> lk(st->shape_mu);
                    auto hit = st->shape_variant.find(key);
                    if (hit != st->shape_variant.end())
                        cached = hit->second;
                }
                if (cached >= 0) {
                    it.variant = cached;
                    sch = schedule(sc.band, row0, nrows, kVariants[it.variant][0], kVariants[it.variant][1]);
                } else {
                    it.variant = choose_variant(sc.band, row0, nrows, sch, h->slot_cost);
                    if (sch.s_end > 0) {
                        std::lock_guard<std::mutex> lk(st->shape_mu);
                        if (st->shape_variant.size() < 4096)
                            st->shape_variant[key] = it.variant;
                    }
                }
                if (sch.s_end <= 0) {
                    it.variant = 0;
                } else {
                    sc.plan_rows = nrows;
                    sc.plan_variant = it.variant;
                    sc.csched.init(sc.band, (int64_t)row0 + nrows, nrows, kVariants[it.variant][0],
                                   kVariants[it.variant][1]);
                }
            }
            if (lo_last < 0) {
                lo_last = sc.band.lo(last_row);
                hi_last = sc.band.hi(last_row);
            }
            wd.fout_lo = (int32_t)lo_last;
            wd.dC = sch.dC;
            wd.a0 = sch.a0;
            wd.s_end = sch.s_end;
            if (sch.s_end <= 0)
                cells = 0;
            else if (cells == UINT64_MAX)
                cells = band_cells(sc.band, row0, (int64_t)row0 + nrows);
            wd.cells = cells;
            it.cost = (double)sch.s_end * kVariants[it.variant][0];
            it.cap = ring_need(wd, kVariants[it.variant][0], h->plan.ring_bin_shift);
            read_of[first + c] = (int)ci;
            // the band of this piece's last row is the row above the next piece
            Update u{&sc, sc.fr_lo, sc.fr_wid, sc.dead};
            if (!sc.dead) {
                if (hi_last >= lo_last && sch.s_end > 0) {
                    u.fr_lo = (int32_t)lo_last;
                    u.fr_wid = (int32_t)(hi_last - lo_last);
                } else {
                    u.dead = true;
                }
            }
            updates[first + c] = u;
        }
    };
    {
        // one thread unless the flush is large: waking the worker threads
        // costs more than planning a few thousand pieces (measured on GB300's
        // host: 121 GCUPS served with one thread, 103 with sixteen)
        const unsigned T = (unsigned)std::min<size_t>(
            {(size_t)host_threads(), n_pend, std::max<size_t>(1, (size_t)item_first[n_pend] / 32768)});
        run_tasks(T, [&](unsigned t) {
            for (size_t ci = n_pend * t / T; ci < n_pend * (t + 1) / T; ++ci)
                plan_chunk(ci);
        });
    }
    const uint32_t n_items = (uint32_t)items.size();
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
    std::vector<int> &order = sc_.order;
    std::vector<ClassLaunch> &classes = sc_.classes;
    classes.clear();
    if (!make_classes_binned(items.data(), items.size(), order, classes, sc_.sort, h->plan.ring_bin_shift,
                             /*longest_first=*/false)) {
        delete f;
        return RA_EINVAL;
    }
    // device memory for this flush
    auto take = [&](uint64_t bytes) -> void * {
        void *p = h->arena.alloc(std::max<uint64_t>(bytes, 256));
        if (p)
            f->blocks.push_back(p);
        return p;
    };
    // the flush's inputs live in one arena block and travel in one copy:
    // events, signal descriptors, work records, read slots, and the zeroed
    // per-chunk best keys and queue counters
    auto al256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_ev = sizeof(float) * n_ev, b_sig = sizeof(SigDesc) * sig.size();
    const size_t b_work = sizeof(WorkDesc) * n_items, b_rd = sizeof(int) * n_items;
    const size_t b_keys = sizeof(unsigned long long) * chunk_idx, b_q = sizeof(int) * (kMaxClasses + 2);
    const size_t o_sig = al256(b_ev), o_work = o_sig + al256(b_sig), o_rd = o_work + al256(b_work);
    const size_t o_keys = o_rd + al256(b_rd), o_q = o_keys + al256(b_keys), in_bytes = o_q + al256(b_q);
    char *d_in = (char *)take(in_bytes);
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
        delete f;
        return RA_ENOMEM;
    }
    float *d_ev = (float *)d_in;
    SigDesc *d_sig = (SigDesc *)(d_in + o_sig);
    WorkDesc *d_work = (WorkDesc *)(d_in + o_work);
    int *d_read_of = (int *)(d_in + o_rd);
    unsigned long long *d_keys = (unsigned long long *)(d_in + o_keys);
    int *d_queue = (int *)(d_in + o_q);
    char *hin = (char *)f->h_in;
    {
        // pack the pinned input block on the worker threads: each takes a
        // range of chunks (their events) and a range of work records (in
        // launch order)
        WorkDesc *hw = (WorkDesc *)(hin + o_work);
        float *hev = (float *)hin;
        const unsigned T = (unsigned)std::min<size_t>(
            {(size_t)host_threads(), n_pend, std::max<size_t>(1, (size_t)n_items / 32768)});
        run_tasks(T, [&](unsigned t) {
            for (size_t ci = n_pend * t / T; ci < n_pend * (t + 1) / T; ++ci) {
                const PendingChunk &pc = st->pending[ci];
                if (!pc.ev.empty())
                    memcpy(hev + ev_first[ci], pc.ev.data(), sizeof(float) * pc.ev.size());
            }
            for (size_t x = (size_t)n_items * t / T; x < (size_t)n_items * (t + 1) / T; ++x)
                hw[x] = items[order[x]].wd;
        });
    }
    memcpy(hin + o_sig, sig.data(), b_sig);
    memcpy(hin + o_rd, read_of.data(), b_rd);
    memset(hin + o_keys, 0, in_bytes - o_keys);
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
    if (!sig.empty())
        RA_CUDA(launch_expected_signal(d_sig, (int)sig.size(), h->d_ref, h->d_pore, h->cfg.k, abase, s));
    RA_CUDA(cudaEventRecord(h->fork, s));
    for (size_t ci = 0; ci < classes.size(); ++ci) {
        auto &cl = classes[ci];
        cudaStream_t cs = h->aux[ci];
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
        RA_CUDA(launch_stripe(cl.G, cl.HR, p, cl.grid, kBlock, cl.smem, cs));
        RA_CUDA(cudaEventRecord(h->join[ci], cs));
        RA_CUDA(cudaStreamWaitEvent(s, h->join[ci], 0));
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
    // launched: advance the host-side read state
    for (auto &u : updates) {
        if (!u.sc->dead)
            u.sc->cur = 1 - u.sc->cur;
        u.sc->fr_lo = u.fr_lo;
        u.sc->fr_wid = u.fr_wid;
        u.sc->dead = u.dead;
    }
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
        if (st->ready.count(t))
            continue;
        auto tf = st->ticket_flush.find(t);
        if (tf != st->ticket_flush.end()) {
            wait_for.push_back(tf->second);
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
        auto r = st->ready.find(tickets[x]);
        if (r == st->ready.end())
            return RA_EDEVICE;
        total += r->second.count;
    }
    if (total > cap)
        return RA_EINVAL;
    uint64_t pos = 0;
    for (uint32_t x = 0; x < n_tickets; ++x) {
        const uint32_t n = take_ready(st, st->ready.find(tickets[x]), out + pos, UINT32_MAX);
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
