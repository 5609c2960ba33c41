// engine.cu -- host side of librawalign_dtw: the C ABI, the arena, batch
// planning and launch, tickets, and the Read-Until serving loop.
//
// Planning turns every (read, candidate) pair into a WorkDesc: the band of
// Sec. 2.4.3 (slope num/den, half-width w_eff), the stripe period dC of the
// striped kernel, the first column and the step count.  The host picks, per
// alignment, the lanes-per-alignment variant that wastes the fewest lane
// steps, orders the queue longest-first, and records the launches of one run
// in a CUDA graph that later runs replay.
#include "engine.h"

namespace {

void free_batch(rawalign_dtw *h, Batch &b)
{
    for (auto &g : b.graph_part)
        if (g)
            cudaGraphExecDestroy(g);
    for (auto &e : b.ev)
        if (e)
            cudaEventDestroy(e);
    for (void *p : b.blocks)
        h->arena.release(p);
    b.blocks.clear();
}

template <typename T>
T *take(rawalign_dtw *h, Batch &b, uint64_t count)
{
    void *p = h->arena.alloc(sizeof(T) * std::max<uint64_t>(count, 1));
    if (p)
        b.blocks.push_back(p);
    return (T *)p;
}

// One DTW work item: rows from event ev0 on (n of them) against the m
// expected values from r0 on, result slot `slot`, per-read key slot `read`.
void fill_work(PlanItem &it, uint64_t ev0, uint64_t r0, int64_t n, int64_t m, const BandDef &band, int32_t wrep,
               int32_t slot, int32_t read, int32_t n_read)
{
    memset(&it.wd, 0, sizeof(WorkDesc));
    WorkDesc &wd = it.wd;
    wd.ev_off = ev0;
    wd.r_off = r0;
    wd.fin_off = ~0ull;
    wd.num = band.num;
    wd.den = band.den;
    wd.row0 = 0;
    wd.nrows = (int32_t)n;
    wd.m = (int32_t)m;
    wd.w = (int32_t)band.w;
    wd.cand = slot;
    wd.read = read;
    wd.n_read = n_read;
    wd.fin_lo = -1;
    wd.fin_wid = 0;
    wd.w_report = wrep;
}

// Anchors of one candidate are valid when sorted, disjoint in both sequences,
// non-empty and inside the n x m table.
bool anchors_valid(const rawalign_anchor_t *A, uint64_t K, int64_t n, int64_t m)
{
    int64_t pq = 0, pt = 0;
    for (uint64_t a = 0; a < K; ++a) {
        if (A[a].len < 1 || (int64_t)A[a].q < pq || (int64_t)A[a].t < pt)
            return false;
        pq = (int64_t)A[a].q + A[a].len;
        pt = (int64_t)A[a].t + A[a].len;
        if (pq > n || pt > m)
            return false;
    }
    return true;
}

int plan_and_upload(rawalign_dtw *h, Batch &b, const float *events, const uint64_t *offs,
                    uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                    const rawalign_anchor_t *anchors = nullptr, const uint64_t *anchor_offs = nullptr)
{
    const auto t_plan = std::chrono::steady_clock::now();
    const int k = h->cfg.k;
    b.n_reads = n_reads;
    b.n_cands = n_cands;
    b.n_events = n_reads ? offs[n_reads] : 0;
    b.plain = (h->cfg.kernel == RA_KERNEL_PLAIN);
    // validation (host part; event values are checked on the device)
    for (uint32_t q = 0; q < n_reads; ++q)
        if (offs[q + 1] <= offs[q])
            return RA_EINVAL;
    if (n_reads && offs[0] != 0)
        return RA_EINVAL;
    if (b.n_events >= (1ull << 40))
        return RA_EINVAL;
    b.anchored = anchor_offs != nullptr;
    if (b.anchored && !anchors && n_cands && anchor_offs[n_cands] != anchor_offs[0])
        return RA_EINVAL;
    // anchor offsets must not decrease: checked before any range reads anchors
    if (b.anchored)
        for (uint32_t c = 0; c < n_cands; ++c)
            if (anchor_offs[c + 1] < anchor_offs[c])
                return RA_EINVAL;
    b.et = h->cfg.early_termination && !b.anchored && !b.plain && h->cfg.end_mode == RA_END_GLOBAL;
    // planning runs on threads over candidate ranges: checks and sizes first,
    // then every range writes its records straight to their final places
    struct Part {
        uint32_t c0 = 0, c1 = 0;
        uint64_t r_sum = 0;                // expected values of the range
        uint64_t n_items = 0, n_plan = 0;  // this range's records
        uint64_t rb = 0, ib = 0, pb = 0;   // their first global indices
        int max_rows = 1;
        int rc = RA_OK;
    };
    const uint32_t n_parts = std::max<uint32_t>(1, std::min<uint32_t>(host_threads(), (n_cands + 4095) / 4096));
    std::vector<Part> parts(n_parts);
    for (uint32_t t = 0; t < n_parts; ++t) {
        parts[t].c0 = (uint32_t)((uint64_t)n_cands * t / n_parts);
        parts[t].c1 = (uint32_t)((uint64_t)n_cands * (t + 1) / n_parts);
    }
    auto over_parts = [&](auto fn) {
        parallel_for(n_parts, [&](uint64_t t0, uint64_t t1) {
            for (uint64_t t = t0; t < t1; ++t)
                fn(parts[t]);
        }, 1);
        for (auto &pt_ : parts)
            if (pt_.rc != RA_OK)
                return pt_.rc;
        return (int)RA_OK;
    };
    // the pieces of one anchored candidate in path order (Sec. 2.4.2): gap 0,
    // anchor 1, gap 1, ..., anchor K, gap K; each gap with rows and columns is
    // a DTW work item, an anchor or a gap with only rows or only columns a
    // fixed run of cells
    auto gaps = [&](uint32_t c, auto on_gap, auto on_run) {
        const rawalign_candidate_t &cd = cands[c];
        const int64_t n = (int64_t)(offs[cd.read_id + 1] - offs[cd.read_id]);
        const int64_t m = (int64_t)cd.ref_len_bases - k + 1;
        const rawalign_anchor_t *A = anchors ? anchors + anchor_offs[c] : nullptr;
        const uint64_t K = anchor_offs[c + 1] - anchor_offs[c];
        int64_t pq = 0, pt = 0;
        for (uint64_t a = 0; a <= K; ++a) {
            const int64_t q1 = a < K ? (int64_t)A[a].q : n, t1 = a < K ? (int64_t)A[a].t : m;
            const int64_t nr = q1 - pq, nc = t1 - pt;
            if (nr > 0 && nc > 0) {
                if (!on_gap(pq, pt, nr, nc))
                    return false;
            } else if (nr > 0) {
                // events aligned to one value: the previous anchor's last (the first anchor's first)
                on_run(pq, a > 0 ? pt - 1 : t1, nr, 1, 0);
            } else if (nc > 0) {
                // values aligned to one event: the previous anchor's last (the first anchor's first)
                on_run(a > 0 ? pq - 1 : q1, pt, nc, 0, 1);
            }
            if (a < K) {
                on_run((int64_t)A[a].q, (int64_t)A[a].t, (int64_t)A[a].len, 1, 1);
                pq = (int64_t)A[a].q + A[a].len;
                pt = (int64_t)A[a].t + A[a].len;
            }
        }
        return true;
    };
    // pass 1: candidate checks, expected values per range, and (anchored)
    // the exact count of gaps and pieces
    int rc = over_parts([&](Part &pt_) {
        for (uint32_t c = pt_.c0; c < pt_.c1; ++c) {
            const rawalign_candidate_t &cd = cands[c];
            if (cd.read_id >= n_reads || cd.strand > 1 || cd.ref_offset > h->ref_len ||
                cd.ref_len_bases > h->ref_len - cd.ref_offset || (int64_t)cd.ref_len_bases < k) {
                pt_.rc = RA_EINVAL;
                return;
            }
            const int64_t n = (int64_t)(offs[cd.read_id + 1] - offs[cd.read_id]);
            const int64_t m = (int64_t)cd.ref_len_bases - k + 1;
            if (n >= (1 << 30) || m >= (1 << 30)) {
                pt_.rc = RA_EINVAL;
                return;
            }
            pt_.r_sum += (uint64_t)m;
            if (!b.anchored)
                continue;
            const uint64_t K = anchor_offs[c + 1] - anchor_offs[c];
            if (!anchors_valid(anchors ? anchors + anchor_offs[c] : nullptr, K, n, m)) {
                pt_.rc = RA_EINVAL;
                return;
            }
            gaps(
                c,
                [&](int64_t, int64_t, int64_t, int64_t) {
                    ++pt_.n_items;
                    ++pt_.n_plan;
                    return true;
                },
                [&](int64_t, int64_t, int64_t, int, int) { ++pt_.n_plan; });
        }
        if (!b.anchored)
            pt_.n_items = pt_.c1 - pt_.c0;
    });
    if (rc != RA_OK)
        return rc;
    uint64_t r_total = 0, n_items = 0, n_plan = 0;
    for (auto &pt_ : parts) {
        pt_.rb = r_total;
        pt_.ib = n_items;
        pt_.pb = n_plan;
        r_total += pt_.r_sum;
        n_items += pt_.n_items;
        n_plan += pt_.n_plan;
    }
    if (n_plan >= (1ull << 32) || n_items >= (1ull << 31))
        return RA_EINVAL;
    // early termination queues each read's first candidate first
    std::vector<uint32_t> first_of_read(b.et ? n_reads : 0, UINT32_MAX);
    if (b.et)
        for (uint32_t c = n_cands; c-- > 0;)
            first_of_read[cands[c].read_id] = c;
    b.n_work = (uint32_t)n_items;
    // planned records are written to a pinned staging buffer (one fast copy
    // each); the plan items live in the handle's scratch, reused across batches
    auto al256 = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t n_cdesc = b.anchored ? n_cands : 0;
    const uint64_t o_sig = 0, o_read = al256(o_sig + sizeof(SigDesc) * (uint64_t)n_cands);
    const uint64_t o_cdesc = al256(o_read + sizeof(int) * (uint64_t)n_cands);
    const uint64_t o_plan = al256(o_cdesc + sizeof(CombineDesc) * n_cdesc);
    const uint64_t o_work = al256(o_plan + sizeof(PieceRef) * n_plan);
    const uint64_t stage_need = al256(o_work + sizeof(WorkDesc) * n_items) + 256;
    if (h->stage_bytes < stage_need) {
        if (h->stage)
            cudaFreeHost(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        RA_CUDA(cudaHostAlloc((void **)&h->stage, stage_need, cudaHostAllocDefault));
        h->stage_bytes = stage_need;
    }
    WorkDesc *work = (WorkDesc *)(h->stage + o_work);
    SigDesc *sig = (SigDesc *)(h->stage + o_sig);
    PieceRef *plan_h = (PieceRef *)(h->stage + o_plan);
    CombineDesc *cdesc_h = (CombineDesc *)(h->stage + o_cdesc);
    int *read_of = (int *)(h->stage + o_read);
    if (h->plan_items.size() < n_items)
        h->plan_items.resize(n_items);
    PlanItem *items = h->plan_items.data();
    // band, work items and schedules
    b.cells = 0;
    b.max_rows = 1;
    const int forced = h->cfg.kernel >= RA_KERNEL_VARIANT0 ? h->cfg.kernel - RA_KERNEL_VARIANT0 : -1;
    rc = over_parts([&](Part &pt_) {
        // alignments of one shape (rows, band) get one schedule: a small
        // direct-mapped cache of choose_variant's answers (exact keys)
        struct Choice {
            int64_t n = -1, num = 0, den = 0, w = 0, m = 0;
            int variant = 0;
            Sched sc;
            uint64_t cells = 0;
        };
        std::vector<Choice> cache(1024);
        auto schedule_item = [&](PlanItem &it, const BandDef &band, int64_t n) {
            Sched sc;
            uint64_t cells = 0;
            if (b.plain || (forced >= 0 && forced < kNumVariants)) {
                it.variant = b.plain ? 0 : forced;
                sc = schedule(band, 0, n, kVariants[it.variant][0], kVariants[it.variant][1]);
                cells = band_cells(band, 0, n);
            } else {
                const uint64_t hk = ((uint64_t)n * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)band.m * 0xC2B2AE3D27D4EB4Full) ^
                                    ((uint64_t)band.w * 0x165667B19E3779F9ull) ^ ((uint64_t)band.num << 17) ^
                                    (uint64_t)band.den;
                Choice &ch = cache[(hk ^ (hk >> 29)) & 1023];
                if (ch.n == n && ch.m == band.m && ch.w == band.w && ch.num == band.num && ch.den == band.den) {
                    it.variant = ch.variant;
                    sc = ch.sc;
                    cells = ch.cells;
                } else {
                    it.variant = choose_variant(band, 0, n, sc, h->slot_cost);
                    cells = band_cells(band, 0, n);
                    ch.n = n;
                    ch.m = band.m;
                    ch.w = band.w;
                    ch.num = band.num;
                    ch.den = band.den;
                    ch.variant = it.variant;
                    ch.sc = sc;
                    ch.cells = cells;
                }
            }
            it.wave = 0;
            set_schedule(it, sc, h->plan.ring_bin_shift);
            // the striped kernel reports this count instead of counting
            it.wd.cells = sc.s_end > 0 ? cells : 0;
            pt_.max_rows = std::max<int>(pt_.max_rows, (int)n);
        };
        uint64_t ix = pt_.ib, px = pt_.pb, rx = pt_.rb;
        for (uint32_t c = pt_.c0; c < pt_.c1; ++c) {
            const rawalign_candidate_t &cd = cands[c];
            const int64_t n = (int64_t)(offs[cd.read_id + 1] - offs[cd.read_id]);
            const int64_t m = (int64_t)cd.ref_len_bases - k + 1;
            const uint64_t r0 = rx;
            rx += (uint64_t)m;
            sig[c].ref_off = cd.ref_offset;
            sig[c].r_off = r0;
            sig[c].len = cd.ref_len_bases;
            sig[c].strand = cd.strand;
            read_of[c] = (int)cd.read_id;
            BandDef band;
            int32_t wrep;
            if (band_for(n, m, cd.band_w, cd.slope_num, cd.slope_den, band, wrep) != 0) {
                pt_.rc = RA_EINVAL;
                return;
            }
            const uint64_t ev0 = offs[cd.read_id];
            if (!b.anchored) {
                PlanItem &it = items[c];
                fill_work(it, ev0, r0, n, m, band, wrep, (int32_t)c, (int32_t)cd.read_id, (int32_t)n);
                schedule_item(it, band, n);
                it.wave = (b.et && first_of_read[cd.read_id] != c) ? 1 : 0;
                continue;
            }
            CombineDesc &cdc = cdesc_h[c];
            cdc.first = (uint32_t)px;
            cdc.n = (int32_t)n;
            cdc.m = (int32_t)m;
            cdc.read = (int32_t)cd.read_id;
            cdc.w_report = cd.band_w < 0 ? -1 : cd.band_w;
            const bool ok = gaps(
                c,
                [&](int64_t pq, int64_t pt, int64_t nr, int64_t nc) {
                    // a gap aligned by banded DTW into its own result slot
                    BandDef gb;
                    int32_t gw;
                    if (band_for(nr, nc, cd.band_w, 0, 0, gb, gw) != 0)
                        return false;
                    const int32_t slot = (int32_t)ix++;
                    PlanItem &it = items[slot];
                    fill_work(it, ev0 + pq, r0 + pt, nr, nc, gb, gw, slot, slot, (int32_t)nr);
                    schedule_item(it, gb, nr);
                    PieceRef pr{};
                    pr.kind = 0;
                    pr.idx = (uint32_t)slot;
                    plan_h[px++] = pr;
                    return true;
                },
                [&](int64_t q, int64_t t, int64_t len, int ev_step, int r_step) {
                    PieceRef pr{};
                    pr.kind = 1;
                    pr.ev = ev0 + q;
                    pr.r = r0 + t;
                    pr.len = (uint32_t)len;
                    pr.ev_step = (uint16_t)ev_step;
                    pr.r_step = (uint16_t)r_step;
                    plan_h[px++] = pr;
                });
            if (!ok) {
                pt_.rc = RA_EINVAL;
                return;
            }
            cdc.count = (uint32_t)(px - cdc.first);
        }
    });
    if (rc != RA_OK)
        return rc;
    for (auto &pt_ : parts)
        b.max_rows = std::max(b.max_rows, pt_.max_rows);
    uint64_t slots[kNumVariants];
    if (!b.plain && h->cfg.kernel == RA_KERNEL_AUTO) {
        PlanParams pp = h->plan;
        pp.split = !b.et;  // early termination checks run per group, not across a block
        shorten_longest(items, n_items, h->sm_count, h->slot_cost, slots, pp);
    } else {
        if (h->cfg.kernel == RA_KERNEL_SPLIT) {
            // every alignment on a block of four warps (tests)
            parallel_for(n_items, [&](uint64_t x0, uint64_t x1) {
                for (uint64_t x = x0; x < x1; ++x) {
                    PlanItem &it = items[x];
                    if (it.wd.s_end <= 0)
                        continue;
                    BandDef band;
                    band.num = it.wd.num;
                    band.den = it.wd.den;
                    band.w = it.wd.w;
                    band.m = it.wd.m;
                    const Sched s24 = schedule(band, it.wd.row0, it.wd.nrows, 32, 24);
                    if (s24.s_end <= 0)
                        continue;
                    it.variant = kSplitVariant;
                    it.split = true;
                    set_schedule(it, s24, h->plan.ring_bin_shift);
                    it.cap = split_row_cap(it.wd);
                }
            });
        }
        variant_slots(items, n_items, slots);
    }
    b.slots = 0;
    for (int v = 0; v < kNumVariants; ++v)
        b.slots += slots[v];
    b.n_split = 0;
    for (uint64_t x = 0; x < n_items; ++x)
        b.n_split += items[x].split ? 1u : 0u;
    // launch order and classes (variant x ring size), longest first
    std::vector<int> &order = h->plan_order;
    b.classes.clear();
    if (!make_classes_binned(items, n_items, order, b.classes, h->plan_sort, h->plan.ring_bin_shift))
        return RA_EINVAL;
    if (b.plain)
        b.classes.clear();
    parallel_for(n_items, [&](uint64_t x0, uint64_t x1) {
        for (uint64_t x = x0; x < x1; ++x)
            work[x] = items[order[x]].wd;
    });
    // device memory
    b.d_events = take<float>(h, b, b.n_events);
    b.d_sig = take<SigDesc>(h, b, n_cands);
    b.d_r = take<float>(h, b, r_total);
    b.n_r = r_total;
    b.d_work = take<WorkDesc>(h, b, b.n_work);
    b.d_results = take<rawalign_result_t>(h, b, n_cands);
    b.d_keys = take<unsigned long long>(h, b, n_reads);
    b.d_read_of = take<int>(h, b, n_cands);
    b.d_queue = take<int>(h, b, kMaxClasses + 2);
    if (!b.d_events || !b.d_sig || !b.d_r || !b.d_work || !b.d_results || !b.d_keys || !b.d_read_of ||
        !b.d_queue)
        return RA_ENOMEM;
    b.d_err = b.d_queue + kMaxClasses;
    if (b.anchored) {
        b.d_pres = take<rawalign_result_t>(h, b, b.n_work);
        b.d_pkeys = take<unsigned long long>(h, b, b.n_work);
        b.d_plan = take<PieceRef>(h, b, n_plan);
        b.d_cdesc = take<CombineDesc>(h, b, n_cands);
        if (!b.d_pres || !b.d_pkeys || !b.d_plan || !b.d_cdesc)
            return RA_ENOMEM;
    }
    if (b.plain) {
        b.d_plain_diag = take<float>(h, b, 3ull * (b.max_rows + 2));
        if (!b.d_plain_diag)
            return RA_ENOMEM;
    }
    // launch geometry and global rings where shared memory is too small
    rc = finalize_classes(h->sm_count, b.classes, [&](uint64_t bytes) { return (void *)take<char>(h, b, bytes); });
    if (rc != RA_OK)
        return rc;
    // uploads go on their own stream so that planning and copying this batch
    // overlap the kernels of the batch before it; the handle's stream waits
    // for them, and the host only for the copies themselves
    cudaStream_t s = h->upload;
    const auto t_upload = std::chrono::steady_clock::now();
    b.host_plan_ms = std::chrono::duration<double, std::milli>(t_upload - t_plan).count();
    RA_CUDA(cudaMemcpyAsync(b.d_events, events, sizeof(float) * b.n_events, cudaMemcpyHostToDevice, s));
    RA_CUDA(cudaMemcpyAsync(b.d_sig, sig, sizeof(SigDesc) * n_cands, cudaMemcpyHostToDevice, s));
    RA_CUDA(cudaMemcpyAsync(b.d_work, work, sizeof(WorkDesc) * b.n_work, cudaMemcpyHostToDevice, s));
    if (b.anchored && n_plan)
        RA_CUDA(cudaMemcpyAsync(b.d_plan, plan_h, sizeof(PieceRef) * n_plan, cudaMemcpyHostToDevice, s));
    if (b.anchored && n_cands)
        RA_CUDA(cudaMemcpyAsync(b.d_cdesc, cdesc_h, sizeof(CombineDesc) * n_cands, cudaMemcpyHostToDevice, s));
    RA_CUDA(cudaMemcpyAsync(b.d_read_of, read_of, sizeof(int) * n_cands, cudaMemcpyHostToDevice, s));
    for (auto &e : b.ev)
        RA_CUDA(cudaEventCreate(&e));
    RA_CUDA(cudaEventRecord(h->uploaded, s));
    RA_CUDA(cudaStreamWaitEvent(h->stream, h->uploaded, 0));
    // the caller may free its buffers on return
    RA_CUDA(cudaEventSynchronize(h->uploaded));
    b.host_upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_upload).count();
    return RA_OK;
}

// The path in three parts: pre (reset, event check, expected signal), the DTW
// kernels, post (decision).  Timing events sit between the parts, outside any
// graph.
int record_part(rawalign_dtw *h, Batch &b, int part, uint32_t &launches)
{
    cudaStream_t s = h->stream;
    if (part == 0) {
        RA_CUDA(cudaMemsetAsync(b.d_keys, 0, sizeof(unsigned long long) * std::max<uint32_t>(b.n_reads, 1), s));
        RA_CUDA(cudaMemsetAsync(b.d_queue, 0, sizeof(int) * (kMaxClasses + 2), s));
        RA_CUDA(launch_check_events(b.d_events, b.n_events, b.d_err, s));
        launches += b.n_events ? 1 : 0;
        RA_CUDA(launch_expected_signal(b.d_sig, (int)b.n_cands, h->d_ref, h->d_pore, h->cfg.k, b.d_r, s));
        launches += b.n_cands ? 1 : 0;
    } else if (part == 1) {
        // anchored batches run their gaps as GLOBAL alignments into per-gap
        // results, then combine them per candidate (Sec. 2.4.2)
        rawalign_result_t *res = b.anchored ? b.d_pres : b.d_results;
        unsigned long long *keys = b.anchored ? b.d_pkeys : b.d_keys;
        const int end_free = !b.anchored && h->cfg.end_mode == RA_END_FREE;
        if (b.plain) {
            for (uint32_t x = 0; x < b.n_work; ++x) {
                RA_CUDA(launch_plain(b.d_work + x, b.d_events, b.d_r, b.d_plain_diag, res, keys, h->cfg.b_match,
                                     end_free, s));
                ++launches;
            }
        } else {
            // launch classes: a dependent-launch chain on the stream, or
            // parallel branches (classes_as_chain)
            const bool chain = classes_as_chain(b.n_work, h->sm_count);
            if (!chain)
                RA_CUDA(cudaEventRecord(h->fork, s));
            int qi = 0;
            for (size_t ci = 0; ci < b.classes.size(); ++ci) {
                auto &cl = b.classes[ci];
                const bool dependent = chain && ci > 0;
                cudaStream_t cs = chain ? s : h->aux[ci];
                if (!chain)
                    RA_CUDA(cudaStreamWaitEvent(cs, h->fork, 0));
                StripeParams p{};
                p.work = b.d_work + cl.first;
                p.n_work = cl.count;
                p.queue = b.d_queue + (qi++);
                p.events = b.d_events;
                p.r_all = b.d_r;
                p.fstore = nullptr;
                p.fstore_out = nullptr;
                p.results = res;
                p.best_keys = keys;
                p.gring = cl.gring;
                p.ring_cap = cl.ring_cap;
                p.ring_in_smem = cl.ring_in_smem;
                p.b_match = h->cfg.b_match;
                p.end_free = end_free;
                p.early_term = b.et;
                p.err = b.d_err;
                p.n_events = b.n_events;
                p.n_r = b.n_r;
                p.n_fstore = 0;
                p.n_results = (int)(b.anchored ? b.n_work : b.n_cands);
                p.n_keys = (int)(b.anchored ? b.n_work : b.n_reads);
                p.stall_handoff = h->cfg.test_stall_handoff;
                if (cl.split)
                    RA_CUDA(launch_split(cl.HR, p, cl.grid, cs, dependent));
                else
                    RA_CUDA(launch_stripe(cl.G, cl.HR, p, cl.grid, kBlock, cl.smem, cs, dependent));
                ++launches;
                if (!chain) {
                    RA_CUDA(cudaEventRecord(h->join[ci], cs));
                    RA_CUDA(cudaStreamWaitEvent(s, h->join[ci], 0));
                }
            }
        }
        if (b.anchored) {
            RA_CUDA(launch_combine(b.d_cdesc, (int)b.n_cands, b.d_plan, b.d_pres, b.d_events, b.d_r, b.d_results,
                                   b.d_keys, h->cfg.b_match, s));
            launches += b.n_cands ? 1 : 0;
        }
    } else {
        RA_CUDA(launch_decide(b.d_results, (int)b.n_cands, b.d_keys, b.d_read_of, h->cfg.score_threshold, 1, s));
        launches += b.n_cands ? 1 : 0;
    }
    return RA_OK;
}

int record_run(rawalign_dtw *h, Batch &b)
{
    uint32_t launches = 0;
    for (int part = 0; part < 3; ++part) {
        RA_CUDA(cudaEventRecord(b.ev[part], h->stream));
        int rc = record_part(h, b, part, launches);
        if (rc != RA_OK)
            return rc;
    }
    RA_CUDA(cudaEventRecord(b.ev[3], h->stream));
    b.launches = launches;
    return RA_OK;
}

int run_batch(rawalign_dtw *h, Batch &b)
{
    if (b.plain)
        return record_run(h, b);
    if (!b.graph_part[0]) {
        uint32_t launches = 0;
        for (int part = 0; part < 3; ++part) {
            cudaGraph_t g = nullptr;
            RA_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            int rc = record_part(h, b, part, launches);
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (rc != RA_OK) {
                if (g)
                    cudaGraphDestroy(g);
                return rc;
            }
            RA_CUDA(e);
            e = cudaGraphInstantiate(&b.graph_part[part], g, 0);
            cudaGraphDestroy(g);
            RA_CUDA(e);
        }
        b.launches = launches;
    }
    for (int part = 0; part < 3; ++part) {
        RA_CUDA(cudaEventRecord(b.ev[part], h->stream));
        RA_CUDA(cudaGraphLaunch(b.graph_part[part], h->stream));
    }
    RA_CUDA(cudaEventRecord(b.ev[3], h->stream));
    return RA_OK;
}

int new_ticket(rawalign_dtw *h, uint64_t batch_id, Batch &b, uint64_t *ticket)
{
    Ticket t;
    t.batch = batch_id;
    t.d_results = b.d_results;
    t.n = b.n_cands;
    t.d_err = b.d_err;
    RA_CUDA(cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming));
    RA_CUDA(cudaEventRecord(t.done, h->stream));
    uint64_t id = h->next_id++;
    h->tickets[id] = std::move(t);
    *ticket = id;
    return RA_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" int rawalign_dtw_create(const rawalign_dtw_config_t *config, const float *pore_model,
                                   const uint8_t *ref_2bit, uint64_t ref_len, rawalign_dtw_t **out)
{
    if (!config || !pore_model || !out || (!ref_2bit && ref_len))
        return RA_EINVAL;
    *out = nullptr;
    if (config->k < 1 || config->k > 8 || !config->arena_dev || config->arena_bytes < 4096)
        return RA_EINVAL;
    if (((uintptr_t)config->arena_dev & 255) != 0)
        return RA_EINVAL;
    if (!std::isfinite(config->b_match) || !std::isfinite(config->score_threshold))
        return RA_EINVAL;
    if (config->end_mode != RA_END_GLOBAL && config->end_mode != RA_END_FREE)
        return RA_EINVAL;
    if (config->serve_slots < 0 || config->serve_max_events < 0 || config->max_candidates < 0)
        return RA_EINVAL;
    if (config->kernel < RA_KERNEL_AUTO || config->kernel == 3 ||
        config->kernel >= RA_KERNEL_VARIANT0 + kNumVariants)
        return RA_EINVAL;
    const uint64_t n_pore = 1ull << (2 * config->k);
    for (uint64_t x = 0; x < n_pore; ++x)
        if (!std::isfinite(pore_model[x]))
            return RA_EINVAL;
    rawalign_dtw *h = new (std::nothrow) rawalign_dtw();
    if (!h)
        return RA_ENOMEM;
    h->cfg = *config;
    for (int v = 0; v < kNumVariants; ++v)
        h->slot_cost[v] = kSlotCost[v];
    if (config->autotune_path) {
        // lines "G HR cost": the measured relative cost of one lane-cell
        // slot; "ring_bins S" and "latency_split X": the planner's knobs
        FILE *f = fopen(config->autotune_path, "r");
        if (!f) {
            delete h;
            return RA_EINVAL;
        }
        char line[256];
        bool bad = false;
        while (fgets(line, sizeof line, f)) {
            int G, HR, sh;
            double c;
            if (sscanf(line, "%d %d %lf", &G, &HR, &c) == 3) {
                for (int v = 0; v < kNumVariants; ++v)
                    if (kVariants[v][0] == G && kVariants[v][1] == HR && c > 0 && std::isfinite(c))
                        h->slot_cost[v] = c;
            } else if (sscanf(line, " ring_bins %d", &sh) == 1) {
                if (sh == 1 || sh == 2)
                    h->plan.ring_bin_shift = sh;
                else
                    bad = true;
            } else if (sscanf(line, " latency_split %lf", &c) == 1) {
                if (std::isfinite(c) && c >= 0)
                    h->plan.latency_split = c;
                else
                    bad = true;
            } else if (sscanf(line, " block_split %lf", &c) == 1) {
                if (std::isfinite(c) && c >= 0)
                    h->plan.split_factor = c;
                else
                    bad = true;
            }
        }
        fclose(f);
        if (bad) {
            delete h;
            return RA_EINVAL;
        }
    }
    h->cfg.autotune_path = nullptr;
    h->stream = (cudaStream_t)config->cuda_stream;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    for (int v = 0; v < kMaxClasses; ++v) {
        if (cudaStreamCreateWithFlags(&h->aux[v], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->join[v], cudaEventDisableTiming) != cudaSuccess) {
            delete h;
            return RA_EDEVICE;
        }
    }
    if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->upload, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->uploaded, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        return RA_EDEVICE;
    }
    h->arena.init(config->arena_dev, config->arena_bytes);
    h->d_pore = (float *)h->arena.alloc(sizeof(float) * n_pore);
    // 16 bytes of zero padding: the expected-signal kernel reads the packed
    // reference as pairs of 32-bit words
    h->d_ref = (uint8_t *)h->arena.alloc((ref_len + 3) / 4 + 16);
    if (!h->d_pore || !h->d_ref) {
        delete h;
        return RA_ENOMEM;
    }
    h->ref_len = ref_len;
    int rc = RA_OK;
    if (cudaMemcpyAsync(h->d_pore, pore_model, sizeof(float) * n_pore, cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(h->d_ref + (ref_len + 3) / 4, 0, 16, h->stream) != cudaSuccess ||
        (ref_len && cudaMemcpyAsync(h->d_ref, ref_2bit, (ref_len + 3) / 4, cudaMemcpyHostToDevice, h->stream) !=
                        cudaSuccess) ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        rc = RA_EDEVICE;
    if (rc != RA_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return RA_OK;
}

extern "C" int rawalign_dtw_prepare_batch(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                          uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                          uint64_t *batch)
{
    NvtxRange nvtx_range("rawalign_dtw_prepare_batch");
    if (!h || !batch || !read_offsets || (n_cands && !cands) || (!events && n_reads))
        return RA_EINVAL;
    cudaSetDevice(h->device);
    uint64_t id = h->next_id++;
    Batch &b = h->batches[id];
    int rc = plan_and_upload(h, b, events, read_offsets, n_reads, cands, n_cands);
    if (rc != RA_OK) {
        free_batch(h, b);
        h->batches.erase(id);
        return rc;
    }
    *batch = id;
    return RA_OK;
}

extern "C" int rawalign_dtw_prepare_anchored(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                             uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                             const rawalign_anchor_t *anchors, const uint64_t *anchor_offsets,
                                             uint64_t *batch)
{
    NvtxRange nvtx_range("rawalign_dtw_prepare_anchored");
    if (!h || !batch || !read_offsets || !anchor_offsets || (n_cands && !cands) || (!events && n_reads))
        return RA_EINVAL;
    cudaSetDevice(h->device);
    uint64_t id = h->next_id++;
    Batch &b = h->batches[id];
    int rc = plan_and_upload(h, b, events, read_offsets, n_reads, cands, n_cands, anchors, anchor_offsets);
    if (rc != RA_OK) {
        free_batch(h, b);
        h->batches.erase(id);
        return rc;
    }
    *batch = id;
    return RA_OK;
}

extern "C" int rawalign_dtw_submit_anchored(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                            uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                            const rawalign_anchor_t *anchors, const uint64_t *anchor_offsets,
                                            uint64_t *ticket)
{
    NvtxRange nvtx_range("rawalign_dtw_submit_anchored");
    if (!ticket)
        return RA_EINVAL;
    uint64_t bid = 0;
    int rc = rawalign_dtw_prepare_anchored(h, events, read_offsets, n_reads, cands, n_cands, anchors,
                                           anchor_offsets, &bid);
    if (rc != RA_OK)
        return rc;
    Batch &b = h->batches[bid];
    b.auto_release = true;
    rc = record_run(h, b);
    if (rc != RA_OK) {
        rawalign_dtw_release_batch(h, bid);
        return rc;
    }
    b.ran = true;
    return new_ticket(h, bid, b, ticket);
}

extern "C" int rawalign_dtw_run_batch(rawalign_dtw_t *h, uint64_t batch, uint64_t *ticket)
{
    NvtxRange nvtx_range("rawalign_dtw_run_batch");
    if (!h || !ticket)
        return RA_EINVAL;
    auto it = h->batches.find(batch);
    if (it == h->batches.end())
        return RA_EINVAL;
    cudaSetDevice(h->device);
    int rc = run_batch(h, it->second);
    if (rc != RA_OK)
        return rc;
    it->second.ran = true;
    return new_ticket(h, batch, it->second, ticket);
}

extern "C" int rawalign_dtw_release_batch(rawalign_dtw_t *h, uint64_t batch)
{
    if (!h)
        return RA_EINVAL;
    auto it = h->batches.find(batch);
    if (it == h->batches.end())
        return RA_EINVAL;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (auto &tk : h->tickets)
        if (tk.second.batch == batch)
            tk.second.batch = ~0ull;  // results no longer available
    free_batch(h, it->second);
    h->batches.erase(it);
    return RA_OK;
}

extern "C" int rawalign_dtw_submit_batch(rawalign_dtw_t *h, const float *events, const uint64_t *read_offsets,
                                         uint32_t n_reads, const rawalign_candidate_t *cands, uint32_t n_cands,
                                         uint64_t *ticket)
{
    NvtxRange nvtx_range("rawalign_dtw_submit_batch");
    if (!ticket)
        return RA_EINVAL;
    uint64_t bid = 0;
    int rc = rawalign_dtw_prepare_batch(h, events, read_offsets, n_reads, cands, n_cands, &bid);
    if (rc != RA_OK)
        return rc;
    Batch &b = h->batches[bid];
    b.auto_release = true;
    rc = record_run(h, b);
    if (rc != RA_OK) {
        rawalign_dtw_release_batch(h, bid);
        return rc;
    }
    b.ran = true;
    return new_ticket(h, bid, b, ticket);
}

extern "C" int rawalign_dtw_poll(rawalign_dtw_t *h, uint64_t ticket, rawalign_result_t *out, uint32_t cap,
                                 uint32_t *n_out, int64_t timeout_us)
{
    NvtxRange nvtx_range("rawalign_dtw_poll");
    if (!h || !n_out || (cap && !out))
        return RA_EINVAL;
    *n_out = 0;
    cudaSetDevice(h->device);
    {
        bool handled = false;
        int rc = serve_poll(h, ticket, out, cap, n_out, timeout_us, &handled);
        if (handled)
            return rc;
    }
    auto it = h->tickets.find(ticket);
    if (it == h->tickets.end())
        return RA_EINVAL;
    Ticket &t = it->second;
    auto t0 = std::chrono::steady_clock::now();
    while (true) {
        cudaError_t e = cudaEventQuery(t.done);
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
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    int rc = RA_OK;
    if (t.serving) {
        uint32_t n = std::min<uint32_t>(cap, (uint32_t)t.host.size());
        if (n)
            memcpy(out, t.host.data(), sizeof(rawalign_result_t) * n);
        *n_out = n;
    } else {
        if (t.batch == ~0ull)
            rc = RA_EINVAL;
        else {
            int err[2] = {0, 0};
            RA_CUDA(cudaMemcpy(err, t.d_err, sizeof(err), cudaMemcpyDeviceToHost));
            if (err[1])
                rc = RA_EINVAL;
            else if (err[0])
                rc = RA_EDEVICE;  // checked build: a work item failed its device-side checks
            uint32_t n = std::min<uint32_t>(cap, t.n);
            if (n && rc == RA_OK)
                RA_CUDA(cudaMemcpy(out, t.d_results, sizeof(rawalign_result_t) * n, cudaMemcpyDeviceToHost));
            *n_out = rc == RA_OK ? n : 0;
        }
    }
    cudaEventDestroy(t.done);
    uint64_t bid = t.batch;
    bool serving = t.serving;
    h->tickets.erase(it);
    if (!serving && bid != ~0ull) {
        auto bt = h->batches.find(bid);
        if (bt != h->batches.end() && bt->second.auto_release) {
            free_batch(h, bt->second);
            h->batches.erase(bt);
        }
    }
    return rc;
}

extern "C" int rawalign_dtw_batch_stats(rawalign_dtw_t *h, uint64_t batch, rawalign_dtw_stats_t *out)
{
    if (!h || !out)
        return RA_EINVAL;
    auto it = h->batches.find(batch);
    if (it == h->batches.end() || !it->second.ran)
        return RA_EINVAL;
    Batch &b = it->second;
    float ms = 0, tot = 0;
    RA_CUDA(cudaEventSynchronize(b.ev[3]));
    if (b.cells == 0 && b.n_cands) {
        std::vector<rawalign_result_t> res(b.n_cands);
        RA_CUDA(cudaMemcpy(res.data(), b.d_results, sizeof(rawalign_result_t) * b.n_cands, cudaMemcpyDeviceToHost));
        for (auto &r : res)
            b.cells += r.cells;
    }
    RA_CUDA(cudaEventElapsedTime(&ms, b.ev[1], b.ev[2]));
    RA_CUDA(cudaEventElapsedTime(&tot, b.ev[0], b.ev[3]));
    out->dtw_ms = ms;
    out->total_ms = tot;
    out->cells = b.cells;
    out->split = b.n_split;
    out->slots = b.slots;
    out->launches = b.launches;
    out->host_plan_ms = b.host_plan_ms;
    out->host_upload_ms = b.host_upload_ms;
    return RA_OK;
}

extern "C" uint64_t rawalign_dtw_batch_bytes(uint64_t n_events, uint32_t n_reads, uint32_t n_cands,
                                             uint64_t total_ref_values)
{
    uint64_t b = 0;
    auto add = [&](uint64_t x) { b += (x + 255) & ~255ull; };
    add(4 * n_events);
    add(sizeof(SigDesc) * (uint64_t)n_cands);
    add(4 * total_ref_values);
    add(sizeof(WorkDesc) * (uint64_t)n_cands);
    add(sizeof(rawalign_result_t) * (uint64_t)n_cands);
    add(8ull * n_reads);
    add(4ull * n_cands);
    add(256);
    return b + (64ull << 20);  // ring buffers and slack
}

extern "C" int rawalign_dtw_destroy(rawalign_dtw_t *h)
{
    if (!h)
        return RA_EINVAL;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->upload)
        cudaStreamSynchronize(h->upload);
    serve_destroy(h);
    for (auto &tk : h->tickets)
        if (tk.second.done)
            cudaEventDestroy(tk.second.done);
    for (auto &b : h->batches)
        free_batch(h, b.second);
    for (int v = 0; v < kMaxClasses; ++v) {
        if (h->aux[v])
            cudaStreamDestroy(h->aux[v]);
        if (h->join[v])
            cudaEventDestroy(h->join[v]);
    }
    if (h->fork)
        cudaEventDestroy(h->fork);
    if (h->uploaded)
        cudaEventDestroy(h->uploaded);
    if (h->stage)
        cudaFreeHost(h->stage);
    if (h->upload)
        cudaStreamDestroy(h->upload);
    delete h;
    return RA_OK;
}

extern "C" int rawalign_dtw_set_variant_costs(rawalign_dtw_t *h, const double *costs, uint32_t n)
{
    if (!h || !costs || n != (uint32_t)kNumVariants)
        return RA_EINVAL;
    for (int v = 0; v < kNumVariants; ++v)
        if (!(costs[v] > 0) || !std::isfinite(costs[v]))
            return RA_EINVAL;
    for (int v = 0; v < kNumVariants; ++v)
        h->slot_cost[v] = costs[v];
    return RA_OK;
}

// Band of one alignment for callers outside this file (same rule as the batch
// planner): num/den/w as the kernels take them, and the w_eff to report.
int ra::host_band(int64_t n, int64_t m, int32_t band_w, int64_t num, int64_t den, int64_t *num_out,
                  int64_t *den_out, int64_t *w_out, int32_t *w_report)
{
    BandDef b;
    if (band_for(n, m, band_w, num, den, b, *w_report) != 0)
        return RA_EINVAL;
    *num_out = b.num;
    *den_out = b.den;
    *w_out = b.w;
    return RA_OK;
}

// Serving entry points are defined in serve.cu.
