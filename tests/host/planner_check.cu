// planner_check.cu -- host-only check of the batch planner (engine.h), run by
// tests/test_host_planner.py on the CPU.  It replays the striped kernel's
// lane schedule step by step for random alignments and every variant, and
// verifies what the planner's closed-form period dC promises:
//   - a lane enters each stripe at least one column before the first
//     in-band column of its rows (its first step there is fully out of band);
//   - every value lane 0 takes from the ring (the row above its stripe, in
//     band) is the one the last lane of the previous stripe wrote, with the
//     ring size ring_need() gives, lanes kLag columns apart, and the kernel's
//     timing taken at its loosest: a write is seen only two steps later (two
//     columns go together, one warp barrier per pair), a read may happen two
//     steps before the value is used (two-deep prefetch), and nothing may
//     overwrite the entry between the write and the use;
//   - the lane holding the last row leaves it within s_end steps.
// It also checks make_classes: classes are runs of one variant and ring
// size, longest first inside a class (first candidates before the others),
// classes ordered by their longest alignment; and the O(1) row step of the
// band DDA (ra::row_dda, used by the kernel at every stripe change) against
// stepping row by row; and that the planner's parallel loops visit every
// index once, with concurrent and nested callers; choose_variant against the
// plain loop over schedule(); and the serving path's flat hash map
// (FlatMap64) against std::unordered_map.
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"
#include "serve_expand.cuh"

using namespace ra_host;

static int fails = 0;
#define CHECK(c, ...)                       \
    do {                                    \
        if (!(c)) {                         \
            if (fails < 20)                 \
                printf(__VA_ARGS__);        \
            ++fails;                        \
        }                                   \
    } while (0)

static void check_schedule(const BandDef &band, int64_t n, int G, int HR, uint64_t &steps_checked)
{
    const Sched sc = schedule(band, 0, n, G, HR);
    if (sc.s_end <= 0)
        return;
    const int64_t H = (int64_t)G * HR, K = (n + H - 1) / H, dC = sc.dC;
    WorkDesc wd{};
    wd.dC = (int32_t)dC;
    wd.fin_wid = 0;
    const int64_t cap = ring_need(wd, G), mask = cap - 1;
    auto lane_rows = [&](int64_t k, int t, int64_t &r0, int64_t &r1) {
        r0 = k * H + (int64_t)t * HR;
        r1 = std::min(r0 + HR - 1, n - 1);
    };
    std::vector<int64_t> j(G), k(G, 0), b(G);
    auto set_b = [&](int t) {
        int64_t r0, r1;
        lane_rows(k[t], t, r0, r1);
        b[t] = (r0 > n - 1) ? -1 : band.hi(r1);
    };
    for (int t = 0; t < G; ++t) {
        j[t] = sc.a0 - 2 - (int64_t)kLag * t;  // the first step computes column a0 - 1 - kLag t
        set_b(t);
        int64_t r0, r1;
        lane_rows(0, t, r0, r1);
        if (r0 <= n - 1)
            CHECK(j[t] + 1 < band.lo(r0), "start not out of band: G%d HR%d t%d\n", G, HR, t);
    }
    // per ring slot: every write as (step, stripe, column)
    struct Wr {
        int64_t step, stripe, col;
    };
    std::vector<std::vector<Wr>> writes(cap);
    struct Use {
        int64_t step, stripe, col;
    };
    std::vector<Use> uses;
    const int t_last = (int)((n - 1 - (K - 1) * H) / HR);
    int64_t holder_done = -1;
    for (int64_t s = 0; s < sc.s_end; ++s) {
        for (int t = 0; t < G; ++t) {
            ++j[t];
            if (j[t] > b[t]) {
                if (k[t] == K - 1 && t == t_last && holder_done < 0)
                    holder_done = s;
                ++k[t];
                if (k[t] < K) {
                    j[t] -= dC;
                    set_b(t);
                    int64_t r0, r1;
                    lane_rows(k[t], t, r0, r1);
                    if (r0 <= n - 1)
                        CHECK(j[t] < band.lo(r0), "late entry: G%d HR%d n%lld k%lld t%d j%lld lo%lld\n", G, HR,
                              (long long)n, (long long)k[t], t, (long long)j[t], (long long)band.lo(r0));
                } else {
                    b[t] = INT64_MAX;
                }
            }
        }
        if (k[0] >= 1 && k[0] < K) {
            const int64_t above = k[0] * H - 1, c = j[0];
            if (c >= band.lo(above) && c <= band.hi(above))
                uses.push_back({s, k[0], c});
        }
        const int w = G - 1;
        if (k[w] < K - 1)
            writes[j[w] & mask].push_back({s, k[w], j[w]});
        ++steps_checked;
    }
    for (const Use &u : uses) {
        // the entry must hold (stripe - 1, column) from two steps before the
        // earliest read (use - 2) to the use, written by nothing else meanwhile
        const auto &ws = writes[u.col & mask];
        const Wr *last = nullptr;
        bool clobbered = false;
        for (const Wr &w : ws) {
            if (w.step <= u.step - 4)
                last = &w;
            else if (w.step <= u.step)
                clobbered = true;
        }
        CHECK(last && last->stripe == u.stripe - 1 && last->col == u.col && !clobbered,
              "ring: G%d HR%d n%lld stripe %lld column %lld step %lld cap %lld dC %lld\n", G, HR, (long long)n,
              (long long)u.stripe, (long long)u.col, (long long)u.step, (long long)cap, (long long)dC);
    }
    CHECK(holder_done >= 0 && holder_done < sc.s_end, "holder not done: G%d HR%d n%lld\n", G, HR, (long long)n);
}

int main()
{
    std::mt19937_64 rng(20240531);
    uint64_t steps = 0, cases = 0;
    for (int rep = 0; rep < 600; ++rep) {
        const int64_t n = 1 + (int64_t)(rng() % (rep < 300 ? 200 : 2500));
        const int64_t m = std::max<int64_t>(1, (int64_t)(n * (0.5 + (rng() % 1000) / 1000.0)) + (int64_t)(rng() % 7));
        const int kind = (int)(rng() % 4);
        int32_t band_w = kind == 0 ? -1 : (int32_t)(rng() % std::max<int64_t>(2, m / (kind == 1 ? 2 : 8)));
        int64_t num = 0, den = 0;
        if (kind == 3) {
            num = 1 + (int64_t)(rng() % 9);
            den = 1 + (int64_t)(rng() % 9);
        }
        BandDef band;
        int32_t wrep;
        if (band_for(n, m, band_w, num, den, band, wrep) != 0)
            continue;
        for (int v = 0; v < kNumVariants; ++v) {
            check_schedule(band, n, kVariants[v][0], kVariants[v][1], steps);
            ++cases;
        }
    }
    // the planner's parallel loops: every index once, also with two callers
    // at a time (one falls back to threads of its own) and nested loops
    {
        auto sum_loop = [](uint64_t n, bool nested) {
            std::vector<std::atomic<uint32_t>> hit(n);
            for (auto &h : hit)
                h = 0;
            parallel_for(n, [&](uint64_t lo, uint64_t hi) {
                if (nested)
                    parallel_for(hi - lo, [&](uint64_t a, uint64_t b) {
                        for (uint64_t x = lo + a; x < lo + b; ++x)
                            hit[x]++;
                    }, 1 << 10);
                else
                    for (uint64_t x = lo; x < hi; ++x)
                        hit[x]++;
            }, 1 << 12);
            for (auto &h : hit)
                if (h != 1)
                    return false;
            return true;
        };
        std::atomic<int> bad{0};
        std::vector<std::thread> callers;
        for (int c = 0; c < 3; ++c)
            callers.emplace_back([&, c] {
                for (int rep = 0; rep < 40; ++rep)
                    if (!sum_loop(1000 + 7919 * (uint64_t)(rep + c), (rep + c) % 3 == 0))
                        bad++;
            });
        for (auto &t : callers)
            t.join();
        CHECK(bad == 0, "parallel_for missed or repeated indices (%d loops)\n", (int)bad);
    }
    // O(1) row step of the band DDA against r single steps
    for (int rep = 0; rep < 200000; ++rep) {
        const int den = 1 + (int)(rng() % (rep % 3 == 0 ? 7 : (1u << 30) - 1));
        const int64_t num = (int64_t)(rng() % (rep % 2 ? 4ull * den : (1ull << 30)));
        const int q1 = (int)(num / den), r1 = (int)(num % den);
        const int Q0 = (int)(rng() % 2000000) - 1000000, R0 = (int)(rng() % den);
        const int r = (int)(rng() % 32);
        int64_t Q = Q0, R = R0;
        for (int x = 0; x < r; ++x) {
            Q += q1;
            R += r1;
            if (R >= den) {
                Q += 1;
                R -= den;
            }
        }
        if (Q > INT32_MAX)
            continue;  // not a band edge: columns stay below 2^31
        int Qf, Rf;
        ra::row_dda(Q0, R0, q1, r1, den, r, Qf, Rf);
        CHECK(Qf == Q && Rf == R, "row_dda den %d num %lld r %d: %d/%d vs %lld/%lld\n", den, (long long)num, r, Qf,
              Rf, (long long)Q, (long long)R);
        ++cases;
    }
    // launch classes
    for (int rep = 0; rep < 50; ++rep) {
        // small plans take the comparison sort, large ones the radix passes
        std::vector<PlanItem> items(1 + rng() % (rep % 2 ? 5000 : 60000));
        for (auto &it : items) {
            it.variant = (int)(rng() % kNumVariants);
            it.cap = 128 << (2 * (int)(rng() % 4));
            it.wave = (int)(rng() % 2);
            it.wd.s_end = (int32_t)(1 + rng() % 200000);
            it.cost = (double)it.wd.s_end * kVariants[it.variant][0];
        }
        std::vector<int> order;
        std::vector<ClassLaunch> cls;
        if (!make_classes(items, order, cls)) {
            CHECK(false, "make_classes refused\n");
            continue;
        }
        std::vector<int> seen(items.size(), 0);
        for (int x : order)
            seen[x]++;
        for (int c : seen)
            CHECK(c == 1, "order is not a permutation\n");
        size_t covered = 0;
        for (size_t ci = 0; ci < cls.size(); ++ci) {
            const ClassLaunch &cl = cls[ci];
            covered += cl.count;
            double mx = 0;
            for (int p = cl.first; p < cl.first + cl.count; ++p) {
                const PlanItem &it = items[order[p]];
                CHECK(kVariants[it.variant][0] == cl.G && kVariants[it.variant][1] == cl.HR && it.cap == cl.ring_cap,
                      "class mixes variants or rings\n");
                mx = std::max(mx, it.cost);
                if (p > cl.first) {
                    const PlanItem &pv = items[order[p - 1]];
                    CHECK(pv.wave < it.wave || (pv.wave == it.wave && pv.wd.s_end >= it.wd.s_end) ||
                              (pv.wave > it.wave && false),
                          "class order: wave %d/%d steps %d/%d\n", pv.wave, it.wave, pv.wd.s_end, it.wd.s_end);
                }
            }
            CHECK(mx == cl.max_cost, "max cost\n");
            if (ci > 0)
                CHECK(cls[ci - 1].max_cost >= cl.max_cost, "classes not longest first\n");
        }
        CHECK(covered == items.size(), "classes do not cover the items\n");
    }
    // the exact in-band cell count the striped kernel reports (floor sums,
    // and the O(1) form away from the table's edges) against row-by-row sums
    {
        uint64_t cell_cases = 0;
        for (int rep = 0; rep < 60000; ++rep) {
            BandDef b;
            const int64_t n = 1 + (int64_t)(rng() % 3000);
            b.m = 1 + (int64_t)(rng() % 4000);
            if (rng() % 5 == 0) {
                b.num = 0;
                b.den = 1;
                b.w = (rng() % 2) ? b.m : 1 + (int64_t)(rng() % 50);
            } else {
                b.num = 1 + (int64_t)(rng() % 3000);
                b.den = 1 + (int64_t)(rng() % 3000);
                b.w = 1 + (int64_t)(rng() % 80);
                if (rng() % 2)
                    prepare_cell_count(b);
            }
            if (rep % 1000 == 0) {  // slopes and widths at the planner's limits
                b.num = 1 + (int64_t)(rng() % (1ll << 30));
                b.den = 1 + (int64_t)(rng() % (1ll << 30));
                b.w = 1 + (int64_t)(rng() % 5000);
                b.m = 1 + (int64_t)(rng() % 200000);
                b.per = 0;
            }
            const int64_t r0 = (int64_t)(rng() % (n + 1)), r1 = r0 + (int64_t)(rng() % 400);
            uint64_t brute = 0;
            for (int64_t i = r0; i < r1; ++i) {
                const int64_t c = b.hi(i) - b.lo(i) + 1;
                if (c > 0)
                    brute += (uint64_t)c;
            }
            const uint64_t got = band_cells(b, r0, r1);
            CHECK(got == brute, "band_cells num %lld den %lld w %lld m %lld rows %lld..%lld: %llu, rows say %llu\n",
                  (long long)b.num, (long long)b.den, (long long)b.w, (long long)b.m, (long long)r0, (long long)r1,
                  (unsigned long long)got, (unsigned long long)brute);
            ++cell_cases;
        }
        cases += cell_cases;
    }
    // serving: the work records the device builds per piece (serve_piece)
    // against the host planner's schedule, band edges and cell count, over
    // runs of consecutive chunks with the frontier state carried along
    {
        for (int rep = 0; rep < 20000; ++rep) {
            BandDef b;
            b.m = 1 + (int64_t)(rng() % 6000);
            b.num = (rep % 97 == 0) ? 0 : 1 + (int64_t)(rng() % 3000);
            b.den = 1 + (int64_t)(rng() % 3000);
            b.w = 1 + (int64_t)(rng() % 200);
            if (rng() % 2)
                prepare_cell_count(b);
            const int v = (int)(rng() % kNumVariants);
            const int G = kVariants[v][0], HR = kVariants[v][1];
            ServeCandDev s{};
            s.r_off = 1000;
            s.fr_off[0] = 5000;
            s.fr_off[1] = 9000;
            s.num = b.num;
            s.den = b.den;
            s.per = b.per;
            s.hi_row = b.hi_row;
            s.m = (int32_t)b.m;
            s.w = (int32_t)b.w;
            s.w_report = 7;
            s.G = G;
            s.HR = HR;
            s.fr_lo = -1;
            // the stripe period as the planner sets it
            s.dC = schedule(b, 0, 1, G, HR).dC;
            {
                const int64_t H = (int64_t)G * HR;
                int64_t span = fdiv(2 * b.w * b.den - (H - HR + 1) * b.num, b.den);
                span = std::min<int64_t>(span, b.m - 1);
                s.dC = (int32_t)std::max<int64_t>((int64_t)kLag * G + 3, span + 2);
            }
            int cur = 0, fr_lo = -1, fr_wid = 0;
            bool dead = false;
            int64_t row0 = 0;
            for (int c = 0; c < 25; ++c) {
                const int64_t rows = 1 + (int64_t)(rng() % 300);
                ServeChunkDev ch{};
                ch.ev_off = 123;
                ch.cand_off = 0;
                ch.n_cands = 1;
                ch.first_piece = 40;
                ch.row0 = (int32_t)row0;
                ch.nrows = (int32_t)rows;
                WorkDesc wd{};
                serve_piece(ch, 3, 0, s, wd);
                const int64_t last = row0 + rows - 1;
                Sched want;
                if (!dead)
                    want = schedule(b, row0, rows, G, HR);
                const uint64_t cells = want.s_end > 0 ? band_cells(b, row0, row0 + rows) : 0;
                const bool fin_ok = row0 == 0 ? (wd.fin_off == ~0ull && wd.fin_lo == -1 && wd.fin_wid == 0)
                                              : (wd.fin_off == (uint64_t)(cur ? 9000 : 5000) && wd.fin_lo == fr_lo &&
                                                 wd.fin_wid == fr_wid);
                CHECK(fin_ok && wd.fout_off == (uint64_t)(cur ? 5000 : 9000) && wd.fout_lo == (int32_t)b.lo(last) &&
                          wd.a0 == want.a0 && wd.s_end == want.s_end && wd.dC == want.dC && wd.cells == cells &&
                          wd.cand == 40 && wd.read == 3 && wd.n_read == (int32_t)(row0 + rows) && wd.m == (int32_t)b.m,
                      "serve_piece num %lld den %lld w %lld m %lld row0 %lld rows %lld: a0 %d/%d s_end %d/%d dC %d/%d "
                      "cells %llu/%llu\n",
                      (long long)b.num, (long long)b.den, (long long)b.w, (long long)b.m, (long long)row0,
                      (long long)rows, wd.a0, want.a0, wd.s_end, want.s_end, wd.dC, want.dC,
                      (unsigned long long)wd.cells, (unsigned long long)cells);
                // the host planner's frontier update
                if (!dead) {
                    cur = 1 - cur;
                    const int64_t lo = b.lo(last), hi = b.hi(last);
                    if (hi >= lo && want.s_end > 0) {
                        fr_lo = (int32_t)lo;
                        fr_wid = (int32_t)(hi - lo);
                    } else {
                        dead = true;
                    }
                }
                CHECK(s.cur == cur && s.fr_lo == fr_lo && s.fr_wid == fr_wid && (s.dead != 0) == dead,
                      "serve_piece state\n");
                row0 += rows;
                ++cases;
            }
        }
    }
    // more launch classes than allowed with ring sizes binned by powers of
    // two: the planner falls back to powers of four
    {
        std::vector<PlanItem> items;
        for (int v = 0; v < kNumVariants; ++v)
            for (int c = 0; c < 9; ++c) {
                PlanItem it;
                memset(&it.wd, 0, sizeof(WorkDesc));
                it.variant = v;
                it.wd.dC = (128 << c) - 2 - (c ? 1 : 0);  // ring_need: the next power of two at or above dC + 2
                it.wd.s_end = 100;
                it.cap = ring_need(it.wd, kVariants[v][0], 1);
                it.cost = 100.0 * kVariants[v][0];
                items.push_back(it);
            }
        std::vector<int> order;
        std::vector<ClassLaunch> cls;
        SortScratch scr;
        CHECK(!make_classes(items.data(), items.size(), order, cls, scr), "expected more than kMaxClasses classes\n");
        CHECK(make_classes_binned(items.data(), items.size(), order, cls, scr, 1), "fallback to coarser bins failed\n");
        CHECK(cls.size() <= (size_t)kMaxClasses, "fallback still has too many classes\n");
        for (const PlanItem &it : items)
            CHECK(it.cap == ring_need(it.wd, kVariants[it.variant][0], 2), "fallback ring size\n");
        ++cases;
    }
    // the arena allocator: live blocks never overlap and stay inside the
    // arena; once everything is released the whole arena is one free range
    {
        const uint64_t kArena = 1ull << 24;
        Arena ar;
        ar.init((void *)0x10000, kArena);
        std::map<uint64_t, uint64_t> live;  // offset -> bytes asked (rounded up to 256)
        for (int op = 0; op < 200000; ++op) {
            if (live.empty() || rng() % 3 != 0) {
                const uint64_t n = 1 + rng() % (rng() % 8 == 0 ? 400000 : 5000);
                void *p = ar.alloc(n);
                if (!p)
                    continue;
                const uint64_t off = (uint64_t)((char *)p - (char *)0x10000), sz = (n + 255) & ~255ull;
                CHECK(off % 256 == 0 && off + sz <= kArena, "arena block outside the arena\n");
                auto nx = live.lower_bound(off);
                if (nx != live.end())
                    CHECK(off + sz <= nx->first, "arena blocks overlap\n");
                if (nx != live.begin()) {
                    auto pv = std::prev(nx);
                    CHECK(pv->first + pv->second <= off, "arena blocks overlap\n");
                }
                live[off] = sz;
            } else {
                auto it = live.begin();
                std::advance(it, (long)(rng() % live.size()));
                ar.release((char *)0x10000 + it->first);
                live.erase(it);
            }
            ++cases;
        }
        for (auto &kv : live)
            ar.release((char *)0x10000 + kv.first);
        CHECK(ar.alloc(kArena) != nullptr, "released arena does not merge back into one range\n");
    }
    // choose_variant (each variant's schedule from the shared band edges,
    // with compile-time G and HR) against the plain loop over schedule():
    // the same variant and the same schedule, bit for bit, for random bands,
    // slopes, widths and first rows (serving pieces start mid-read)
    {
        for (int rep = 0; rep < 300000; ++rep) {
            BandDef band;
            int32_t wr;
            const int64_t n = 1 + (int64_t)(rng() % 5000), m = 1 + (int64_t)(rng() % 6000);
            const int64_t num = rng() % 3 ? (int64_t)(rng() % 7000) : 0, den = 1 + (int64_t)(rng() % 7000);
            const int32_t bw = rng() % 3 ? (int32_t)(rng() % 400) : -1;
            if (band_for(n + 2, m, bw, num, den, band, wr) != 0)
                continue;
            const int64_t row0 = rng() % 2 ? 0 : (int64_t)(rng() % 4000), rows = 1 + (int64_t)(rng() % 800);
            Sched ref{};
            int vref = -1;
            double best = -1;
            for (int v = 0; v < kNumVariants; ++v) {
                const Sched sv = schedule(band, row0, rows, kVariants[v][0], kVariants[v][1]);
                if (sv.s_end <= 0) {
                    ref = sv;
                    vref = 0;
                    break;
                }
                const double score = sv.eff / kSlotCost[v] * (1.0 + 0.02 * (kNumVariants - v));
                if (score > best) {
                    best = score;
                    vref = v;
                    ref = sv;
                }
            }
            Sched got{};
            const int v = choose_variant(band, row0, rows, got);
            CHECK(v == vref && got.dC == ref.dC && got.a0 == ref.a0 && got.s_end == ref.s_end &&
                      got.cells_est == ref.cells_est && got.eff == ref.eff,
                  "choose_variant differs from the loop over schedule() (n %lld m %lld row0 %lld)\n", (long long)rows,
                  (long long)m, (long long)row0);
            ++cases;
        }
    }
    // the serving path's flat hash map against std::unordered_map: random
    // inserts, lookups and erases (backward-shift deletion across the
    // array's wrap-around), keys from a small range (long probe runs), from
    // the whole 64-bit range (0 and ~0 included) and sequential (tickets),
    // with growth from the smallest size and clear()
    {
        for (int mode = 0; mode < 3; ++mode) {
            FlatMap64<uint64_t> fm;
            std::unordered_map<uint64_t, uint64_t> ref;
            uint64_t seq = 1;
            auto key = [&]() -> uint64_t {
                if (mode == 0)
                    return rng() % 512;
                if (mode == 1) {
                    const uint64_t k = ((uint64_t)rng() << 32) ^ rng();
                    return rng() % 16 == 0 ? (rng() % 2 ? 0ull : ~0ull) : k;
                }
                return rng() % 4 ? seq++ : seq - 1 - rng() % std::min<uint64_t>(seq, 300);
            };
            for (int op = 0; op < 300000; ++op) {
                const uint64_t k = key();
                const unsigned r = rng() % 10;
                if (r < 4) {
                    const uint64_t v = rng();
                    fm[k] = v;
                    ref[k] = v;
                } else if (r < 7) {
                    CHECK(fm.erase(k) == (ref.erase(k) == 1), "flat map erase disagrees (key %llu)\n",
                          (unsigned long long)k);
                } else {
                    const uint64_t *v = fm.find(k);
                    auto it = ref.find(k);
                    CHECK((v != nullptr) == (it != ref.end()) && (!v || *v == it->second),
                          "flat map lookup disagrees (key %llu)\n", (unsigned long long)k);
                }
                if (op % 50000 == 49999) {
                    for (auto &kv : ref) {
                        const uint64_t *v = fm.find(kv.first);
                        CHECK(v && *v == kv.second, "flat map lost a key\n");
                    }
                    CHECK(fm.size() == ref.size(), "flat map size %zu, expected %zu\n", fm.size(), ref.size());
                }
                if (op == 150000) {
                    fm.clear();
                    ref.clear();
                    CHECK(fm.size() == 0 && !fm.contains(k), "flat map clear\n");
                }
                ++cases;
            }
        }
    }
    printf("cases %llu steps %llu fails %d\n", (unsigned long long)cases, (unsigned long long)steps, fails);
    return fails ? 1 : 0;
}
