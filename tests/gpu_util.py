"""Helpers shared by the GPU tests: run a workload through the C ABI and
compare it with the oracle field by field."""
import numpy as np

import oracle as O
from paper_2310_05037_gb300 import binding as B
from paper_2310_05037_gb300 import synth as S

FIELDS_EXACT = ["read_id", "cand_idx", "end_i", "end_j", "w_eff", "cells", "is_best", "decision"]


def arena_bytes_for(w: S.Workload, slack=64 << 20):
    k = w.k
    m_total = int(np.sum(w.cands["ref_len_bases"].astype(np.int64) - k + 1)) if w.n_cands else 0
    need = B.rawalign_dtw_batch_bytes(len(w.events), w.n_reads, w.n_cands, m_total)
    need += len(w.ref2bit) + 4 * 4 ** k + slack
    max_n = int(w.read_lengths().max()) if w.n_reads else 1
    need += 12 * (max_n + 2) + (1 << 20)
    return (need + 255) // 256 * 256


def run_gpu(w: S.Workload, kernel=B.RA_KERNEL_AUTO, end_mode=None, graph_runs=0, **kw):
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w), k=w.k,
                   b_match=w.b_match, score_threshold=w.score_threshold,
                   end_mode=w.end_mode if end_mode is None else end_mode, kernel=kernel, **kw)
    try:
        if graph_runs:
            b = al.prepare(w.events, w.read_offsets, w.cands)
            outs = []
            for _ in range(graph_runs):
                t = al.run(b)
                outs.append(al.poll(t, w.n_cands))
            al.release(b)
            return outs
        return al.align(w.events, w.read_offsets, w.cands)
    finally:
        al.close()


def run_oracle(w: S.Workload, end_mode=None, use_f64=False):
    return O.map_batch(w.k, w.b_match, w.score_threshold, w.end_mode if end_mode is None else end_mode,
                       w.pore, w.ref2bit, w.ref_len, w.events, w.read_offsets, w.cands, use_f64=use_f64)


def assert_bit_exact(gpu, ora, idx=None, check_best=True):
    """Every result field equal; cost and score compared as bit patterns."""
    if idx is not None:
        ora_sel = ora
        gpu = gpu[idx]
    else:
        ora_sel = ora
    assert len(gpu) == len(ora_sel)
    assert np.all(gpu["status"] == 0)
    gc = gpu["cost"].view(np.uint32)
    oc = ora_sel["cost"].astype(np.float32).view(np.uint32)
    bad = np.nonzero(gc != oc)[0]
    assert len(bad) == 0, "cost differs at %s: gpu %s oracle %s" % (
        bad[:8], gpu["cost"][bad[:8]], ora_sel["cost"][bad[:8]])
    gs = gpu["score"].view(np.uint32)
    os_ = ora_sel["score"].astype(np.float32).view(np.uint32)
    assert np.array_equal(gs, os_), "score differs"
    for f in FIELDS_EXACT:
        if not check_best and f in ("is_best", "decision"):
            continue
        a = gpu[f].astype(np.int64)
        b = ora_sel[f].astype(np.int64)
        bad = np.nonzero(a != b)[0]
        assert len(bad) == 0, "%s differs at %s: gpu %s oracle %s" % (f, bad[:8], a[bad[:8]], b[bad[:8]])


def tiny_workload(seed, n_cands=3000, max_n=9, max_m=9, k=6):
    """Thousands of tiny alignments: random events, random regions, random
    bands (including none, w=0 and given slopes), both strands."""
    rng = np.random.default_rng(seed)
    pore = S.pore_table(seed)
    ref_len = 20000
    ref = S.hashed_reference(seed + 1, ref_len)
    reads = []
    rows = []
    for c in range(n_cands):
        n = int(rng.integers(1, max_n + 1))
        kind = rng.integers(0, 3)
        if kind == 0:
            ev = rng.normal(size=n)
        elif kind == 1:
            ev = rng.integers(-2, 3, size=n).astype(np.float64)
        else:
            ev = rng.normal(size=n) * 10.0 ** rng.integers(-3, 3, size=n)
        reads.append(ev.astype(np.float32))
        m = int(rng.integers(1, max_m + 1))
        span = m + k - 1
        off = int(rng.integers(0, ref_len - span))
        bw = int(rng.integers(-1, 5))
        if rng.random() < 0.3:
            num, den = int(rng.integers(0, 5)), int(rng.integers(1, 5))
        else:
            num, den = 0, 0
        rows.append((c, off, span, int(rng.random() < 0.3), bw, num, den))
    return S._finish("tiny", pore, ref, ref_len, reads, rows, dict(seed=seed))


def edge_workload(seed=7, k=6):
    """Shapes at the edges of the tiling: single row / column, no band, band
    wider than the table, given slopes whose end lies outside the band, rows
    equal to and around stripe heights (32, 64, 128, 256), reverse strand."""
    rng = np.random.default_rng(seed)
    pore = S.pore_table(seed)
    ref_len = 200000
    ref = S.hashed_reference(seed + 3, ref_len)
    reads, rows = [], []

    def add(n, m, bw=-1, num=0, den=0, strand=0, exact=False):
        q = len(reads)
        span = m + k - 1
        off = int(rng.integers(0, ref_len - span - 10))
        if exact:  # events equal the expected signal: cost 0 on the diagonal
            codes = S.unpack_bases(ref, off, span)
            if strand:
                codes = (3 - codes[::-1]).astype(np.uint8)
            means = S._kmer_means(codes, pore)
            ev = means[:n].astype(np.float32)
        else:
            ev = rng.normal(size=n).astype(np.float32)
        reads.append(ev)
        rows.append((q, off, span, strand, bw, num, den))

    for n, m in [(1, 1), (1, 40), (40, 1), (2, 2), (3, 700), (700, 3)]:
        add(n, m)
        add(n, m, bw=0)
    for n in [31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1000]:
        m = int(n * rng.uniform(0.9, 1.3))
        add(n, m, bw=int(0.1 * m))
        add(n, m, bw=3)
        add(n, m, bw=-1)
        add(n, m, bw=m + 5)
        add(n, m, bw=40, num=11, den=10)        # given slope: may end outside the band
        add(n, m, bw=64, num=7, den=10, strand=1)
    add(300, 300, bw=10, exact=True)
    add(300, 300, bw=-1, exact=True, strand=1)
    return S._finish("edges", pore, ref, ref_len, reads, rows, dict(seed=seed))


def run_gpu_anchored(w: S.Workload, kernel=B.RA_KERNEL_AUTO, graph_runs=0, **kw):
    """Anchor-guided batch through rawalign_dtw_submit_anchored (or, with
    graph_runs, prepare_anchored + replays)."""
    arena = arena_bytes_for(w) + 256 * (len(w.anchors) + w.n_cands) * 4
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=(arena + 255) // 256 * 256, k=w.k,
                   b_match=w.b_match, score_threshold=w.score_threshold, kernel=kernel, **kw)
    try:
        if graph_runs:
            b = al.prepare_anchored(w.events, w.read_offsets, w.cands, w.anchors, w.anchor_offsets)
            outs = [al.poll(al.run(b), w.n_cands) for _ in range(graph_runs)]
            al.release(b)
            return outs
        return al.align_anchored(w.events, w.read_offsets, w.cands, w.anchors, w.anchor_offsets)
    finally:
        al.close()


def run_oracle_anchored(w: S.Workload, use_f64=False):
    return O.map_anchored(w.k, w.b_match, w.score_threshold, w.pore, w.ref2bit, w.ref_len, w.events,
                          w.read_offsets, w.cands, w.anchors, w.anchor_offsets, use_f64=use_f64)


def tiny_anchored_workload(seed, n_cands=2000, max_n=12, max_m=12, k=6):
    """Small tables with random chains: anchors at the corners, adjacent
    anchors, gaps with rows only or columns only, empty chains; random and
    integer-valued events; both strands."""
    rng = np.random.default_rng(seed)
    pore = S.pore_table(seed)
    ref_len = 20000
    ref = S.hashed_reference(seed + 1, ref_len)
    reads, rows, chains = [], [], []
    for c in range(n_cands):
        n = int(rng.integers(1, max_n + 1))
        m = int(rng.integers(1, max_m + 1))
        ev = rng.normal(size=n) if rng.random() < 0.6 else rng.integers(-2, 3, size=n).astype(np.float64)
        reads.append(ev.astype(np.float32))
        span = m + k - 1
        rows.append((c, int(rng.integers(0, ref_len - span)), span, int(rng.random() < 0.3),
                     int(rng.integers(-1, 6)), 0, 0))
        chain, q, t = [], 0, 0
        for _ in range(int(rng.integers(0, 4))):
            if q >= n or t >= m:
                break
            q0 = int(rng.integers(q, min(n, q + 4)))
            t0 = int(rng.integers(t, min(m, t + 4)))
            ln = int(rng.integers(1, min(n - q0, m - t0) + 1))
            chain.append((q0, t0, ln))
            q, t = q0 + ln, t0 + ln
        chains.append(chain)
    w = S._finish("tiny_anchored", pore, ref, ref_len, reads, rows, dict(seed=seed))
    aoffs = np.zeros(n_cands + 1, np.uint64)
    aoffs[1:] = np.cumsum([len(ch) for ch in chains])
    flat = [a for ch in chains for a in ch]
    w.anchors = np.array(flat, dtype=S.ANCHOR_DTYPE) if flat else np.zeros(0, S.ANCHOR_DTYPE)
    w.anchor_offsets = aoffs
    return w
