"""Full-size parity: each batch workload at its full size, run the way the
benchmark runs it (one prepared batch, automatic variant choice and launch
classes, replays of the captured CUDA graphs), checked three ways:

  * every result against properties that hold at any size: status, record
    identity, GLOBAL end cell (n-1, m-1), score = fl(fl(B_Match * N_Read) - C)
    (Sec. 2.3), per-read best candidate and decision, identical replays;
  * every alignment of the plain, batched-uneven and Read-Until workloads
    against the FP32 oracle, bit for bit on every field (the unchanged
    single-threaded oracle, run on groups of whole reads over all host cores);
    the long-read workload's eight longest alignments and forty random ones
    the same way; sampled reads against the FP64 run within 1e-5 relative;
  * the serving workload: 32 reads carried to 4000 events in 180-event chunks,
    every chunk of every candidate against the oracle's DTW of the prefix.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import run_gpu  # noqa: E402
from oracle_pool import map_parallel  # noqa: E402

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def _dims(w):
    n = w.read_lengths()[w.cands["read_id"].astype(np.int64)]
    m = w.cands["ref_len_bases"].astype(np.int64) - w.k + 1
    return n, m


def _check_properties(w, g):
    n, m = _dims(w)
    assert len(g) == w.n_cands
    assert np.all(g["status"] == 0)
    assert np.array_equal(g["read_id"].astype(np.int64), w.cands["read_id"].astype(np.int64))
    assert np.array_equal(g["cand_idx"].astype(np.int64), np.arange(w.n_cands))
    # default slope: the corner cell is always in band, so every cost is finite
    assert np.all(np.isfinite(g["cost"])) and np.all(g["cost"] >= 0)
    assert np.array_equal(g["end_i"].astype(np.int64), n - 1)
    assert np.array_equal(g["end_j"].astype(np.int64), m - 1)
    sc = np.float32(w.b_match) * n.astype(np.float32)
    sc = (sc.astype(np.float32) - g["cost"]).astype(np.float32)
    assert np.array_equal(sc.view(np.uint32), g["score"].view(np.uint32))
    assert np.all(g["cells"] > 0) and np.all(g["cells"] <= n * m)
    # per read: first candidate with the highest score is the best one
    rid = w.cands["read_id"].astype(np.int64)
    order = np.lexsort((np.arange(w.n_cands), -g["score"].astype(np.float64), rid))
    first = np.ones(w.n_cands, bool)
    first[1:] = rid[order][1:] != rid[order][:-1]
    best = np.zeros(w.n_cands, bool)
    best[order[first]] = True
    assert np.array_equal(g["is_best"].astype(bool), best)
    best_score = np.full(w.n_reads, -np.inf)
    np.maximum.at(best_score, rid, g["score"].astype(np.float64))
    want = np.where(best_score[rid] >= np.float32(w.score_threshold), B.RA_MAPPED, B.RA_UNMAPPED)
    assert np.array_equal(g["decision"].astype(np.int64), want)


def _whole_reads(w, reads):
    rid = w.cands["read_id"].astype(np.int64)
    return np.nonzero(np.isin(rid, np.asarray(reads, np.int64)))[0]


def _check_sample(w, g, idx):
    sub = w.subset(idx)
    o = O.map_batch(sub.k, sub.b_match, sub.score_threshold, sub.end_mode, sub.pore, sub.ref2bit, sub.ref_len,
                    sub.events, sub.read_offsets, sub.cands)
    gs = g[idx]
    assert np.array_equal(gs["cost"].view(np.uint32), o["cost"].astype(np.float32).view(np.uint32)), \
        "cost differs at %s" % idx[np.nonzero(gs["cost"] != o["cost"])[0][:8]]
    assert np.array_equal(gs["score"].view(np.uint32), o["score"].astype(np.float32).view(np.uint32))
    for f in ("end_i", "end_j", "w_eff", "cells", "is_best", "decision"):
        assert np.array_equal(gs[f].astype(np.int64), o[f].astype(np.int64)), f
    o64 = O.map_batch(sub.k, sub.b_match, sub.score_threshold, sub.end_mode, sub.pore, sub.ref2bit, sub.ref_len,
                      sub.events, sub.read_offsets, sub.cands, use_f64=True)
    c64 = o64["cost64"]
    rel = np.abs(gs["cost"].astype(np.float64) - c64) / np.maximum(c64, 1e-30)
    assert rel.max() < 1e-5, rel.max()


def _run_full(name):
    w = S.scaled(name, "full")
    outs = run_gpu(w, graph_runs=2)
    a, b = outs
    for f in a.dtype.names:
        assert np.array_equal(a[f], b[f]), f
    _check_properties(w, a)
    return w, a


def _check_all(w, g, idx=None, label=""):
    """Every selected alignment against the FP32 oracle, bit for bit."""
    o, info = map_parallel(w, idx)
    gs = g if idx is None else g[idx]
    bad = np.nonzero(gs["cost"].view(np.uint32) != o["cost"].astype(np.float32).view(np.uint32))[0]
    assert len(bad) == 0, "cost differs at %s" % (bad[:8] if idx is None else np.asarray(idx)[bad[:8]])
    assert np.array_equal(gs["score"].view(np.uint32), o["score"].astype(np.float32).view(np.uint32))
    for f in ("read_id", "cand_idx", "end_i", "end_j", "w_eff", "cells", "is_best", "decision"):
        assert np.array_equal(gs[f].astype(np.int64), o[f].astype(np.int64)), f
    print("%s: %d alignments bit-exact vs the FP32 oracle (%.3g cells) in %.1f s on %d host threads"
          % (label, len(o), float(o["cells"].sum()), info["seconds"], info["threads"]))


def test_full_plain():
    w, g = _run_full("plain")
    _check_sample(w, g, np.arange(w.n_cands))


def test_full_batched():
    w, g = _run_full("batched")
    _check_all(w, g, label="batched uneven")
    rng = np.random.default_rng(21)
    lens = w.read_lengths()
    counts = np.bincount(w.cands["read_id"].astype(np.int64), minlength=w.n_reads)
    reads = set(rng.choice(w.n_reads, 40, replace=False).tolist())
    reads |= {int(np.argmax(lens)), int(np.argmin(lens)), int(np.argmax(counts))}
    _check_sample(w, g, _whole_reads(w, sorted(reads)))


def test_full_readuntil():
    w, g = _run_full("readuntil")
    _check_all(w, g, label="Read-Until prefix")
    rng = np.random.default_rng(22)
    counts = np.bincount(w.cands["read_id"].astype(np.int64), minlength=w.n_reads)
    reads = set(rng.choice(w.n_reads, 24, replace=False).tolist()) | {int(np.argmax(counts))}
    _check_sample(w, g, _whole_reads(w, sorted(reads)))


def test_full_longread():
    w, g = _run_full("longread")
    n, m = _dims(w)
    rng = np.random.default_rng(24)
    longest = np.argsort(n * m, kind="stable")[-8:]
    others = np.setdiff1d(np.arange(w.n_cands), longest)
    idx = np.concatenate([longest, rng.choice(others, 40, replace=False)])
    # whole reads, so that is_best and the decision are the oracle's too
    idx = _whole_reads(w, np.unique(w.cands["read_id"][idx].astype(np.int64)))
    _check_all(w, g, idx, label="long read (longest and random)")
    # FP64: the rigorous bound (every DP value is a sum of at most n+m-1
    # non-negative terms) and the measured relative difference
    o64, _ = map_parallel(w, longest, use_f64=True)
    rel = np.abs(g["cost"][longest].astype(np.float64) - o64["cost64"]) / o64["cost64"]
    assert np.all(rel <= (n[longest] + m[longest]) * U32), rel
    print("long read: FP32 vs FP64 relative difference of the 8 longest costs: max %.3g" % rel.max())


def test_full_serving_to_max_events():
    """Serving at the serving workload's sizes: 32 reads of up to 32
    candidates carried to 4000 events in 180-event chunks (Sec. 3.1); every
    chunk's result for every candidate equals the oracle's DTW of the prefix
    aligned so far (FREE end, the candidate's slope), bit for bit."""
    import concurrent.futures as cf

    from oracle_pool import cores

    pore, ref, ref_len, reads = S.config_serving(n_reads=32)
    reads = [rd for rd in reads]
    al = B.Aligner(pore, ref, ref_len, arena_bytes=len(ref) + (512 << 20), serve_slots=32,
                   serve_max_events=4000, max_candidates=32)
    got = {rd.read_id: [] for rd in reads}
    try:
        for p in range(0, 4000, 180):
            q = min(p + 180, 4000)
            tickets = [(rd, B.rawalign_dtw_submit_chunk(al.h, rd.read_id, rd.events[p:q],
                                                        rd.cands if p == 0 else None, q == 4000))
                       for rd in reads]
            B.rawalign_dtw_flush(al.h)
            for rd, t in tickets:
                got[rd.read_id].append((q, B.rawalign_dtw_poll(al.h, t, 64)))
    finally:
        al.close()
    O.lib()

    def check(job):
        rd, c = job
        cand = rd.cands[c]
        codes = O.segment_codes(ref, ref_len, int(cand["ref_offset"]), int(cand["ref_len_bases"]),
                                int(cand["strand"]))
        r = O.expected_signal(codes, 6, pore)
        bad = []
        for q, res in got[rd.read_id]:
            cost, ei, ej, cells, weff = O.dtw_f32(rd.events[:q], r, int(cand["band_w"]), int(cand["slope_num"]),
                                                  int(cand["slope_den"]), O.END_FREE)
            sc = O.score_f32(0.4, q, cost)
            gr = res[c]
            if (np.float32(gr["cost"]).view(np.uint32) != np.float32(cost).view(np.uint32)
                    or np.float32(gr["score"]).view(np.uint32) != np.float32(sc).view(np.uint32)
                    or (int(gr["end_i"]), int(gr["end_j"])) != (ei, ej) or int(gr["cand_idx"]) != c
                    or int(gr["read_id"]) != rd.read_id):
                bad.append((rd.read_id, c, q))
        return bad, len(got[rd.read_id])

    jobs = [(rd, c) for rd in reads for c in range(len(rd.cands))]
    with cf.ThreadPoolExecutor(max_workers=cores()) as ex:
        outs = list(ex.map(check, jobs))
    bad = [b for o, _ in outs for b in o]
    assert not bad, bad[:8]
    assert all(len(got[rd.read_id]) == 23 for rd in reads)
    print("serving: %d candidate chunks bit-exact vs the oracle's prefix DTW" % sum(k for _, k in outs))


def test_full_anchored():
    """Anchor-guided batch at the batched workload's full size (Sec. 2.4.2)."""
    from gpu_util import run_gpu_anchored

    w = S.scaled("anchored", "full")
    a, b = run_gpu_anchored(w, graph_runs=2)
    for f in a.dtype.names:
        assert np.array_equal(a[f], b[f]), f
    _check_properties(w, a)
    rng = np.random.default_rng(23)
    lens = w.read_lengths()
    reads = set(rng.choice(w.n_reads, 40, replace=False).tolist()) | {int(np.argmax(lens))}
    idx = _whole_reads(w, sorted(reads))
    sub = w.subset(idx)
    args = (sub.k, sub.b_match, sub.score_threshold, sub.pore, sub.ref2bit, sub.ref_len, sub.events,
            sub.read_offsets, sub.cands, sub.anchors, sub.anchor_offsets)
    o = O.map_anchored(*args)
    gs = a[idx]
    assert np.array_equal(gs["cost"].view(np.uint32), o["cost"].astype(np.float32).view(np.uint32))
    assert np.array_equal(gs["score"].view(np.uint32), o["score"].astype(np.float32).view(np.uint32))
    for f in ("end_i", "end_j", "w_eff", "cells", "is_best", "decision"):
        assert np.array_equal(gs[f].astype(np.int64), o[f].astype(np.int64)), f
    c64 = O.map_anchored(*args, use_f64=True)["cost64"]
    assert (np.abs(gs["cost"].astype(np.float64) - c64) / np.maximum(c64, 1e-30)).max() < 1e-5
