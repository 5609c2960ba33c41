"""Full-size parity: each batch workload at its full size, run the way the
benchmark runs it (one prepared batch, automatic variant choice and launch
classes, replays of the captured CUDA graphs), checked three ways:

  * every result against properties that hold at any size: status, record
    identity, GLOBAL end cell (n-1, m-1), score = fl(fl(B_Match * N_Read) - C)
    (Sec. 2.3), per-read best candidate and decision, identical replays;
  * whole reads sampled at random (plus the extreme ones) against the FP32
    oracle, bit for bit on every field, and against its FP64 run within
    1e-5 relative;
  * the longest alignments, too large for the oracle, between two bounds
    that any warping path fixes: the sum over rows of the smallest in-band
    |e_i - r_j| (every row holds at least one path cell, Sec. 2.2) and the
    cost of one explicit in-band path along the band's centre line.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import run_gpu  # noqa: E402

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


def _expected(w, c):
    cand = w.cands[c]
    codes = O.segment_codes(w.ref2bit, w.ref_len, int(cand["ref_offset"]), int(cand["ref_len_bases"]),
                            int(cand["strand"]))
    return O.expected_signal(codes, w.k, w.pore).astype(np.float64)


def _bounds(w, c):
    """(lower, upper) bounds on the exact DTW cost of candidate c."""
    cand = w.cands[c]
    r0 = int(w.read_offsets[int(cand["read_id"])])
    r1 = int(w.read_offsets[int(cand["read_id"]) + 1])
    e = w.events[r0:r1].astype(np.float64)
    r = _expected(w, c)
    n, m = len(e), len(r)
    band = O.band_params(n, m, int(cand["band_w"]), int(cand["slope_num"]), int(cand["slope_den"]))
    assert not band.unbanded
    num, den, wb = int(band.num), int(band.den), int(band.w_eff)
    # lower: each row's smallest in-band difference (in-band columns of row i
    # are the integers j with |j*den - i*num| <= w*den; checked at the ends)
    lower = 0.0
    for i in range(n):
        lo = max(0, -((wb * den - i * num) // den))
        hi = min(m - 1, (i * num + wb * den) // den)
        assert O.in_band(band, i, lo) and O.in_band(band, i, hi)
        assert not (lo > 0 and O.in_band(band, i, lo - 1)) and not (hi < m - 1 and O.in_band(band, i, hi + 1))
        lower += float(np.min(np.abs(e[i] - r[lo:hi + 1])))
    # upper: the staircase through c_i = floor(i*num/den); along row i it walks
    # c_i .. c_{i+1}-1 and then steps diagonally (or down) to (i+1, c_{i+1})
    ci = (np.arange(n, dtype=np.int64) * num) // den
    upper = 0.0
    for i in range(n):
        j_end = ci[i + 1] - 1 if i + 1 < n else m - 1
        j_end = max(j_end, ci[i])
        js = np.arange(ci[i], j_end + 1)
        for j in (int(js[0]), int(js[-1])):
            assert O.in_band(band, i, j)
        upper += float(np.sum(np.abs(e[i] - r[js])))
    return lower, upper, n + m


def _run_full(name):
    w = S.scaled(name, "full")
    outs = run_gpu(w, graph_runs=2)
    a, b = outs
    for f in a.dtype.names:
        assert np.array_equal(a[f], b[f]), f
    _check_properties(w, a)
    return w, a


def test_full_plain():
    w, g = _run_full("plain")
    _check_sample(w, g, np.arange(w.n_cands))


def test_full_batched():
    w, g = _run_full("batched")
    rng = np.random.default_rng(21)
    lens = w.read_lengths()
    counts = np.bincount(w.cands["read_id"].astype(np.int64), minlength=w.n_reads)
    reads = set(rng.choice(w.n_reads, 40, replace=False).tolist())
    reads |= {int(np.argmax(lens)), int(np.argmin(lens)), int(np.argmax(counts))}
    _check_sample(w, g, _whole_reads(w, sorted(reads)))


def test_full_readuntil():
    w, g = _run_full("readuntil")
    rng = np.random.default_rng(22)
    counts = np.bincount(w.cands["read_id"].astype(np.int64), minlength=w.n_reads)
    reads = set(rng.choice(w.n_reads, 24, replace=False).tolist()) | {int(np.argmax(counts))}
    _check_sample(w, g, _whole_reads(w, sorted(reads)))


def test_full_longread():
    w, g = _run_full("longread")
    lens = w.read_lengths()
    order = np.argsort(lens, kind="stable")
    _check_sample(w, g, _whole_reads(w, order[:2]))
    # the longest alignments: between the row-minimum and the centre-path bounds
    n, m = _dims(w)
    for c in np.argsort(n * m, kind="stable")[-2:]:
        lower, upper, steps = _bounds(w, int(c))
        cost = float(g["cost"][c])
        tol = steps * U32
        assert lower * (1 - tol) <= cost <= upper * (1 + tol), (c, lower, cost, upper)


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
