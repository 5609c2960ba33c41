"""Read-Until serving through the C ABI (submit_chunk / flush / poll).

Each chunk's result must equal the oracle's DTW of the read prefix aligned so
far (FREE end, the candidate's given slope), bit for bit: resuming from the
carried frontier row is the same DP as aligning the prefix at once (Sec. 2.2).
A read's results must not depend on which other reads share its flushes, and
admission must refuse work when read slots or arena memory run out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()


def _serving_inputs(n_reads=12, max_events=900, seed=0x5EED0004):
    pore, ref, ref_len, reads = S.config_serving(seed=seed, n_reads=n_reads, ref_len=2_000_000,
                                                 max_events=max_events, cmax=6)
    return pore, ref, ref_len, reads


def _oracle_prefix(pore, ref, ref_len, cand, ev_prefix, b_match=0.4):
    codes = O.segment_codes(ref, ref_len, int(cand["ref_offset"]), int(cand["ref_len_bases"]), int(cand["strand"]))
    r = O.expected_signal(codes, 6, pore)
    cost, ei, ej, cells, weff = O.dtw_f32(ev_prefix, r, int(cand["band_w"]), int(cand["slope_num"]),
                                          int(cand["slope_den"]), O.END_FREE)
    return cost, O.score_f32(b_match, len(ev_prefix), cost), ei, ej


def _aligner(pore, ref, ref_len, slots=64, arena=256 << 20, max_events=4000):
    return B.Aligner(pore, ref, ref_len, arena_bytes=arena, serve_slots=slots, serve_max_events=max_events,
                     max_candidates=32)


def _run_reads(al, reads, chunk_sizes, rng_chunks=None):
    """Feeds every read chunk by chunk (all reads advance together, one flush
    per round); returns {read_id: [(prefix_len, results)]}."""
    out = {rd.read_id: [] for rd in reads}
    pos = {rd.read_id: 0 for rd in reads}
    rnd = 0
    while any(pos[rd.read_id] < len(rd.events) for rd in reads):
        tickets = []
        for rd in reads:
            p = pos[rd.read_id]
            if p >= len(rd.events):
                continue
            step = chunk_sizes[rnd % len(chunk_sizes)] if rng_chunks is None else int(rng_chunks.integers(1, 300))
            q = min(p + step, len(rd.events))
            last = q >= len(rd.events)
            t = B.rawalign_dtw_submit_chunk(al.h, rd.read_id, rd.events[p:q], rd.cands if p == 0 else None, last)
            tickets.append((rd.read_id, q, t))
            pos[rd.read_id] = q
        B.rawalign_dtw_flush(al.h)
        for rid, q, t in tickets:
            out[rid].append((q, B.rawalign_dtw_poll(al.h, t, 64)))
        rnd += 1
    return out


def _check_against_oracle(pore, ref, ref_len, reads, got, every=1):
    for rd in reads:
        for idx, (q, res) in enumerate(got[rd.read_id]):
            if idx % every and q != len(rd.events):
                continue
            assert len(res) == len(rd.cands)
            for c, cand in enumerate(rd.cands):
                cost, score, ei, ej = _oracle_prefix(pore, ref, ref_len, cand, rd.events[:q])
                g = res[c]
                assert np.float32(g["cost"]).view(np.uint32) == np.float32(cost).view(np.uint32), (rd.read_id, q, c)
                assert np.float32(g["score"]).view(np.uint32) == np.float32(score).view(np.uint32)
                assert (int(g["end_i"]), int(g["end_j"])) == (ei, ej)
                assert int(g["read_id"]) == rd.read_id and int(g["cand_idx"]) == c


def test_chunked_equals_prefix_dtw():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=10, max_events=700)
    al = _aligner(pore, ref, ref_len)
    try:
        got = _run_reads(al, reads, [180])
    finally:
        al.close()
    _check_against_oracle(pore, ref, ref_len, reads, got)


def test_ragged_chunks_equal_prefix_dtw():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=6, max_events=600, seed=77)
    al = _aligner(pore, ref, ref_len)
    try:
        got = _run_reads(al, reads, None, rng_chunks=np.random.default_rng(3))
    finally:
        al.close()
    _check_against_oracle(pore, ref, ref_len, reads, got)


def test_alone_equals_in_mix():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=16, max_events=540, seed=91)
    al = _aligner(pore, ref, ref_len)
    try:
        mix = _run_reads(al, reads, [180])
    finally:
        al.close()
    for rd in reads[:4]:
        al = _aligner(pore, ref, ref_len)
        try:
            alone = _run_reads(al, [rd], [180])
        finally:
            al.close()
        for (qa, ra), (qm, rm) in zip(alone[rd.read_id], mix[rd.read_id]):
            assert qa == qm
            for f in ("cost", "score", "end_i", "end_j", "cells"):
                assert np.array_equal(ra[f], rm[f]), f


def test_admission_by_read_slots():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=3, max_events=360)
    al = _aligner(pore, ref, ref_len, slots=2)
    try:
        t0 = B.rawalign_dtw_submit_chunk(al.h, reads[0].read_id, reads[0].events[:180], reads[0].cands, False)
        t1 = B.rawalign_dtw_submit_chunk(al.h, reads[1].read_id, reads[1].events[:180], reads[1].cands, False)
        with pytest.raises(B.RawAlignError) as ei:
            B.rawalign_dtw_submit_chunk(al.h, reads[2].read_id, reads[2].events[:180], reads[2].cands, False)
        assert ei.value.code == B.RA_EAGAIN
        # closing read 0 frees its slot once the flush carrying the close completes
        t2 = B.rawalign_dtw_submit_chunk(al.h, reads[0].read_id, reads[0].events[180:360], None, True)
        B.rawalign_dtw_flush(al.h)
        for t in (t0, t1, t2):
            assert B.rawalign_dtw_poll(al.h, t, 64) is not None
        t3 = B.rawalign_dtw_submit_chunk(al.h, reads[2].read_id, reads[2].events[:180], reads[2].cands, False)
        B.rawalign_dtw_flush(al.h)
        assert len(B.rawalign_dtw_poll(al.h, t3, 64)) == len(reads[2].cands)
    finally:
        al.close()


def test_admission_by_free_arena_memory():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=40, max_events=200)
    # room for the reference, the pore table and the state of a few reads
    # (a read here holds up to 6 x (384 + 2 x 192) floats of device state)
    arena = (len(ref) + 255) // 256 * 256 + 4 ** 6 * 4 + 256 + 60_000
    al = _aligner(pore, ref, ref_len, slots=1000, arena=(arena + 255) // 256 * 256)
    try:
        admitted, refused = 0, 0
        for rd in reads:
            try:
                B.rawalign_dtw_submit_chunk(al.h, rd.read_id, rd.events[:180], rd.cands, False)
                admitted += 1
            except B.RawAlignError as e:
                assert e.code == B.RA_EAGAIN
                refused += 1
        assert admitted > 0 and refused > 0
    finally:
        al.close()


def test_decision_maps_true_locus():
    """A read simulated from its first candidate's locus is mapped once its
    score passes Score_Threshold = 20 (Sec. 3.1); decisions are MAPPED or
    PENDING before the last chunk and MAPPED or UNMAPPED at the end."""
    pore, ref, ref_len, reads = _serving_inputs(n_reads=8, max_events=900, seed=5)
    al = _aligner(pore, ref, ref_len)
    try:
        got = _run_reads(al, reads, [180])
    finally:
        al.close()
    for rd in reads:
        hist = got[rd.read_id]
        for q, res in hist[:-1]:
            assert set(res["decision"]) <= {B.RA_MAPPED, B.RA_PENDING}
        assert set(hist[-1][1]["decision"]) <= {B.RA_MAPPED, B.RA_UNMAPPED}
        if rd.on_target:
            assert hist[-1][1]["decision"][0] == B.RA_MAPPED


def test_request_loop_closed_and_realtime():
    """The request loop decides every read it admits and keeps latencies."""
    from paper_2310_05037_gb300.serving import ServingLoop

    pore, ref, ref_len, reads = _serving_inputs(n_reads=40, max_events=1200, seed=11)
    al = _aligner(pore, ref, ref_len, slots=16, max_events=1200)
    try:
        st = ServingLoop(al, reads, max_events=1200).run(max_chunks=10 ** 6, in_flight=16)
        assert st.reads_done == len(reads)
        assert st.accepted + st.rejected + st.exhausted == st.reads_done
        assert st.chunks == len(st.latencies_ms) and st.cells > 0
        on = sum(rd.on_target for rd in reads)
        assert st.accepted >= on * 0.8
        rt = ServingLoop(al, reads[:8], max_events=1200).run(max_chunks=10 ** 6, in_flight=8, realtime=True,
                                                            chunk_s=0.05, duration_s=5.0, arrival_rate=100.0)
        assert rt.chunks > 0
    finally:
        al.close()


def test_decision_policy_study():
    """Read-Until decision policy replayed over thresholds: accepting at the
    handle's own threshold happens exactly where the library first says
    MAPPED; accepted counts never grow and rejected counts never shrink as
    the threshold rises; at Score_Threshold = 20 accepted reads map to their
    true locus."""
    from paper_2310_05037_gb300.serving import collect_trajectories, decision_study

    pore, ref, ref_len, reads = _serving_inputs(n_reads=24, max_events=900, seed=17)
    al = _aligner(pore, ref, ref_len, slots=24, max_events=900)
    try:
        trs = collect_trajectories(al, reads, chunk=180, max_events=900, in_flight=24)
    finally:
        al.close()
    assert len(trs) == len(reads)
    for tr in trs:
        k_lib = next((k for k, f in enumerate(tr.mapped) if f), None)
        k_thr = next((k for k, sc in enumerate(tr.best_score) if sc >= np.float32(20.0)), None)
        assert k_lib == k_thr
    thresholds = [5.0, 10.0, 20.0, 40.0, 80.0]
    st = decision_study(trs, thresholds, max_events=900)
    acc = [st[t]["accepted"] for t in thresholds]
    rej = [st[t]["rejected"] for t in thresholds]
    assert acc == sorted(acc, reverse=True) and rej == sorted(rej)
    assert all(st[t]["accepted"] + st[t]["rejected"] + st[t]["undecided"] == len(reads) for t in thresholds)
    assert st[20.0]["accepted"] > 0 and st[20.0]["precision"] >= 0.9
