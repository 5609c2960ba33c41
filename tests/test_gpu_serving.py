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


def _aligner(pore, ref, ref_len, slots=64, arena=256 << 20, max_events=4000, early_reject=False):
    return B.Aligner(pore, ref, ref_len, arena_bytes=arena, serve_slots=slots, serve_max_events=max_events,
                     max_candidates=32, serve_early_reject=early_reject)


def _flat(reads):
    """Every read's events and candidates back to back, for submit_chunks."""
    ev_off = np.zeros(len(reads) + 1, np.int64)
    ev_off[1:] = np.cumsum([len(rd.events) for rd in reads])
    c_off = np.zeros(len(reads) + 1, np.int64)
    c_off[1:] = np.cumsum([len(rd.cands) for rd in reads])
    return (np.concatenate([rd.events for rd in reads]).astype(np.float32), ev_off,
            np.concatenate([rd.cands for rd in reads]), c_off)


def _run_reads_batched(al, reads, chunk=180):
    """As _run_reads with fixed chunks, but every round is one submit_chunks
    call, one flush and one poll_chunks call."""
    ev, ev_off, cands, c_off = _flat(reads)
    out = {rd.read_id: [] for rd in reads}
    pos = np.zeros(len(reads), np.int64)
    lens = np.array([len(rd.events) for rd in reads], np.int64)
    while np.any(pos < lens):
        q = np.nonzero(pos < lens)[0]
        ch = np.zeros(len(q), B.CHUNK_DTYPE)
        stop = np.minimum(pos[q] + chunk, lens[q])
        ch["read_id"] = [reads[x].read_id for x in q]
        ch["ev_offset"] = ev_off[q] + pos[q]
        ch["n_events"] = stop - pos[q]
        ch["cand_offset"] = np.where(pos[q] == 0, c_off[q], 0)
        ch["n_cands"] = np.where(pos[q] == 0, c_off[q + 1] - c_off[q], 0)
        ch["last"] = stop >= lens[q]
        tickets, status = B.rawalign_dtw_submit_chunks(al.h, ch, ev, cands)
        assert np.all(status == B.RA_OK) and np.all(tickets > 0)
        B.rawalign_dtw_flush(al.h)
        res, counts = B.rawalign_dtw_poll_chunks(al.h, tickets, int(c_off[-1]))
        at = 0
        for x, n in zip(q, counts):
            out[reads[x].read_id].append((int(stop[list(q).index(x)]), res[at:at + n]))
            at += n
        pos[q] = stop
    return out


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
        assert st.chunks == sum(len(x) for x in st.latencies_ms) and st.cells > 0
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


def test_batched_submit_and_poll_equal_one_by_one():
    """submit_chunks / poll_chunks give, chunk for chunk, the results of one
    submit_chunk / poll per chunk, and those equal the oracle's prefix DTW."""
    pore, ref, ref_len, reads = _serving_inputs(n_reads=10, max_events=700, seed=41)
    al = _aligner(pore, ref, ref_len)
    try:
        one = _run_reads(al, reads, [180])
    finally:
        al.close()
    al = _aligner(pore, ref, ref_len)
    try:
        many = _run_reads_batched(al, reads)
        stats = B.rawalign_dtw_serve_stats(al.h)
    finally:
        al.close()
    cells = 0
    for rd in reads:
        assert [q for q, _ in one[rd.read_id]] == [q for q, _ in many[rd.read_id]]
        for (_, a), (_, b) in zip(one[rd.read_id], many[rd.read_id]):
            for f in a.dtype.names:
                if f != "pad":  # padding is not part of the record's value
                    assert np.array_equal(a[f], b[f]), f
            cells += int(b["cells"].sum())
    _check_against_oracle(pore, ref, ref_len, reads[:3], many)
    assert stats.flushes == 4 and stats.chunks == 40 and stats.cells == cells
    assert stats.device_ms > 0 and stats.h2d_ms >= 0 and stats.d2h_ms >= 0


def test_poll_chunks_refuses_without_consuming():
    pore, ref, ref_len, reads = _serving_inputs(n_reads=2, max_events=360, seed=43)
    al = _aligner(pore, ref, ref_len)
    try:
        t0 = B.rawalign_dtw_submit_chunk(al.h, reads[0].read_id, reads[0].events[:180], reads[0].cands, False)
        t1 = B.rawalign_dtw_submit_chunk(al.h, reads[1].read_id, reads[1].events[:180], reads[1].cands, False)
        # queued, not flushed: not ready (waiting would not help)
        assert B.rawalign_dtw_poll_chunks(al.h, [t0], 64, timeout_us=-1) is None
        B.rawalign_dtw_flush(al.h)
        need = len(reads[0].cands) + len(reads[1].cands)
        for bad in ([t0, t1, t0], [t0, 12345678], [t0, t1]):
            with pytest.raises(B.RawAlignError) as ei:
                B.rawalign_dtw_poll_chunks(al.h, bad, need if len(bad) != 2 or bad[1] != t1 else need - 1)
            assert ei.value.code == B.RA_EINVAL
        res, counts = B.rawalign_dtw_poll_chunks(al.h, [t1, t0], need)
        assert list(counts) == [len(reads[1].cands), len(reads[0].cands)]
        assert np.all(res["read_id"][: counts[0]] == reads[1].read_id)
        with pytest.raises(B.RawAlignError):
            B.rawalign_dtw_poll_chunks(al.h, [t0], need)  # consumed
    finally:
        al.close()


def test_early_reject_decision():
    """With serve_early_reject a chunk before the last is decided UNMAPPED
    exactly when, for every candidate, fl(fl(B_Match * max_events) - cost)
    is below Score_Threshold (FP32, as the score): no later chunk can map
    the read.  Otherwise MAPPED when the best score reaches the threshold,
    else PENDING."""
    max_ev = 540
    pore, ref, ref_len, reads = _serving_inputs(n_reads=16, max_events=max_ev, seed=47)
    al = _aligner(pore, ref, ref_len, max_events=max_ev, early_reject=True)
    try:
        got = _run_reads_batched(al, reads)
    finally:
        al.close()
    _check_against_oracle(pore, ref, ref_len, reads[:4], got)
    xb = np.float32(0.4) * np.float32(max_ev)
    kinds = set()
    for rd in reads:
        for q, res in got[rd.read_id]:
            dec = set(res["decision"].tolist())
            assert len(dec) == 1
            dec = dec.pop()
            if q == len(rd.events):
                assert dec in (B.RA_MAPPED, B.RA_UNMAPPED)
                continue
            if np.max(res["score"]) >= np.float32(20.0):
                want = B.RA_MAPPED
            elif np.all((xb - res["cost"]).astype(np.float32) < np.float32(20.0)):
                want = B.RA_UNMAPPED
            else:
                want = B.RA_PENDING
            assert dec == want, (rd.read_id, q)
            kinds.add(want)
    assert B.RA_UNMAPPED in kinds and B.RA_PENDING in kinds


def test_serving_loop_with_early_reject():
    """The request loop with the library's reject decision: every read is
    accepted, rejected before its end or runs to max_events; rejects happen
    for off-target reads; the counters add up."""
    from paper_2310_05037_gb300.serving import ServingLoop

    pore, ref, ref_len, reads = _serving_inputs(n_reads=48, max_events=1080, seed=53)
    al = _aligner(pore, ref, ref_len, slots=16, max_events=1080, early_reject=True)
    try:
        st = ServingLoop(al, reads, max_events=1080).run(max_chunks=10 ** 6, in_flight=16)
        assert st.reads_done == len(reads)
        assert st.accepted + st.rejected + st.exhausted == st.reads_done
        assert st.rejected > 0 and st.accepted >= 0.8 * sum(rd.on_target for rd in reads)
        summ = st.summary()
        assert summ["chunks"] == st.chunks > 0 and summ["breakdown_ms"]["device_kernels"] > 0
        # every slot and block came back: a fresh batch of the same reads is admitted again
        st2 = ServingLoop(al, reads[:16], max_events=1080).run(max_chunks=10 ** 6, in_flight=16)
        assert st2.reads_done == 16
    finally:
        al.close()
