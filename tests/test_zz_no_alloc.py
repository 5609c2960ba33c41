"""The allocation-free single-alignment call against the batch call and the
oracle.

rawalign_dtw_align_noalloc serves callers that may not allocate device memory
(its working rows sit in a fixed array inside the library).  Here it runs
several times in a row on different alignments (derived band, no band, FREE
end, the largest read the fixed array holds), and each result must equal the
batch call's result for the same alignment and the FP32 oracle's, bit for bit
(the tolerance the other GPU tests use).  This file is collected last so that
a run stopping at the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_ROWS = 65536


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()


def _expected_signal(w, c):
    codes = S.unpack_bases(w.ref2bit, int(c["ref_offset"]), int(c["ref_len_bases"]))
    if c["strand"]:
        codes = (3 - codes[::-1]).astype(np.uint8)
    return S._kmer_means(codes, w.pore).astype(np.float32)


def _noalloc(ev, r, band_w, num, den, end_mode, b_match, stream):
    dev = torch.device("cuda:0")
    d_ev = torch.from_numpy(np.ascontiguousarray(ev, dtype=np.float32)).to(dev)
    d_r = torch.from_numpy(np.ascontiguousarray(r, dtype=np.float32)).to(dev)
    d_res = torch.zeros(B.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    rc = B.rawalign_dtw_align_noalloc(d_ev.data_ptr(), len(ev), d_r.data_ptr(), len(r), int(band_w), int(num),
                                      int(den), end_mode, float(b_match), d_res.data_ptr(), stream.cuda_stream)
    assert rc == B.RA_OK
    stream.synchronize()
    return np.frombuffer(d_res.cpu().numpy().tobytes(), dtype=B.RESULT_DTYPE)[0]


def _same_as_oracle(g, ev, r, band_w, num, den, end_mode, b_match):
    cost, ei, ej, cells, weff = O.dtw_f32(ev, r, band_w, num, den, end_mode)
    assert np.float32(g["cost"]).view(np.uint32) == np.float32(cost).view(np.uint32)
    sc = O.score_f32(b_match, len(ev), cost)
    assert np.float32(g["score"]).view(np.uint32) == np.float32(sc).view(np.uint32)
    assert (int(g["end_i"]), int(g["end_j"]), int(g["cells"]), int(g["w_eff"])) == (ei, ej, cells, weff)
    assert int(g["status"]) == 0


@pytest.mark.parametrize("end_mode", [B.RA_END_GLOBAL, B.RA_END_FREE])
def test_noalloc_matches_batch_call_and_oracle(end_mode):
    w = S.scaled("batched", "small")
    picks = [3, 11, 20]
    sub = w.subset(np.array(picks))
    cands = sub.cands.copy()
    cands[2]["band_w"] = -1  # one alignment without a band
    al = B.Aligner(sub.pore, sub.ref2bit, sub.ref_len, arena_bytes=64 << 20, kernel=B.RA_KERNEL_PLAIN,
                   end_mode=end_mode)
    try:
        want = al.align(sub.events, sub.read_offsets, cands)
    finally:
        al.close()
    stream = torch.cuda.Stream(device=torch.device("cuda:0"))
    got = []
    for q in range(len(picks)):  # back-to-back calls share the library's one scratch array
        c = cands[q]
        ev = sub.events[sub.read_offsets[c["read_id"]]: sub.read_offsets[c["read_id"] + 1]]
        r = _expected_signal(sub, c)
        g = _noalloc(ev, r, c["band_w"], c["slope_num"], c["slope_den"], end_mode, sub.b_match, stream)
        _same_as_oracle(g, ev, r, int(c["band_w"]), int(c["slope_num"]), int(c["slope_den"]), end_mode,
                        sub.b_match)
        got.append(g)
    for q in range(len(picks)):
        g, e = got[q], want[q]
        assert np.float32(g["cost"]).view(np.uint32) == np.float32(e["cost"]).view(np.uint32)
        assert np.float32(g["score"]).view(np.uint32) == np.float32(e["score"]).view(np.uint32)
        for f in ("end_i", "end_j", "cells", "w_eff", "status"):
            assert int(g[f]) == int(e[f]), f


def test_noalloc_largest_read_it_holds():
    """Exactly as many events as the fixed array has rows, twice in a row
    (both end modes), against the oracle."""
    rng = np.random.default_rng(65536)
    pore = S.pore_table(3)
    ref = S.hashed_reference(4, 200000)
    m = 700
    r = S._kmer_means(S.unpack_bases(ref, 1000, m + S.K - 1), pore).astype(np.float32)
    ev = rng.normal(size=MAX_ROWS).astype(np.float32)
    stream = torch.cuda.Stream(device=torch.device("cuda:0"))
    for end_mode, band_w in ((B.RA_END_GLOBAL, 40), (B.RA_END_FREE, -1)):
        g = _noalloc(ev, r, band_w, 0, 0, end_mode, 0.4, stream)
        _same_as_oracle(g, ev, r, band_w, 0, 0, end_mode, 0.4)


def test_noalloc_rejects_more_rows_than_its_scratch():
    dev = torch.device("cuda:0")
    d_ev = torch.zeros(MAX_ROWS + 1, dtype=torch.float32, device=dev)
    d_r = torch.zeros(100, dtype=torch.float32, device=dev)
    d_res = torch.zeros(B.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    rc = B.rawalign_dtw_align_noalloc(d_ev.data_ptr(), MAX_ROWS + 1, d_r.data_ptr(), 100, -1, 0, 0,
                                      B.RA_END_GLOBAL, 0.4, d_res.data_ptr(), s)
    assert rc == B.RA_EINVAL
    # an expected-signal length whose diagonal index would not fit: rejected
    # before anything is launched, so the small buffer is never read
    rc = B.rawalign_dtw_align_noalloc(d_ev.data_ptr(), 100, d_r.data_ptr(), 1 << 31, -1, 0, 0,
                                      B.RA_END_GLOBAL, 0.4, d_res.data_ptr(), s)
    assert rc == B.RA_EINVAL
    torch.cuda.synchronize()
