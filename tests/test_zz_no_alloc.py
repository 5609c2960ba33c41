"""The allocation-free single-alignment call against the batch call.

rawalign_dtw_align_noalloc serves callers that may not allocate device memory
(its working rows sit in a fixed array inside the library).  Here it runs
twice in a row, on two different alignments, and each result must equal the
batch call's result for the same alignment bit for bit (the tolerance the
other GPU tests use).  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()


def _expected_signal(w, c):
    codes = S.unpack_bases(w.ref2bit, int(c["ref_offset"]), int(c["ref_len_bases"]))
    if c["strand"]:
        codes = (3 - codes[::-1]).astype(np.uint8)
    return S._kmer_means(codes, w.pore).astype(np.float32)


def test_noalloc_matches_batch_call_twice():
    w = S.scaled("batched", "small")
    picks = [3, 11]  # two different alignments, one call each, back to back
    sub = w.subset(np.array(picks))
    al = B.Aligner(sub.pore, sub.ref2bit, sub.ref_len, arena_bytes=64 << 20, kernel=B.RA_KERNEL_PLAIN)
    try:
        want = al.align(sub.events, sub.read_offsets, sub.cands)
    finally:
        al.close()
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    lens = sub.read_lengths()
    got = []
    for q in range(len(picks)):
        c = sub.cands[q]
        ev = sub.events[sub.read_offsets[c["read_id"]]: sub.read_offsets[c["read_id"] + 1]]
        r = _expected_signal(sub, c)
        d_ev = torch.from_numpy(np.ascontiguousarray(ev)).to(dev)
        d_r = torch.from_numpy(r).to(dev)
        d_res = torch.zeros(B.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        rc = B.rawalign_dtw_align_noalloc(d_ev.data_ptr(), int(lens[c["read_id"]]), d_r.data_ptr(), len(r),
                                          int(c["band_w"]), int(c["slope_num"]), int(c["slope_den"]),
                                          B.RA_END_GLOBAL, float(sub.b_match), d_res.data_ptr(), stream.cuda_stream)
        assert rc == B.RA_OK
        stream.synchronize()
        got.append(np.frombuffer(d_res.cpu().numpy().tobytes(), dtype=B.RESULT_DTYPE)[0])
    for q in range(len(picks)):
        g, e = got[q], want[q]
        assert np.float32(g["cost"]).view(np.uint32) == np.float32(e["cost"]).view(np.uint32)
        assert np.float32(g["score"]).view(np.uint32) == np.float32(e["score"]).view(np.uint32)
        for f in ("end_i", "end_j", "cells", "w_eff", "status"):
            assert int(g[f]) == int(e[f]), f


def test_noalloc_rejects_more_rows_than_its_scratch():
    dev = torch.device("cuda:0")
    d_ev = torch.zeros(70000, dtype=torch.float32, device=dev)
    d_r = torch.zeros(100, dtype=torch.float32, device=dev)
    d_res = torch.zeros(B.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    rc = B.rawalign_dtw_align_noalloc(d_ev.data_ptr(), 70000, d_r.data_ptr(), 100, -1, 0, 0, B.RA_END_GLOBAL, 0.4,
                                      d_res.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == B.RA_EINVAL
