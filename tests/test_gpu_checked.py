"""The checked build of the library (RAWALIGN_CHECKED: every planned work
item's extents and ring size are checked on the device before it runs; a
failing item is reported through the error word, and poll returns
RA_EDEVICE instead of touching memory outside its arrays).  Here it runs the
tiny, tiling-edge, anchored and serving workloads: no item may fail its
checks, and the results must equal the oracle's bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import (assert_bit_exact, edge_workload, run_gpu, run_gpu_anchored, run_oracle,  # noqa: E402
                      run_oracle_anchored, tiny_anchored_workload, tiny_workload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2310_05037_gb300 import build

    path = build.build(checked=True)
    saved = B._lib
    B._lib = None
    B.load(path)
    yield path
    B._lib = saved


@pytest.mark.parametrize("kernel", [B.RA_KERNEL_AUTO, B.RA_KERNEL_PLAIN, B.RA_KERNEL_VARIANT0 + 9])
def test_checked_tiny_and_edges(checked_lib, kernel):
    for w in (tiny_workload(31, n_cands=1500), edge_workload(8)):
        for end in (O.END_GLOBAL, O.END_FREE):
            assert_bit_exact(run_gpu(w, kernel=kernel, end_mode=end), run_oracle(w, end_mode=end))


def test_checked_batches(checked_lib):
    for name in ("batched", "readuntil", "longread"):
        w = S.scaled(name, "small")
        assert_bit_exact(run_gpu(w), run_oracle(w))
    w = tiny_anchored_workload(5, n_cands=800)
    assert_bit_exact(run_gpu_anchored(w), run_oracle_anchored(w))


def test_checked_serving(checked_lib):
    pore, ref, ref_len, reads = S.config_serving(seed=61, n_reads=6, ref_len=2_000_000, max_events=540, cmax=6)
    al = B.Aligner(pore, ref, ref_len, arena_bytes=256 << 20, serve_slots=8, serve_max_events=540, max_candidates=32)
    try:
        for p in range(0, 540, 180):
            tickets = [B.rawalign_dtw_submit_chunk(al.h, rd.read_id, rd.events[p:p + 180], rd.cands if p == 0 else None,
                                                   p + 180 >= 540) for rd in reads]
            B.rawalign_dtw_flush(al.h)
            for rd, t in zip(reads, tickets):
                res = B.rawalign_dtw_poll(al.h, t, 64)
                assert np.all(res["status"] == 0)
                for c, cand in enumerate(rd.cands):
                    codes = O.segment_codes(ref, ref_len, int(cand["ref_offset"]), int(cand["ref_len_bases"]), 0)
                    r = O.expected_signal(codes, 6, pore)
                    cost, ei, ej, cells, weff = O.dtw_f32(rd.events[:p + 180], r, int(cand["band_w"]),
                                                          int(cand["slope_num"]), int(cand["slope_den"]), O.END_FREE)
                    assert np.float32(res["cost"][c]).view(np.uint32) == np.float32(cost).view(np.uint32)
                    assert (int(res["end_i"][c]), int(res["end_j"][c])) == (ei, ej)
    finally:
        al.close()
