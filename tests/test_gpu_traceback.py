"""Warping-path output (rawalign_dtw_traceback) through the C ABI against the
oracle's traceback: the same path cell for cell (NW, N, W on ties), the same
cost bit for bit, for tiny tables with every band shape, the tiling edges,
both end modes and both strands, and against the batch path's cost."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import arena_bytes_for, edge_workload, run_gpu, tiny_workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def _oracle_one(w, c, end_mode):
    cand = w.cands[c]
    rid = int(cand["read_id"])
    e = w.events[w.read_offsets[rid]:w.read_offsets[rid + 1]]
    codes = O.segment_codes(w.ref2bit, w.ref_len, int(cand["ref_offset"]), int(cand["ref_len_bases"]),
                            int(cand["strand"]))
    r = O.expected_signal(codes, w.k, w.pore)
    cost, path = O.traceback_f32(e, r, int(cand["band_w"]), int(cand["slope_num"]), int(cand["slope_den"]),
                                 end_mode)
    return e, cost, path


def _check(w, idx, end_mode):
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w) + (64 << 20), k=w.k,
                   b_match=w.b_match)
    try:
        for c in idx:
            e, cost, path = _oracle_one(w, c, end_mode)
            res, gpath = al.traceback(e, w.cands[c], end_mode)
            assert np.float32(res["cost"]).view(np.uint32) == np.float32(cost).view(np.uint32), c
            assert np.array_equal(gpath, path), (c, gpath[:6], path[:6])
            if len(path):
                assert (int(res["end_i"]), int(res["end_j"])) == tuple(int(x) for x in path[-1])
    finally:
        al.close()


@pytest.mark.parametrize("end_mode", [B.RA_END_GLOBAL, B.RA_END_FREE])
def test_tiny_tables(end_mode):
    w = tiny_workload(71 + end_mode, n_cands=400)
    _check(w, range(w.n_cands), end_mode)


@pytest.mark.parametrize("end_mode", [B.RA_END_GLOBAL, B.RA_END_FREE])
def test_tiling_edges(end_mode):
    w = edge_workload()
    _check(w, range(w.n_cands), end_mode)


def test_batched_candidates_and_batch_cost():
    w = S.scaled("batched", "small").subset(np.arange(30))
    _check(w, range(w.n_cands), B.RA_END_GLOBAL)
    batch = run_gpu(w)
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w) + (64 << 20), k=w.k)
    try:
        for c in range(w.n_cands):
            rid = int(w.cands[c]["read_id"])
            res, _ = al.traceback(w.events[w.read_offsets[rid]:w.read_offsets[rid + 1]], w.cands[c])
            for f in ("cost", "score", "end_i", "end_j", "cells", "w_eff"):
                assert res[f] == batch[c][f], f
    finally:
        al.close()


def test_bad_arguments():
    w = S.scaled("batched", "small").subset(np.arange(2))
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w) + (64 << 20), k=w.k)
    try:
        e = w.events[: int(w.read_offsets[1])].copy()
        e[3] = np.inf
        with pytest.raises(B.RawAlignError) as ei:
            al.traceback(e, w.cands[0])
        assert ei.value.code == B.RA_EINVAL
        with pytest.raises(B.RawAlignError):
            al.traceback(w.events[:5], w.cands[0], end_mode=7)
    finally:
        al.close()
