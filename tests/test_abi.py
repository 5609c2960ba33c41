"""CPU-only checks of the boundary: the library builds, loads, and exports
every entry point the public header declares; the record layouts seen by C,
by the ctypes binding, by the input generator and by the oracle agree."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2310_05037_gb300 import binding as B
from paper_2310_05037_gb300 import build as BUILD
from paper_2310_05037_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rawalign_dtw.h")


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load()


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(rawalign_dtw_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rawalign_dtw_create", "rawalign_dtw_submit_batch", "rawalign_dtw_submit_chunk",
              "rawalign_dtw_poll", "rawalign_dtw_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(rawalign_dtw_\w+)$", out, re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert s in B.SIGNATURES, s
        getattr(lib, s)


def _c_layout():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "rawalign_dtw.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("cand %zu\nres %zu\ncfg %zu\nstats %zu\nanchor %zu\nchunk %zu\nsstats %zu\n",
         sizeof(rawalign_candidate_t), sizeof(rawalign_result_t), sizeof(rawalign_dtw_config_t),
         sizeof(rawalign_dtw_stats_t), sizeof(rawalign_anchor_t), sizeof(rawalign_chunk_t),
         sizeof(rawalign_dtw_serve_stats_t));
  O(rawalign_chunk_t, read_id); O(rawalign_chunk_t, ev_offset); O(rawalign_chunk_t, n_events);
  O(rawalign_chunk_t, cand_offset); O(rawalign_chunk_t, n_cands); O(rawalign_chunk_t, last);
  O(rawalign_dtw_serve_stats_t, cells); O(rawalign_dtw_serve_stats_t, host_submit_ms);
  O(rawalign_dtw_serve_stats_t, d2h_ms);
  O(rawalign_dtw_stats_t, split); O(rawalign_dtw_stats_t, host_plan_ms); O(rawalign_dtw_stats_t, host_upload_ms);
  O(rawalign_anchor_t, q); O(rawalign_anchor_t, t); O(rawalign_anchor_t, len);
  O(rawalign_candidate_t, read_id); O(rawalign_candidate_t, ref_offset); O(rawalign_candidate_t, ref_len_bases);
  O(rawalign_candidate_t, strand); O(rawalign_candidate_t, band_w); O(rawalign_candidate_t, slope_num);
  O(rawalign_candidate_t, slope_den);
  O(rawalign_result_t, cand_idx); O(rawalign_result_t, cost); O(rawalign_result_t, score); O(rawalign_result_t, end_i);
  O(rawalign_result_t, end_j); O(rawalign_result_t, w_eff); O(rawalign_result_t, cells); O(rawalign_result_t, status);
  O(rawalign_result_t, is_best); O(rawalign_result_t, decision);
  O(rawalign_dtw_config_t, arena_dev); O(rawalign_dtw_config_t, arena_bytes); O(rawalign_dtw_config_t, cuda_stream);
  O(rawalign_dtw_config_t, max_candidates); O(rawalign_dtw_config_t, kernel); O(rawalign_dtw_config_t, autotune_path);
  O(rawalign_dtw_config_t, early_termination); O(rawalign_dtw_config_t, serve_early_reject);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    return dict(l.split() for l in lines if l.strip())


def test_record_layouts_agree():
    lay = _c_layout()
    assert int(lay["cand"]) == C.sizeof(B.Candidate) == S.CANDIDATE_DTYPE.itemsize == C.sizeof(O.Candidate) == 48
    assert int(lay["res"]) == C.sizeof(B.Result) == B.RESULT_DTYPE.itemsize == 56
    assert int(lay["cfg"]) == C.sizeof(B.Config)
    assert int(lay["stats"]) == C.sizeof(B.Stats)
    assert int(lay["anchor"]) == B.ANCHOR_DTYPE.itemsize == S.ANCHOR_DTYPE.itemsize == C.sizeof(O.Anchor) == 12
    assert int(lay["chunk"]) == B.CHUNK_DTYPE.itemsize == 32
    assert int(lay["sstats"]) == C.sizeof(B.ServeStats)
    for k, v in lay.items():
        if "." not in k:
            continue
        T, f = k.split(".")
        if T == "rawalign_anchor_t":
            assert S.ANCHOR_DTYPE.fields[f][1] == int(v) == getattr(O.Anchor, f).offset, k
            continue
        if T == "rawalign_chunk_t":
            assert B.CHUNK_DTYPE.fields[f][1] == int(v), k
            continue
        if T == "rawalign_dtw_serve_stats_t":
            assert getattr(B.ServeStats, f).offset == int(v), k
            continue
        if T == "rawalign_dtw_stats_t":
            assert getattr(B.Stats, f).offset == int(v), k
            continue
        py = {"rawalign_candidate_t": B.Candidate, "rawalign_result_t": B.Result, "rawalign_dtw_config_t": B.Config}[T]
        assert getattr(py, f).offset == int(v), k
        if T == "rawalign_candidate_t":
            assert S.CANDIDATE_DTYPE.fields[f][1] == int(v), k
            assert getattr(O.Candidate, f).offset == int(v), k
        if T == "rawalign_result_t":
            assert getattr(O.Result, f).offset == int(v), k


def test_product_path_does_not_reach_the_oracle():
    """The package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2310_05037_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "rawalign_oracle" not in txt and "liboracle" not in txt, f
    out = subprocess.run(["ldd", B.LIB_PATH], capture_output=True, text=True).stdout if os.path.exists(B.LIB_PATH) else ""
    assert "oracle" not in out


def test_missing_library_fails_loudly(tmp_path):
    saved = B._lib
    try:
        B._lib = None
        with pytest.raises(RuntimeError):
            B.load(str(tmp_path / "nope.so"))
    finally:
        B._lib = saved


def test_poll_rejects_an_unusable_output_buffer():
    """rawalign_dtw_poll(out=...) and rawalign_dtw_poll_chunks(out=...) write
    into the caller's array only when it can hold cap records of the result
    layout; anything else is refused before the library is called."""
    with pytest.raises(TypeError):
        B.rawalign_dtw_poll(None, 1, 4, out=np.zeros(4, np.float64))
    with pytest.raises(TypeError):
        B.rawalign_dtw_poll(None, 1, 4, out=np.zeros(3, B.RESULT_DTYPE))
    with pytest.raises(TypeError):
        B.rawalign_dtw_poll(None, 1, 4, out=np.zeros(8, B.RESULT_DTYPE)[::2])
    tickets = np.arange(1, 3, dtype=np.uint64)
    with pytest.raises(TypeError):
        B.rawalign_dtw_poll_chunks(None, tickets, 4, out=np.zeros(4, np.float64))
    with pytest.raises(TypeError):
        B.rawalign_dtw_poll_chunks(None, tickets, 4, out=np.zeros(3, B.RESULT_DTYPE))
