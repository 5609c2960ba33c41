"""The block-split kernel: one long alignment on a block of four warps, each
warp computing every fourth stripe, the bottom row of a stripe handed to the
next warp through a ring in shared memory with bounded waits.

Results must equal the oracle's bit for bit, whether every alignment is
forced onto it (RA_KERNEL_SPLIT: tiny cases, tiling edges, the small
workloads, both end modes) or the planner sends it the alignments that would
outlast the rest of a batch (long reads).  With the hand-off stalled on
purpose (a test-only switch: no stripe publishes its bottom row), the waits
give up within their bound, the affected results carry RA_ETIMEDOUT, and
the handle keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import arena_bytes_for, assert_bit_exact, edge_workload, run_gpu, run_oracle, tiny_workload  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()


@pytest.mark.parametrize("end_mode", [O.END_GLOBAL, O.END_FREE])
def test_split_forced_tiny_and_edges(end_mode):
    for w in (tiny_workload(71, n_cands=1500), edge_workload(9)):
        assert_bit_exact(run_gpu(w, kernel=B.RA_KERNEL_SPLIT, end_mode=end_mode), run_oracle(w, end_mode=end_mode))


@pytest.mark.parametrize("name", ["batched", "readuntil", "longread", "plain"])
def test_split_forced_workloads(name):
    w = S.scaled(name, "small")
    for end_mode in (O.END_GLOBAL, O.END_FREE):
        assert_bit_exact(run_gpu(w, kernel=B.RA_KERNEL_SPLIT, end_mode=end_mode), run_oracle(w, end_mode=end_mode))


def test_planner_splits_long_reads():
    """A long-read batch with few alignments and the tuning file's
    block_split on: the planner gives the longest alignments to the split
    kernel (the batch counters say how many), and every result is the
    oracle's."""
    import os
    import tempfile

    from paper_2310_05037_gb300 import autotune as T

    w = S.config_longread(n_reads=12, ref_len=4_000_000, nmin=8000, nmax=16000)
    path = os.path.join(tempfile.mkdtemp(), "tune.txt")
    T.write_table(path, {}, {"block_split": 1.0})
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w) + (1 << 30), autotune_path=path)
    try:
        b = al.prepare(w.events, w.read_offsets, w.cands)
        got = al.poll(al.run(b), w.n_cands)
        n_split = al.stats(b).split
        al.release(b)
    finally:
        al.close()
    assert n_split > 0
    assert_bit_exact(got, run_oracle(w))


def test_stalled_handoff_times_out_and_handle_survives():
    w = S.config_longread(n_reads=3, ref_len=2_000_000, nmin=3000, nmax=4000)
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w) + (256 << 20),
                   kernel=B.RA_KERNEL_SPLIT, test_stall_handoff=True)
    try:
        got = al.align(w.events, w.read_offsets, w.cands)
    finally:
        al.close()
    # every alignment here spans several stripes: its second stripe waits for
    # a bottom row nobody publishes, gives up, and the alignment stops
    assert np.all(got["status"] == B.RA_ETIMEDOUT)
    assert np.all(np.isinf(got["cost"]))
    # a fresh handle on the same device runs normally afterwards
    assert_bit_exact(run_gpu(w, kernel=B.RA_KERNEL_SPLIT), run_oracle(w))
