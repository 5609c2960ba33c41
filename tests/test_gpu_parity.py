"""GPU parity: the CUDA path through the C ABI against the oracle, bit-exact
on every cost, score, end cell, cell count and decision (FP32, Sec. 2.2-2.4.3
and 2.3), on tiny brute-force-sized cases, tiling edges, oracle-sized versions
of the benchmark workloads, every kernel variant and the plain kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import arena_bytes_for, assert_bit_exact, edge_workload, run_gpu, run_oracle, tiny_workload  # noqa: E402

pytestmark = pytest.mark.gpu

VARIANTS = [B.RA_KERNEL_AUTO] + [B.RA_KERNEL_STRIPE[gh] for gh in B.VARIANTS]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("kernel", VARIANTS + [B.RA_KERNEL_PLAIN])
@pytest.mark.parametrize("end_mode", [B.RA_END_GLOBAL, B.RA_END_FREE])
def test_tiny_cases(kernel, end_mode):
    w = tiny_workload(11 + kernel, n_cands=1500)
    assert_bit_exact(run_gpu(w, kernel=kernel, end_mode=end_mode), run_oracle(w, end_mode=end_mode))


@pytest.mark.parametrize("kernel", VARIANTS + [B.RA_KERNEL_PLAIN])
@pytest.mark.parametrize("end_mode", [B.RA_END_GLOBAL, B.RA_END_FREE])
def test_tiling_edges(kernel, end_mode):
    w = edge_workload()
    assert_bit_exact(run_gpu(w, kernel=kernel, end_mode=end_mode), run_oracle(w, end_mode=end_mode))


def test_exact_signal_costs_zero():
    w = edge_workload()
    g = run_gpu(w)
    # the last two alignments use events equal to the expected signal
    assert g["cost"][-1] == 0 and g["cost"][-2] == 0


@pytest.mark.parametrize("name", ["plain", "batched", "readuntil", "longread"])
@pytest.mark.parametrize("kernel", VARIANTS)
def test_workloads_small(name, kernel):
    w = S.scaled(name, "full" if name == "plain" else "small")
    assert_bit_exact(run_gpu(w, kernel=kernel), run_oracle(w))


def test_plain_kernel_on_plain_config():
    w = S.scaled("plain", "full").subset(np.arange(16))
    assert_bit_exact(run_gpu(w, kernel=B.RA_KERNEL_PLAIN), run_oracle(w))


def test_graph_replays_match_and_repeat():
    w = S.scaled("batched", "small")
    outs = run_gpu(w, graph_runs=3)
    ora = run_oracle(w)
    for o in outs:
        assert_bit_exact(o, ora)


def test_batch_stats():
    """Counters of a run: the batch's cells are the results' cells, the plan's
    lane-cell slots cover them, and the timed parts are positive."""
    w = S.scaled("batched", "small")
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes_for(w), k=w.k, b_match=w.b_match,
                   score_threshold=w.score_threshold, end_mode=w.end_mode)
    try:
        b = al.prepare(w.events, w.read_offsets, w.cands)
        r = al.poll(al.run(b), w.n_cands)
        st = al.stats(b)
        assert st.cells == int(r["cells"].sum())
        assert st.slots >= st.cells > 0
        assert st.launches >= 3
        assert 0 < st.dtw_ms <= st.total_ms
        al.release(b)
    finally:
        al.close()


def test_fp64_agreement():
    """FP32 cost within 1e-5 relative of the FP64 run (and within the
    (n+m) * 2^-24 rounding bound)."""
    w = S.scaled("batched", "small")
    g = run_gpu(w)
    o64 = run_oracle(w, use_f64=True)
    c64 = o64["cost64"]
    rel = np.abs(g["cost"].astype(np.float64) - c64) / np.maximum(c64, 1e-30)
    assert rel.max() < 1e-5


def test_band_widening_never_raises_cost():
    base = S.scaled("batched", "small").subset(np.arange(40))
    costs = []
    for wv in (2, 8, 32, 128, 100000):
        w = S.Workload(**{**base.__dict__, "cands": base.cands.copy()})
        w.cands["band_w"] = wv
        costs.append(run_gpu(w)["cost"])
    for a, b in zip(costs, costs[1:]):
        assert np.all(b <= a)


def test_nonfinite_event_rejected_at_poll():
    w = S.scaled("batched", "small").subset(np.arange(10))
    w.events = w.events.copy()
    w.events[5] = np.nan
    with pytest.raises(B.RawAlignError) as ei:
        run_gpu(w)
    assert ei.value.code == B.RA_EINVAL


def test_bad_candidates_rejected_at_submit():
    w = S.scaled("batched", "small").subset(np.arange(10))
    for field, val in [("ref_offset", w.ref_len), ("ref_len_bases", 3), ("read_id", 10 ** 6), ("strand", 2)]:
        bad = S.Workload(**{**w.__dict__, "cands": w.cands.copy()})
        bad.cands[field][3] = val
        with pytest.raises(B.RawAlignError) as ei:
            run_gpu(bad)
        assert ei.value.code == B.RA_EINVAL


def test_arena_too_small():
    w = S.scaled("batched", "small")
    with pytest.raises(B.RawAlignError) as ei:
        al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=1 << 20)
        try:
            al.align(w.events, w.read_offsets, w.cands)
        finally:
            al.close()
    assert ei.value.code == B.RA_ENOMEM


@pytest.mark.parametrize("k", [1, 2, 3, 5, 6, 7, 8])
def test_kmer_lengths_and_word_offsets(k):
    """Expected signal (Sup. A.1.1) for every supported k, both strands, with
    regions starting at every base offset within a packed 16-base word and
    ending at the reference's last base."""
    rng = np.random.default_rng(100 + k)
    pore = rng.standard_normal(4 ** k).astype(np.float32)
    ref_len = 4099
    ref = S.hashed_reference(k, ref_len)
    reads, rows = [], []
    for off in list(range(0, 40)) + [ref_len - 200, ref_len - 64 - k]:
        for strand in (0, 1):
            span = min(64 + k - 1 + off % 7, ref_len - off)
            n = int(rng.integers(20, 90))
            reads.append(rng.standard_normal(n).astype(np.float32))
            rows.append((len(reads) - 1, off, span, strand, int(rng.integers(-1, 12)), 0, 0))
    w = S._finish("kmers", pore, ref, ref_len, reads, rows, dict(k=k))
    w.k = k
    assert_bit_exact(run_gpu(w), run_oracle(w))
