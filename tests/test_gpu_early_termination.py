"""Early termination (branch and bound, Sec. 2.4.1) through the C ABI.

With config.early_termination the first candidate of each read is queued
first, and any candidate stops once its stripe-end lower bound cannot beat
the read's best score so far.  Checked against the oracle (which computes every
candidate in full): unstopped results are bit-exact, stopped ones carry a
cost bound <= the true cost and a score bound strictly below the read's best
score, and every read's best candidate and decision are unchanged."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import assert_bit_exact, run_gpu, run_gpu_anchored, run_oracle, run_oracle_anchored  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()
    assert torch.cuda.is_available()


def _workload(true_first, seed=0x5EED0002):
    return S.config_batched(seed=seed, n_reads=60, ref_len=2_000_000, median=500, lo=80, hi=1800,
                            true_first=true_first)


def _check(w, g, ora):
    pruned = g["status"] == B.RA_RESULT_PRUNED
    full = g["status"] == 0
    assert np.all(pruned | full)
    assert_bit_exact(g[full], ora[full])
    rid = w.cands["read_id"].astype(np.int64)
    best = np.full(w.n_reads, -np.inf, np.float32)
    np.maximum.at(best, rid, ora["score"].astype(np.float32))
    assert np.all(g["cost"][pruned] <= ora["cost"][pruned].astype(np.float32))
    assert np.all(g["score"][pruned] < best[rid[pruned]])
    assert np.all(g["end_i"][pruned] == -1) and np.all(g["end_j"][pruned] == -1)
    assert np.array_equal(g["is_best"], ora["is_best"]) and np.array_equal(g["decision"], ora["decision"])
    return int(pruned.sum())


@pytest.mark.parametrize("kernel", [B.RA_KERNEL_AUTO, B.RA_KERNEL_STRIPE[(4, 8)], B.RA_KERNEL_STRIPE[(16, 16)],
                                    B.RA_KERNEL_STRIPE[(8, 24)]])
@pytest.mark.parametrize("true_first", [True, False])
def test_pruned_and_kept_results(kernel, true_first):
    w = _workload(true_first)
    ora = run_oracle(w)
    n_pruned = 0
    for rep in range(2):
        n_pruned += _check(w, run_gpu(w, kernel=kernel, early_termination=True), ora)
    if true_first and kernel == B.RA_KERNEL_STRIPE[(4, 8)]:
        assert n_pruned > 0


def test_graph_replays_keep_best_and_decision():
    w = _workload(True)
    ora = run_oracle(w)
    for g in run_gpu(w, graph_runs=3, early_termination=True):
        _check(w, g, ora)


def test_free_end_and_anchored_batches_run_in_full():
    w = _workload(True)
    g = run_gpu(w, end_mode=B.RA_END_FREE, early_termination=True)
    assert_bit_exact(g, run_oracle(w, end_mode=B.RA_END_FREE))
    a = S.scaled("anchored", "small")
    assert_bit_exact(run_gpu_anchored(a, early_termination=True), run_oracle_anchored(a))
