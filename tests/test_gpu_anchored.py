"""Anchor-guided alignment (Sec. 2.4.2) on the GPU through the C ABI
(rawalign_dtw_prepare_anchored / submit_anchored), bit-exact against the
oracle's piecewise evaluation: gaps aligned by their own banded DTW in the
striped kernels, anchors and one-sided gaps summed along their cells, the
pieces added in path order, then score and per-read decision."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_05037_gb300 import binding as B  # noqa: E402
from paper_2310_05037_gb300 import synth as S  # noqa: E402

from gpu_util import (assert_bit_exact, run_gpu, run_gpu_anchored, run_oracle,  # noqa: E402
                      run_oracle_anchored, tiny_anchored_workload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2310_05037_gb300 import build

    build.build()
    assert torch.cuda.is_available()


KERNELS = [B.RA_KERNEL_AUTO, B.RA_KERNEL_PLAIN, B.RA_KERNEL_STRIPE[(16, 24)], B.RA_KERNEL_STRIPE[(4, 8)],
           B.RA_KERNEL_STRIPE[(32, 16)]]


@pytest.mark.parametrize("kernel", KERNELS)
def test_tiny_chains(kernel):
    w = tiny_anchored_workload(31 + kernel, n_cands=1500)
    assert_bit_exact(run_gpu_anchored(w, kernel=kernel), run_oracle_anchored(w))


@pytest.mark.parametrize("kernel", [B.RA_KERNEL_AUTO, B.RA_KERNEL_PLAIN])
def test_anchored_workload_small(kernel):
    w = S.scaled("anchored", "small")
    assert_bit_exact(run_gpu_anchored(w, kernel=kernel), run_oracle_anchored(w))


def test_graph_replays_match():
    w = S.scaled("anchored", "small")
    ora = run_oracle_anchored(w)
    for out in run_gpu_anchored(w, graph_runs=3):
        assert_bit_exact(out, ora)


def test_empty_chains_equal_plain_batch():
    """With no anchors the only piece is the whole table, aligned with the
    band around its own diagonal: the plain batch's cost, score and end."""
    w = S.scaled("batched", "small")
    w.anchors = np.zeros(0, S.ANCHOR_DTYPE)
    w.anchor_offsets = np.zeros(w.n_cands + 1, np.uint64)
    a = run_gpu_anchored(w)
    p = run_gpu(w)
    for f in ("cost", "score", "end_i", "end_j", "cells", "is_best", "decision"):
        assert np.array_equal(a[f], p[f]), f


def test_fp64_agreement():
    w = S.scaled("anchored", "small")
    g = run_gpu_anchored(w)
    c64 = run_oracle_anchored(w, use_f64=True)["cost64"]
    assert (np.abs(g["cost"].astype(np.float64) - c64) / np.maximum(c64, 1e-30)).max() < 1e-5


def test_bad_chains_rejected():
    w = S.scaled("anchored", "small").subset(np.arange(6))
    for bad in ([(0, 0, 0)], [(5, 5, 4), (6, 20, 2)], [(0, 10 ** 6, 1)], [(10 ** 6, 0, 1)]):
        x = S.Workload(**{**w.__dict__})
        x.anchors = np.array(bad, dtype=S.ANCHOR_DTYPE)
        x.anchor_offsets = np.array([0] * 3 + [len(bad)] * (w.n_cands - 2), np.uint64)
        with pytest.raises(B.RawAlignError) as ei:
            run_gpu_anchored(x)
        assert ei.value.code == B.RA_EINVAL
