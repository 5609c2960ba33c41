"""The autotuner's tuning file (CPU) and a short tuning run (GPU).

The file holds "G HR cost" lines (relative cost of one lane-cell slot per
striped variant) and the planner's bin edges ("ring_bins S": ring sizes
binned by powers of 2^S; "latency_split X").  The library reads it at
create time; results never depend on it (only the launch plan does), which
the GPU test checks bit for bit."""
import numpy as np
import pytest

from paper_2310_05037_gb300 import autotune as T
from paper_2310_05037_gb300 import binding as B


def test_table_round_trip(tmp_path):
    costs = {(32, 24): 1.0, (16, 24): 1.013, (4, 8): 2.124}
    plan = {"ring_bins": 1, "latency_split": 0.75}
    p = tmp_path / "tune.txt"
    T.write_table(str(p), costs, plan)
    c2, p2 = T.read_table(str(p))
    assert c2 == pytest.approx(costs) and p2 == pytest.approx(plan)
    T.write_table(str(p), costs)
    c3, p3 = T.read_table(str(p))
    assert c3 == pytest.approx(costs) and p3 == {}


def test_calibration_batch_shape():
    for G, HR in B.VARIANTS:
        pore, ref, ref_len, ev, offs, cands = T.calibration_batch(G, HR, 8, seed=1)
        n = 4 * G * HR
        assert len(ev) == 8 * n and offs[-1] == len(ev) and len(cands) == 8
        assert np.all(cands["ref_len_bases"] - 5 == n)
        # the band is just wide enough for the variant's period: 2w >= H - HR + 1 + G + 4
        assert np.all(2 * cands["band_w"] >= G * HR - HR + 1 + G + 4)
        assert np.all(cands["ref_offset"] + cands["ref_len_bases"] <= ref_len)


@pytest.mark.gpu
def test_tuning_runs_and_never_changes_results(tmp_path):
    torch = pytest.importorskip("torch")
    from paper_2310_05037_gb300 import build
    from paper_2310_05037_gb300 import synth as S

    build.build()
    assert torch.cuda.is_available()
    costs = T.tune(variants=[(16, 24), (4, 8)], runs=1, groups_factor=1)
    assert set(costs) == {(16, 24), (4, 8)} and min(costs.values()) == pytest.approx(1.0)
    assert all(c >= 1.0 for c in costs.values())
    w = S.scaled("batched", "small")
    plan, times = T.tune_plan(w, costs, runs=1, ring_bins=(2, 1), latency_splits=(0.0, 1.0))
    assert set(times) == {(2, 0.0), (2, 1.0), (1, 0.0), (1, 1.0)} and plan["ring_bins"] in (1, 2)
    path = tmp_path / "tune.txt"
    T.write_table(str(path), costs, {"ring_bins": 1, "latency_split": 0.25})
    outs = []
    for tune_path in (None, str(path)):
        al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=256 << 20, autotune_path=tune_path)
        try:
            outs.append(al.align(w.events, w.read_offsets, w.cands))
        finally:
            al.close()
    for f in outs[0].dtype.names:
        if f != "pad":
            assert np.array_equal(outs[0][f], outs[1][f]), f
    bad = tmp_path / "bad.txt"
    bad.write_text("ring_bins 3\n")
    with pytest.raises(B.RawAlignError):
        B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=256 << 20, autotune_path=str(bad))
