"""The serving workload generator's near-duplicate reads (CPU only).

The Read-Until decision study (Sec. 3.1) is informative only when some reads
have a decoy candidate that is a near-copy of their true locus.  These tests
check that the generator really produces such reads, and that it refuses a
block size too short to hold one read's walk instead of silently producing
none."""
import numpy as np
import pytest

from paper_2310_05037_gb300 import synth as S


def _identity(ref, a, b, n):
    x = S.unpack_bases(ref, a, n)
    y = S.unpack_bases(ref, b, n)
    return float(np.mean(x == y))


def test_repeat_reads_have_a_near_copy_candidate():
    pore, ref, ref_len, reads = S.config_serving(seed=7, n_reads=64, ref_len=8_000_000, dup_frac=0.05,
                                                 block=20_000, ident=0.98, repeat_reads=1.0, off_target=0.0)
    assert all(r.on_target for r in reads)
    found = 0
    for r in reads:
        span = int(r.cands[0][2])
        true_off = int(r.cands[r.true_cand][1])
        best = max(_identity(ref, true_off, int(c[1]), span)
                   for i, c in enumerate(r.cands) if i != r.true_cand)
        # a copy at 98 % identity (mutations drawn per base), against about
        # 25 % for an unrelated locus
        assert best > 0.95, best
        found += 1
    assert found == len(reads)


def test_no_repeat_reads_by_default():
    pore, ref, ref_len, reads = S.config_serving(seed=7, n_reads=64, ref_len=8_000_000, off_target=0.0)
    for r in reads:
        span = int(r.cands[0][2])
        true_off = int(r.cands[r.true_cand][1])
        others = [_identity(ref, true_off, int(c[1]), span) for i, c in enumerate(r.cands) if i != r.true_cand]
        assert not others or max(others) < 0.5


def test_blocks_too_short_for_a_read_are_refused():
    with pytest.raises(ValueError):
        S.config_serving(seed=7, n_reads=8, ref_len=4_000_000, dup_frac=0.05, block=5000, repeat_reads=0.25)
