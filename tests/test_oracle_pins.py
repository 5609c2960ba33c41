"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(not by retyping the oracle's own formulas):

* hand-worked DTW tables (tests/golden/hand_worked.txt)            Sec. 2.2
* brute-force minimum over warping paths, bit-exact in FP32/FP64    Sec. 2.2
* closed forms for a single row / column                            Sec. 2.2
* invariants: identical signals cost 0, widening the band never
  raises a cell, band >= table equals no band, transpose symmetry,
  power-of-two scaling, FP32 within the rounding bound of FP64      Sec. 2.2-2.4.3
* k-mer indexing and reverse complement worked by hand             Sup. A.1.1
* score and threshold decision                                     Sec. 2.3, 3.1
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2310_05037_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _hand_cases():
    for line in open(os.path.join(GOLD, "hand_worked.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = [x.strip() for x in line.split("|")]
        yield (f[0], [float(x) for x in f[1].split()], [float(x) for x in f[2].split()], int(f[3]),
               O.END_GLOBAL if f[4] == "global" else O.END_FREE, float(f[5]), int(f[6]), int(f[7]))


@pytest.mark.parametrize("case", list(_hand_cases()), ids=lambda c: c[0])
def test_hand_worked(case):
    name, e, r, w, mode, cost, ei, ej = case
    c, gi, gj, _, _ = O.dtw_f32(e, r, w, end_mode=mode)
    assert float(c) == cost and (gi, gj) == (ei, ej)
    c64, gi, gj, _, _ = O.dtw_f64(e, r, w, end_mode=mode)
    assert c64 == cost and (gi, gj) == (ei, ej)


def test_hand_worked_score():
    # Score = B_Match * N_Read - C_DTW with B_Match = 0.4 (Sec. 3.1), case a:
    # fl32(0.4) = 0.4000000059604645; * 3 = 1.2000000178813934 rounds to the
    # float 1.2000000476837158203125; minus C = 1 is exact.
    assert float(O.score_f32(0.4, 3, 1.0)) == 0.2000000476837158203125
    # the FP64 run: 0.4 * 3 - 1 = 0.20000000000000007 in binary64
    assert O.score_f64(0.4, 3, 1.0) == 0.4 * 3 - 1.0


def _tiny_cases(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(1, 8))
        m = int(rng.integers(1, 8))
        kind = rng.integers(0, 3)
        if kind == 0:
            e = rng.normal(size=n).astype(np.float32)
            r = rng.normal(size=m).astype(np.float32)
        elif kind == 1:  # small integers: many exact ties
            e = rng.integers(-3, 4, size=n).astype(np.float32)
            r = rng.integers(-3, 4, size=m).astype(np.float32)
        else:  # wide dynamic range: rounding matters
            e = (rng.normal(size=n) * 10.0 ** rng.integers(-3, 4, size=n)).astype(np.float32)
            r = (rng.normal(size=m) * 10.0 ** rng.integers(-3, 4, size=m)).astype(np.float32)
        w = int(rng.integers(-1, 4))
        if rng.random() < 0.3:
            num, den = int(rng.integers(0, 4)), int(rng.integers(1, 4))
        else:
            num, den = 0, 0
        mode = int(rng.integers(0, 2))
        yield e, r, w, num, den, mode


def test_brute_force_fp32_bit_exact():
    """DP == min over all warping paths (FP32, accumulation from the start)."""
    count = 0
    for e, r, w, num, den, mode in _tiny_cases(1, 3000):
        c, ei, ej, cells, _ = O.dtw_f32(e, r, w, num, den, mode)
        bc, bj, paths = O.brute_f32(e, r, w, num, den, mode)
        if paths == 0:  # no in-band path to the end cell (possible with a given slope)
            assert math.isinf(c)
            continue
        assert np.float32(c).tobytes() == np.float32(bc).tobytes(), (e, r, w, num, den, mode)
        if mode == O.END_FREE:
            assert ej == bj
        count += 1
    assert count > 2000


def test_brute_force_fp64_bit_exact():
    for e, r, w, num, den, mode in _tiny_cases(2, 1500):
        c, ei, ej, cells, _ = O.dtw_f64(e, r, w, num, den, mode)
        bc, bj, paths = O.brute_f64(e, r, w, num, den, mode)
        if paths == 0:
            assert math.isinf(c)
            continue
        assert c == bc
        if mode == O.END_FREE:
            assert ej == bj


def test_path_counts_are_delannoy():
    # unbanded paths from (0,0) to (a,b) by E, S, SE steps: Delannoy numbers
    # D(a,b) = sum_k C(a,k) C(b,k) 2^k, e.g. D(2,6) = 1 + 2*6*2 + 15*4 = 85
    delannoy = {(2, 2): 13, (3, 3): 63, (6, 6): 8989, (2, 6): 85}
    for (a, b), want in delannoy.items():
        _, _, paths = O.brute_f32(np.zeros(a + 1), np.zeros(b + 1))
        assert paths == want


def test_single_row_and_column_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(200):
        m = int(rng.integers(1, 300))
        e0 = np.float32(rng.normal())
        r = rng.normal(size=m).astype(np.float32)
        acc = np.float32(0)
        for x in r:  # sequential FP32 accumulation of |e0 - r_j|
            acc = np.float32(np.float32(abs(np.float32(e0 - x))) + acc)
        c, ei, ej, cells, _ = O.dtw_f32([e0], r)
        assert c == acc and (ei, ej) == (0, m - 1) and cells == m
        c, _, _, _, _ = O.dtw_f32(r, [e0])  # single column, same sum
        assert c == acc


def test_identical_sequences_cost_zero():
    rng = np.random.default_rng(4)
    for _ in range(50):
        n = int(rng.integers(1, 400))
        x = rng.normal(size=n).astype(np.float32)
        assert O.dtw_f32(x, x)[0] == 0
        assert O.dtw_f32(x, x, band_w=0)[0] == 0  # the diagonal is always in the band
        rep = np.repeat(x, rng.integers(1, 4, size=n))  # stretched copy: warping absorbs it
        assert O.dtw_f32(rep, x)[0] == 0


def test_band_widening_is_monotone_cellwise():
    rng = np.random.default_rng(5)
    for _ in range(40):
        n, m = int(rng.integers(2, 120)), int(rng.integers(2, 120))
        e = rng.normal(size=n).astype(np.float32)
        r = rng.normal(size=m).astype(np.float32)
        prev = None
        for w in range(0, max(n, m) + 2, 3):
            c, _, _, cells, _, D = O.dtw_f32(e, r, w, full=True)
            if prev is not None:
                assert np.all(D <= prev[0]) and c <= prev[1] and cells >= prev[2]
            prev = (D, c, cells)
        cu, _, _, cellsu, _ = O.dtw_f32(e, r, -1)
        cw, _, _, cellsw, _ = O.dtw_f32(e, r, n + m)
        assert cu == cw and cellsu == cellsw == n * m


def test_transpose_symmetry_unbanded():
    rng = np.random.default_rng(6)
    for _ in range(50):
        e = rng.normal(size=int(rng.integers(1, 150))).astype(np.float32)
        r = rng.normal(size=int(rng.integers(1, 150))).astype(np.float32)
        assert O.dtw_f32(e, r)[0] == O.dtw_f32(r, e)[0]


def test_power_of_two_scaling_exact():
    rng = np.random.default_rng(7)
    for _ in range(40):
        e = rng.normal(size=int(rng.integers(1, 200))).astype(np.float32)
        r = rng.normal(size=int(rng.integers(1, 200))).astype(np.float32)
        for p in (-3, 1, 5):
            s = np.float32(2.0 ** p)
            assert O.dtw_f32(e * s, r * s, 7)[0] == O.dtw_f32(e, r, 7)[0] * s


def test_fp32_within_rounding_bound_of_fp64():
    """|C32 - C64| <= (path length) * u * C64 (u = 2^-24): each of the at most
    n+m-1 adds on the optimal path is rounded once."""
    rng = np.random.default_rng(8)
    for _ in range(30):
        n, m = int(rng.integers(50, 400)), int(rng.integers(50, 400))
        e = rng.normal(size=n).astype(np.float32)
        r = rng.normal(size=m).astype(np.float32)
        c32 = float(O.dtw_f32(e, r, 40)[0])
        c64 = O.dtw_f64(e, r, 40)[0]
        assert abs(c32 - c64) <= (n + m) * 2.0 ** -24 * c64 + 1e-30
        assert abs(c32 - c64) / c64 < 1e-5


def _closed_form_band(n, m, w, num, den):
    """Band rows from the inequality |j den - i num| <= w den solved for j."""
    tot = 0
    for i in range(n):
        lo = max(0, -((w * den - i * num) // den))  # ceil((i num - w den)/den)
        hi = min(m - 1, (i * num + w * den) // den)
        tot += max(0, hi - lo + 1)
    return tot


def test_band_predicate_matches_solved_rows_and_connects():
    rng = np.random.default_rng(9)
    for _ in range(300):
        n, m = int(rng.integers(2, 200)), int(rng.integers(2, 200))
        w = int(rng.integers(0, 50))
        b = O.band_params(n, m, w)
        assert b.num == m - 1 and b.den == n - 1
        assert b.w_eff == max(w, -(-(m - 1) // (2 * (n - 1))), 1)
        assert O.band_cells(b, n, m) == _closed_form_band(n, m, b.w_eff, b.num, b.den)
        # a monotone path always exists with the derived slope: finite cost
        e = rng.normal(size=n).astype(np.float32)
        r = rng.normal(size=m).astype(np.float32)
        assert np.isfinite(O.dtw_f32(e, r, w)[0])


def test_kmer_index_and_reverse_complement():
    code = {c: i for i, c in enumerate("ACGT")}
    enc = lambda s: np.array([code[c] for c in s], np.uint8)
    assert O.kmer_index(enc("AAAAAA"), 6) == 0
    assert O.kmer_index(enc("TTTTTT"), 6) == 4095
    assert O.kmer_index(enc("CAAAAA"), 6) == 1024  # first base is most significant
    assert O.kmer_index(enc("AAAAAC"), 6) == 1
    assert O.kmer_index(enc("ACGTAC"), 6) == 256 + 2 * 64 + 3 * 16 + 1  # 433
    pore = np.arange(4096, dtype=np.float32)
    assert list(O.expected_signal(enc("ACGTACG"), 6, pore)) == [433.0, 4 * 433 % 4096 + 2]
    # reference packed LSB-first, 4 bases per byte: "ACGTTGCA"
    seq = "ACGTTGCA"
    packed = S.pack_bases(enc(seq))
    assert list(packed) == [0 | 1 << 2 | 2 << 4 | 3 << 6, 3 | 2 << 2 | 1 << 4 | 0 << 6]
    fwd = O.segment_codes(packed, 8, 1, 5, 0)
    assert "".join("ACGT"[c] for c in fwd) == "CGTTG"
    rev = O.segment_codes(packed, 8, 1, 5, 1)  # reverse complement of CGTTG
    assert "".join("ACGT"[c] for c in rev) == "CAACG"


def _batch(cands_rows, events_list, ref_seq):
    code = {c: i for i, c in enumerate("ACGT")}
    ref = S.pack_bases(np.array([code[c] for c in ref_seq], np.uint8))
    offs = np.zeros(len(events_list) + 1, np.uint64)
    offs[1:] = np.cumsum([len(x) for x in events_list])
    ev = np.concatenate(events_list).astype(np.float32)
    c = np.zeros(len(cands_rows), S.CANDIDATE_DTYPE)
    for i, row in enumerate(cands_rows):
        c[i]["read_id"], c[i]["ref_offset"], c[i]["ref_len_bases"] = row[0], row[1], row[2]
        c[i]["band_w"] = row[3] if len(row) > 3 else -1
    return ref, len(ref_seq), ev, offs, c


def test_map_batch_decision_threshold_and_ties():
    # k = 1, pore = [0,1,2,3]: the expected signal is the base code itself.
    pore = np.array([0, 1, 2, 3], np.float32)
    ref_seq = "ACGTACGTAAAA"
    read = np.array([0, 1, 2, 3], np.float32)  # matches ACGT exactly: cost 0
    ref, rl, ev, offs, c = _batch([(0, 0, 4), (0, 4, 4), (0, 8, 4)], [read], ref_seq)
    # B = 5, N = 4: score = 20 - C.  Candidates 0 and 1 tie at 20 -> smallest index wins.
    out = O.map_batch(1, 5.0, 20.0, O.END_GLOBAL, pore, ref, rl, ev, offs, c)
    assert list(out["score"]) == [20.0, 20.0, 20.0 - 6.0]
    assert list(out["is_best"]) == [1, 0, 0]
    assert set(out["decision"]) == {O.MAPPED}  # 20 >= 20: mapped at equality
    out = O.map_batch(1, 5.0, 20.5, O.END_GLOBAL, pore, ref, rl, ev, offs, c)
    assert set(out["decision"]) == {O.UNMAPPED}


def test_map_batch_rejects_bad_inputs():
    pore = np.array([0, 1, 2, 3], np.float32)
    ref, rl, ev, offs, c = _batch([(0, 0, 4)], [np.array([0, 1, 2, 3], np.float32)], "ACGTACGT")
    O.map_batch(1, 0.4, 20, 0, pore, ref, rl, ev, offs, c)
    bad = ev.copy()
    bad[1] = np.nan
    with pytest.raises(ValueError):
        O.map_batch(1, 0.4, 20, 0, pore, ref, rl, bad, offs, c)
    c2 = c.copy()
    c2["ref_offset"] = 6  # runs off the 8-base reference
    with pytest.raises(ValueError):
        O.map_batch(1, 0.4, 20, 0, pore, ref, rl, ev, offs, c2)
    c3 = c.copy()
    c3["read_id"] = 1
    with pytest.raises(ValueError):
        O.map_batch(1, 0.4, 20, 0, pore, ref, rl, ev, offs, c3)


def test_planted_mistakes_are_caught():
    """Sanity of the pins: a DP missing the NW term, or taking max for min,
    disagrees with the brute force on the tiny cases."""
    def dtw_no_nw(e, r):
        n, m = len(e), len(r)
        D = np.full((n, m), np.inf, np.float32)
        for i in range(n):
            for j in range(m):
                d = np.float32(abs(np.float32(e[i] - r[j])))
                if i == 0 and j == 0:
                    p = np.float32(0)
                else:
                    p = min(D[i - 1, j] if i else np.inf, D[i, j - 1] if j else np.inf)
                D[i, j] = np.float32(d + np.float32(p))
        return D[-1, -1]

    diffs = 0
    for e, r, w, num, den, mode in _tiny_cases(11, 300):
        if len(e) < 2 or len(r) < 2:
            continue
        if dtw_no_nw(e, r) != O.brute_f32(e, r)[0]:
            diffs += 1
    assert diffs > 50


# ---------------------------------------------------------------- anchor-guided alignment (Sec. 2.4.2)
def _load_anchored():
    rows = []
    for line in open(os.path.join(GOLD, "anchored_hand_worked.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, ev, rv, an, bw, cost, cells = [x.strip() for x in line.split("|")]
        anchors = [tuple(int(v) for v in a.split(",")) for a in an.split(";") if a]
        rows.append((name, [float(x) for x in ev.split()], [float(x) for x in rv.split()], anchors, int(bw),
                     float(cost), int(cells)))
    return rows


@pytest.mark.parametrize("case", _load_anchored(), ids=lambda c: c[0])
def test_anchored_hand_worked(case):
    name, e, r, anchors, bw, cost, cells = case
    c32, n32 = O.anchored_f32(e, r, anchors, bw)
    c64, n64 = O.anchored_f64(e, r, anchors, bw)
    assert float(c32) == cost and c64 == cost
    assert n32 == cells == n64
    assert O.anchored_brute(e, r, anchors) == cost


def _random_anchors(rng, n, m, max_k=3):
    """Sorted, disjoint anchors inside an n x m table (may be empty)."""
    anchors = []
    q, t = 0, 0
    for _ in range(int(rng.integers(0, max_k + 1))):
        if q >= n or t >= m:
            break
        q0 = int(rng.integers(q, n))
        t0 = int(rng.integers(t, m))
        ln = int(rng.integers(1, min(n - q0, m - t0) + 1))
        anchors.append((q0, t0, ln))
        q, t = q0 + ln, t0 + ln
    return anchors


def test_anchored_equals_brute_force_on_integer_tables():
    """The piecewise evaluation equals the minimum over all paths that stay in
    the gap rectangles, one-sided gap lines and anchor diagonals (integer
    values: every sum is exact, so equality is bit for bit)."""
    rng = np.random.default_rng(2024)
    checked = 0
    for _ in range(2500):
        n, m = int(rng.integers(1, 8)), int(rng.integers(1, 8))
        e = rng.integers(-4, 5, size=n).astype(np.float64)
        r = rng.integers(-4, 5, size=m).astype(np.float64)
        anchors = _random_anchors(rng, n, m)
        bf = O.anchored_brute(e, r, anchors)
        c64, _ = O.anchored_f64(e, r, anchors)
        c32, _ = O.anchored_f32(e, r, anchors)
        assert c64 == bf and float(c32) == bf, (e, r, anchors, bf, c64, c32)
        checked += len(anchors) > 0
    assert checked > 1500


def test_anchored_without_anchors_is_plain_dtw_and_never_below_it():
    rng = np.random.default_rng(7)
    for _ in range(400):
        n, m = int(rng.integers(1, 12)), int(rng.integers(1, 12))
        e = rng.integers(-5, 6, size=n).astype(np.float32)
        r = rng.integers(-5, 6, size=m).astype(np.float32)
        bw = int(rng.integers(-1, 4))
        plain = O.dtw_f32(e, r, bw)[0]
        assert O.anchored_f32(e, r, [], bw)[0] == plain
        # with anchors (unbanded), the cost can only grow: fewer paths
        anchors = _random_anchors(rng, n, m)
        assert O.anchored_f32(e, r, anchors)[0] >= O.dtw_f32(e, r)[0]


def test_anchored_full_diagonal_closed_form():
    """One anchor over the whole diagonal of an n x n table: the cost is the
    sequential FP32 sum of |e_i - r_i|."""
    rng = np.random.default_rng(9)
    for n in (1, 2, 5, 33, 200):
        e = rng.standard_normal(n).astype(np.float32)
        r = rng.standard_normal(n).astype(np.float32)
        s = np.float32(0)
        for i in range(n):
            d = np.float32(abs(np.float32(e[i] - r[i])))
            s = d if i == 0 else np.float32(s + d)
        c, cells = O.anchored_f32(e, r, [(0, 0, n)])
        assert c == s and cells == n


def test_anchored_rejects_bad_chains():
    e = np.zeros(6, np.float32)
    r = np.zeros(6, np.float32)
    for bad in ([(0, 0, 0)], [(2, 2, 2), (3, 5, 1)], [(2, 2, 2), (5, 3, 1)], [(4, 4, 3)], [(0, 5, 2)]):
        with pytest.raises(ValueError):
            O.anchored_f32(e, r, bad)


def test_planted_anchor_mistake_is_caught():
    """A variant that aligns a one-sided gap to the next anchor's first value
    instead of the previous anchor's last one disagrees with the brute force."""
    def wrong(e, r, anchors):
        C, pq, pt, first = 0.0, 0, 0, True
        n, m = len(e), len(r)
        for a in range(len(anchors) + 1):
            q1, t1 = (anchors[a][0], anchors[a][1]) if a < len(anchors) else (n, m)
            nr, nc = q1 - pq, t1 - pt
            piece = None
            if nr > 0 and nc > 0:
                piece = O.dtw_f64(e[pq:q1], r[pt:t1])[0]
            elif nr > 0:
                col = min(t1, m - 1)  # the planted mistake
                piece = sum(abs(e[i] - r[col]) for i in range(pq, q1))
            elif nc > 0:
                row = pq - 1 if a > 0 else q1
                piece = sum(abs(e[row] - r[j]) for j in range(pt, t1))
            if piece is not None:
                C = piece if first else C + piece
                first = False
            if a < len(anchors):
                q, t, ln = anchors[a]
                s = sum(abs(e[q + x] - r[t + x]) for x in range(ln))
                C = s if first else C + s
                first = False
                pq, pt = q + ln, t + ln
        return C

    rng = np.random.default_rng(5)
    diffs = 0
    for _ in range(1500):
        n, m = int(rng.integers(2, 8)), int(rng.integers(2, 8))
        e = rng.integers(-4, 5, size=n).astype(np.float64)
        r = rng.integers(-4, 5, size=m).astype(np.float64)
        anchors = _random_anchors(rng, n, m)
        if wrong(e, r, anchors) != O.anchored_brute(e, r, anchors):
            diffs += 1
    assert diffs > 20


# ---------------------------------------------------------------- traceback (optional path output)
def _load_traceback():
    rows = []
    for line in open(os.path.join(GOLD, "traceback_hand_worked.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, ev, rv, bw, mode, cost, path = [x.strip() for x in line.split("|")]
        p = [tuple(int(v) for v in c.split(",")) for c in path.split()]
        rows.append((name, [float(x) for x in ev.split()], [float(x) for x in rv.split()], int(bw),
                     O.END_GLOBAL if mode == "global" else O.END_FREE, float(cost), p))
    return rows


@pytest.mark.parametrize("case", _load_traceback(), ids=lambda c: c[0])
def test_traceback_hand_worked(case):
    name, e, r, bw, mode, cost, path = case
    c, p = O.traceback_f32(e, r, bw, end_mode=mode)
    assert float(c) == cost
    assert [tuple(x) for x in p.tolist()] == path


def _all_optimal_paths(e, r, band, end_mode):
    """Every path from (0,0) (N/W/NW steps, in band) ending in the last row
    (FREE) or at the corner (GLOBAL), with its FP64 cost; the optimal ones."""
    n, m = len(e), len(r)
    out = []

    def walk(i, j, acc, path):
        if i == n - 1 and (end_mode == O.END_FREE or j == m - 1):
            out.append((acc, list(path)))
        for di, dj in ((0, 1), (1, 0), (1, 1)):
            a, b = i + di, j + dj
            if a < n and b < m and O.in_band(band, a, b):
                path.append((a, b))
                walk(a, b, acc + abs(float(e[a]) - float(r[b])), path)
                path.pop()

    if O.in_band(band, 0, 0):
        walk(0, 0, abs(float(e[0]) - float(r[0])), [(0, 0)])
    if not out:
        return np.inf, []
    best = min(a for a, _ in out)
    return best, [p for a, p in out if a == best]


def test_traceback_is_an_optimal_path_and_resums_to_the_cost():
    """On small integer tables (exact sums) the returned path is one of the
    optimal warping paths found by enumeration; on random FP32 tables the
    path's cells, summed in path order in FP32, give the cost bit for bit."""
    rng = np.random.default_rng(33)
    for it in range(600):
        n, m = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        if it % 2:
            e = rng.integers(-3, 4, size=n).astype(np.float32)
            r = rng.integers(-3, 4, size=m).astype(np.float32)
        else:
            e = rng.standard_normal(n).astype(np.float32)
            r = rng.standard_normal(m).astype(np.float32)
        bw = int(rng.integers(-1, 3))
        mode = int(rng.integers(0, 2))
        cost, path = O.traceback_f32(e, r, bw, end_mode=mode)
        band = O.band_params(n, m, bw)
        if not np.isfinite(cost):
            assert len(path) == 0
            continue
        assert tuple(path[0]) == (0, 0) and path[-1][0] == n - 1
        if mode == O.END_GLOBAL:
            assert path[-1][1] == m - 1
        steps = np.diff(path, axis=0)
        assert all(tuple(s) in ((0, 1), (1, 0), (1, 1)) for s in steps)
        assert all(O.in_band(band, int(i), int(j)) for i, j in path)
        s = np.float32(0)
        for k, (i, j) in enumerate(path):
            d = np.float32(abs(np.float32(e[i] - r[j])))
            s = d if k == 0 else np.float32(d + s)
        assert s == cost
        if it % 2:
            best, opt = _all_optimal_paths(e, r, band, mode)
            assert float(cost) == best
            assert [tuple(x) for x in path.tolist()] in [[tuple(c) for c in p] for p in opt]
