"""Seeded synthetic workloads for the RawAlign DTW path.

This module only *makes inputs*: a pore (k-mer) table, a reference genome
stored two bits per base, simulated nanopore event sequences and candidate
reference regions.  It holds none of the alignment arithmetic; the CUDA library
and the CPU oracle each compute expected signals, bands, DTW and scores on
their own from what this module returns.

Stand-in for the paper's ONT R9.4 datasets (Sec. 3.1, Tab. datasets): pore
means N(0,1) as if z-scored, about 1.1 events per k-mer, Gaussian event noise,
skipped k-mers, uniform-ACGT references.  The five workloads below follow the
five benchmark configurations (plain, batched uneven, Read-Until prefix,
serving loop, long reads); ``scale`` shrinks a workload for oracle-sized tests.

Reference layout: base p is in bits 2*(p%4)..2*(p%4)+1 of byte p//4
(A=0, C=1, G=2, T=3).  Large references are generated from a counter-based
hash (SplitMix64 of the 32-base word index), so a 3 Gb genome is one
vectorised pass and never needs a sequential random stream.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

K = 6
N_KMERS = 4 ** K
# one anchor of a chain: events q..q+len-1 on the diagonal with expected values t..t+len-1
ANCHOR_DTYPE = np.dtype([("q", "<u4"), ("t", "<u4"), ("len", "<u4")])

CANDIDATE_DTYPE = np.dtype(
    {
        "names": ["read_id", "ref_offset", "ref_len_bases", "strand", "pad0", "band_w", "pad1", "slope_num", "slope_den"],
        "formats": ["<u8", "<u8", "<u4", "u1", ("u1", (3,)), "<i4", "<i4", "<i8", "<i8"],
        "offsets": [0, 8, 16, 20, 21, 24, 28, 32, 40],
        "itemsize": 48,
    }
)

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    z = x.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z += np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def hashed_reference(seed: int, n_bases: int) -> np.ndarray:
    """Uniform-ACGT reference of n_bases, packed 4 bases per byte."""
    n_words = (n_bases + 31) // 32
    out = np.empty(n_words, np.uint64)
    base = np.uint64((seed * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF)
    step = 1 << 24
    for lo in range(0, n_words, step):
        idx = np.arange(lo, min(lo + step, n_words), dtype=np.uint64)
        with np.errstate(over="ignore"):
            out[lo : lo + len(idx)] = splitmix64(idx ^ base)
    packed = out.view(np.uint8)[: (n_bases + 3) // 4].copy()
    tail = n_bases % 4
    if tail:
        packed[-1] &= np.uint8((1 << (2 * tail)) - 1)
    return packed


def unpack_bases(ref2bit: np.ndarray, start: int, length: int) -> np.ndarray:
    """Base codes ref[start:start+length] as uint8 0..3."""
    if length <= 0:
        return np.zeros(0, np.uint8)
    b0 = start // 4
    b1 = (start + length + 3) // 4
    chunk = ref2bit[b0:b1]
    codes = np.empty(len(chunk) * 4, np.uint8)
    for s in range(4):
        codes[s::4] = (chunk >> np.uint8(2 * s)) & np.uint8(3)
    off = start - 4 * b0
    return codes[off : off + length]


def gather_bases(ref2bit: np.ndarray, starts: np.ndarray, length: int) -> np.ndarray:
    """Base codes for many windows of equal length: shape (len(starts), length)."""
    pos = starts.astype(np.int64)[:, None] + np.arange(length, dtype=np.int64)[None, :]
    return ((ref2bit[pos >> 2] >> ((pos & 3) * 2).astype(np.uint8)) & np.uint8(3)).astype(np.uint8)


def pack_bases(codes: np.ndarray) -> np.ndarray:
    codes = np.asarray(codes, np.uint8)
    pad = (-len(codes)) % 4
    c = np.concatenate([codes, np.zeros(pad, np.uint8)]).reshape(-1, 4)
    return (c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)).astype(np.uint8)


def write_bases(ref2bit: np.ndarray, start: int, codes: np.ndarray) -> None:
    """Overwrite ref[start:start+len(codes)] in place."""
    for q, c in enumerate(np.asarray(codes, np.uint8)):
        p = start + q
        sh = 2 * (p % 4)
        ref2bit[p // 4] = (ref2bit[p // 4] & np.uint8(~(3 << sh) & 0xFF)) | np.uint8(int(c) << sh)


def write_bases_fast(ref2bit: np.ndarray, start: int, codes: np.ndarray) -> None:
    n = len(codes)
    pos = start + np.arange(n, dtype=np.int64)
    # unpack the touched bytes, modify, repack
    b0, b1 = start // 4, (start + n + 3) // 4
    cur = unpack_bases(ref2bit, 4 * b0, 4 * (b1 - b0)).copy()
    cur[pos - 4 * b0] = codes
    ref2bit[b0:b1] = pack_bases(cur)


def pore_table(seed: int) -> np.ndarray:
    """4^6 expected k-mer currents drawn N(0,1), as if z-scored."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(N_KMERS).astype(np.float32)


def _kmer_means(codes: np.ndarray, pore: np.ndarray) -> np.ndarray:
    """Sequencer model used to *simulate* reads: mean current of each k-mer."""
    L = len(codes) - K + 1
    idx = np.zeros(L, np.int64)
    for t in range(K):
        idx = idx * 4 + codes[t : t + L].astype(np.int64)
    return pore[idx]


def simulate_events(rng, codes, pore, n_events, noise_sd, skip, stay=0.0, mean_dwell=1.1, return_source=False):
    """Walk the k-mers of ``codes``; each emits Geometric(mean mean_dwell)
    events, or none with probability ``skip``; each event is repeated once
    with probability ``stay``; value = k-mer mean + N(0, noise_sd).
    Returns at most n_events values (fewer if the walk runs out), and with
    ``return_source`` also the index of the k-mer each event came from."""
    means = _kmer_means(codes, pore)
    p = 1.0 / mean_dwell
    cnt = rng.geometric(p, size=len(means))
    cnt[rng.random(len(means)) < skip] = 0
    ev_mean = np.repeat(means, cnt)
    src = np.repeat(np.arange(len(means)), cnt)
    if stay > 0:
        dup = rng.random(len(ev_mean)) < stay
        ev_mean = np.repeat(ev_mean, 1 + dup.astype(np.int64))
        src = np.repeat(src, 1 + dup.astype(np.int64))
    ev_mean = ev_mean[:n_events]
    ev = ev_mean + rng.normal(0.0, noise_sd, size=len(ev_mean))
    if return_source:
        return ev.astype(np.float32), src[:n_events]
    return ev.astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    pore: np.ndarray
    ref2bit: np.ndarray
    ref_len: int
    events: np.ndarray
    read_offsets: np.ndarray
    cands: np.ndarray
    k: int = K
    end_mode: int = 0
    b_match: float = 0.4
    score_threshold: float = 20.0
    meta: dict = dataclasses.field(default_factory=dict)
    anchors: np.ndarray | None = None         # ANCHOR_DTYPE, all candidates' chains back to back
    anchor_offsets: np.ndarray | None = None  # n_cands + 1 offsets into anchors

    @property
    def n_reads(self) -> int:
        return len(self.read_offsets) - 1

    @property
    def n_cands(self) -> int:
        return len(self.cands)

    def read_lengths(self) -> np.ndarray:
        return np.diff(self.read_offsets.astype(np.int64))

    def subset(self, cand_idx) -> "Workload":
        """The candidates cand_idx (with their reads) as a self-contained batch."""
        cand_idx = np.asarray(cand_idx, np.int64)
        sel = self.cands[cand_idx].copy()
        reads, inv = np.unique(sel["read_id"].astype(np.int64), return_inverse=True)
        lens = self.read_lengths()[reads]
        offs = np.zeros(len(reads) + 1, np.uint64)
        offs[1:] = np.cumsum(lens)
        ev = np.concatenate([self.events[self.read_offsets[r] : self.read_offsets[r + 1]] for r in reads])
        sel["read_id"] = inv.astype(np.uint64)
        anchors = aoffs = None
        if self.anchor_offsets is not None:
            parts = [self.anchors[self.anchor_offsets[c] : self.anchor_offsets[c + 1]] for c in cand_idx]
            aoffs = np.zeros(len(cand_idx) + 1, np.uint64)
            aoffs[1:] = np.cumsum([len(a) for a in parts])
            anchors = np.concatenate(parts) if parts else np.zeros(0, ANCHOR_DTYPE)
        return dataclasses.replace(self, events=ev.astype(np.float32), read_offsets=offs, cands=sel,
                                   meta=dict(self.meta, subset=len(cand_idx)), anchors=anchors,
                                   anchor_offsets=aoffs)


def _make_cands(n):
    c = np.zeros(n, CANDIDATE_DTYPE)
    return c


def _finish(name, pore, ref, ref_len, reads, cand_rows, meta, end_mode=0):
    lens = np.array([len(r) for r in reads], np.int64)
    offs = np.zeros(len(reads) + 1, np.uint64)
    offs[1:] = np.cumsum(lens)
    events = np.concatenate(reads).astype(np.float32) if reads else np.zeros(0, np.float32)
    cands = _make_cands(len(cand_rows))
    if cand_rows:
        arr = np.array(cand_rows, dtype=np.int64)
        cands["read_id"] = arr[:, 0]
        cands["ref_offset"] = arr[:, 1]
        cands["ref_len_bases"] = arr[:, 2]
        cands["strand"] = arr[:, 3]
        cands["band_w"] = arr[:, 4]
        cands["slope_num"] = arr[:, 5]
        cands["slope_den"] = arr[:, 6]
    return Workload(name, pore, ref, ref_len, events, offs, cands, end_mode=end_mode, meta=meta)


def config_plain(seed: int = 0x5EED0001, n_reads: int = 64, n_events: int = 500, m: int = 550) -> Workload:
    """Plain DTW: 64 reads x 500 events against their true 550-value segment
    of a 20 kb reference, unbanded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref_len = 20_000
    ref = hashed_reference(seed, ref_len)
    span = m + K - 1
    reads, rows = [], []
    for q in range(n_reads):
        while True:
            loc = int(rng.integers(0, ref_len - span - 4 * n_events))
            walk = unpack_bases(ref, loc, 2 * n_events + K)
            ev = simulate_events(rng, walk, pore, n_events, 0.3, 0.05)
            if len(ev) == n_events:
                break
        reads.append(ev)
        rows.append((q, loc, span, 0, -1, 0, 0))
    return _finish("plain", pore, ref, ref_len, reads, rows,
                   dict(config=1, seed=seed, n_reads=n_reads, n_events=n_events, m=m))


def _lognormal_lengths(rng, n, median, sigma, lo, hi):
    x = np.exp(rng.normal(math.log(median), sigma, size=n))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def config_batched(seed: int = 0x5EED0002, n_reads: int = 20_000, ref_len: int = 100_000_000,
                   median: int = 1500, sigma: float = 0.6, lo: int = 200, hi: int = 8000,
                   max_cands: int = 8, band_frac: float = 0.10, true_first: bool = False) -> Workload:
    """Batched uneven DTW: lognormal read lengths (median 1500, 200..8000),
    1..8 candidates per read (1 true + decoys), span = n * U(0.9,1.3), band
    10 % of the span.  true_first puts the true locus first among a read's
    candidates, as sorting by chaining score would (same random draws)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref = hashed_reference(seed, ref_len)
    lens = _lognormal_lengths(rng, n_reads, median, sigma, lo, hi)
    reads, rows = [], []
    for q in range(n_reads):
        n = int(lens[q])
        while True:
            loc = int(rng.integers(0, ref_len - 3 * n - 64))
            walk = unpack_bases(ref, loc, 2 * n + K)
            ev = simulate_events(rng, walk, pore, n, 0.3, 0.05)
            if len(ev) == n:
                break
        reads.append(ev)
        nc = int(rng.integers(1, max_cands + 1))
        true_slot = int(rng.integers(0, nc))
        if true_first:
            true_slot = 0
        for c in range(nc):
            m = int(math.floor(n * rng.uniform(0.9, 1.3)))
            span = m + K - 1
            if c == true_slot:
                off = loc
            else:
                off = int(rng.integers(0, ref_len - span))
            w = int(math.floor(band_frac * m))
            rows.append((q, off, span, 0, w, 0, 0))
    return _finish("batched_uneven", pore, ref, ref_len, reads, rows,
                   dict(config=2, seed=seed, n_reads=n_reads, ref_len=ref_len))


def true_anchors(src, n, m, min_len=8, max_len=16, every=2):
    """Anchors from a simulated read's event -> k-mer map: runs of events
    that step one k-mer per event (as a seed match would cover them), cut to
    at most max_len, every ``every``-th run kept, inside the n x m table."""
    out = []
    i = 0
    run = 0
    while i < n:
        j = i
        while j + 1 < n and src[j + 1] == src[j] + 1:
            j += 1
        ln = j - i + 1
        if ln >= min_len:
            if run % every == 0:
                ln = min(ln, max_len)
                t = int(src[i])
                if t + ln <= m:
                    out.append((i, t, ln))
            run += 1
        i = j + 1
    return out


def decoy_anchors(rng, n, m, k_max=6, min_len=4, max_len=12):
    """A random chain for a decoy locus: sorted, disjoint anchors scattered
    around the table's diagonal."""
    out = []
    pq = pt = 0
    qs = np.sort(rng.integers(0, n, size=int(rng.integers(0, k_max + 1))))
    for q in qs:
        q = int(max(q, pq))
        t = int(max(pt, min(m - 1, round(q * m / n + rng.integers(-8, 9)))))
        ln = int(rng.integers(min_len, max_len + 1))
        ln = min(ln, n - q, m - t)
        if ln < 1:
            continue
        out.append((q, t, ln))
        pq, pt = q + ln, t + ln
    return out


def config_anchored(seed: int = 0x5EED0006, n_reads: int = 20_000, ref_len: int = 100_000_000,
                    median: int = 1500, sigma: float = 0.6, lo: int = 200, hi: int = 8000,
                    max_cands: int = 8, band_frac: float = 0.10) -> Workload:
    """Anchor-guided batch (Sec. 2.4.2): the batched-uneven shapes, and each
    candidate carries a chain: the true locus's anchors come from the
    simulated read's event -> k-mer map, decoys get random chains."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref = hashed_reference(seed, ref_len)
    lens = _lognormal_lengths(rng, n_reads, median, sigma, lo, hi)
    reads, rows, chains = [], [], []
    for q in range(n_reads):
        n = int(lens[q])
        while True:
            loc = int(rng.integers(0, ref_len - 3 * n - 64))
            walk = unpack_bases(ref, loc, 2 * n + K)
            ev, src = simulate_events(rng, walk, pore, n, 0.3, 0.05, return_source=True)
            if len(ev) == n:
                break
        reads.append(ev)
        nc = int(rng.integers(1, max_cands + 1))
        true_slot = int(rng.integers(0, nc))
        for c in range(nc):
            m = int(math.floor(n * rng.uniform(0.9, 1.3)))
            span = m + K - 1
            if c == true_slot:
                off = loc
                chains.append(true_anchors(src, n, m))
            else:
                off = int(rng.integers(0, ref_len - span))
                chains.append(decoy_anchors(rng, n, m))
            w = int(math.floor(band_frac * m))
            rows.append((q, off, span, 0, w, 0, 0))
    wl = _finish("anchored", pore, ref, ref_len, reads, rows,
                 dict(config="anchored", seed=seed, n_reads=n_reads, ref_len=ref_len))
    aoffs = np.zeros(len(chains) + 1, np.uint64)
    aoffs[1:] = np.cumsum([len(ch) for ch in chains])
    flat = [a for ch in chains for a in ch]
    wl.anchors = np.array(flat, dtype=ANCHOR_DTYPE) if flat else np.zeros(0, ANCHOR_DTYPE)
    wl.anchor_offsets = aoffs
    return wl


def config_readuntil(seed: int = 0x5EED0003, n_reads: int = 100_000, ref_len: int = 3_000_000_000,
                     n_events: int = 450, cmin: int = 16, cmax: int = 64, band: int = 64,
                     dup_frac: float = 0.02, block: int = 5000, ident: float = 0.90) -> Workload:
    """Read-Until prefix mapping: 450-event read prefixes, 16..64 candidates
    each (1 true, about half the decoys inside duplicated blocks) on a
    uniform reference where 2 % of the 5 kb blocks are 90 %-identity copies of
    other blocks; band 64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref = hashed_reference(seed, ref_len)
    n_blocks = ref_len // block
    n_dup = max(1, int(dup_frac * n_blocks))
    dst = rng.choice(n_blocks, size=n_dup, replace=False)
    src = rng.integers(0, n_blocks, size=n_dup)
    for d, s in zip(dst.tolist(), src.tolist()):
        codes = unpack_bases(ref, s * block, block).copy()
        mut = rng.random(block) < (1.0 - ident)
        codes[mut] = (codes[mut] + rng.integers(1, 4, size=int(mut.sum()))).astype(np.uint8) & 3
        write_bases_fast(ref, d * block, codes)
    reads, rows = [], []
    for q in range(n_reads):
        n = n_events
        while True:
            loc = int(rng.integers(0, ref_len - 3 * n - 64))
            walk = unpack_bases(ref, loc, 2 * n + K)
            ev = simulate_events(rng, walk, pore, n, 0.3, 0.05)
            if len(ev) == n:
                break
        reads.append(ev)
        nc = int(rng.integers(cmin, cmax + 1))
        true_slot = int(rng.integers(0, nc))
        for c in range(nc):
            m = int(math.floor(n * rng.uniform(0.9, 1.3)))
            span = m + K - 1
            if c == true_slot:
                off = loc
            elif rng.random() < 0.5:
                b = int(dst[rng.integers(0, n_dup)])
                off = b * block + int(rng.integers(0, max(1, block - span)))
                off = min(off, ref_len - span)
            else:
                off = int(rng.integers(0, ref_len - span))
            rows.append((q, off, span, 0, band, 0, 0))
    return _finish("readuntil_prefix", pore, ref, ref_len, reads, rows,
                   dict(config=3, seed=seed, n_reads=n_reads, ref_len=ref_len, dup_blocks=int(n_dup)))


def config_longread(seed: int = 0x5EED0005, n_reads: int = 2000, ref_len: int = 100_000_000,
                    nmin: int = 20_000, nmax: int = 100_000, band_frac: float = 0.05) -> Workload:
    """Long-read banded DTW: 20k-100k events, 2 candidates (true + decoy),
    band 5 % of the span, 5 % skips + 5 % stays, noise sd 0.4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref = hashed_reference(seed, ref_len)
    lens = rng.integers(nmin, nmax + 1, size=n_reads)
    reads, rows = [], []
    for q in range(n_reads):
        n = int(lens[q])
        while True:
            loc = int(rng.integers(0, ref_len - 3 * n - 64))
            walk = unpack_bases(ref, loc, 2 * n + K)
            ev = simulate_events(rng, walk, pore, n, 0.4, 0.05, stay=0.05)
            if len(ev) == n:
                break
        reads.append(ev)
        true_slot = int(rng.integers(0, 2))
        for c in range(2):
            m = int(math.floor(n * rng.uniform(0.9, 1.3)))
            span = m + K - 1
            off = loc if c == true_slot else int(rng.integers(0, ref_len - span))
            rows.append((q, off, span, 0, int(math.floor(band_frac * m)), 0, 0))
    return _finish("long_read", pore, ref, ref_len, reads, rows,
                   dict(config=5, seed=seed, n_reads=n_reads, ref_len=ref_len))


@dataclasses.dataclass
class ServingRead:
    read_id: int
    events: np.ndarray          # up to max_events values
    cands: np.ndarray           # CANDIDATE_DTYPE rows (read_id field = read_id)
    on_target: bool
    arrival_s: float
    true_cand: int = -1         # index of the true locus among cands (-1: off-target)


def config_serving(seed: int = 0x5EED0004, n_reads: int = 2048, ref_len: int = 100_000_000,
                   max_events: int = 4000, cmax: int = 32, band: int = 64, off_target: float = 0.5,
                   rate_per_s: float = 1280.0, noise_sd: float = 0.3, dup_frac: float = 0.0,
                   block: int = 5000, ident: float = 0.90, repeat_reads: float = 0.0):
    """Serving loop inputs: reads that arrive as a Poisson stream (mean rate
    chosen so that about 512 are in flight at 0.4 s per 180-event chunk),
    <= 4000 events each, up to 32 candidates (1 true when on-target), band 64.
    Each candidate carries the band slope the sequencer model implies:
    1 / (0.95 * 1.1) = 1000/1045 reference values per event (mean dwell 1.1
    events per k-mer, 5 % skipped k-mers).

    With dup_frac > 0 the reference has that share of its `block`-base blocks
    overwritten by copies of other blocks at `ident` identity (as the
    Read-Until prefix workload) and about half of the decoys sit in copied
    blocks.  With repeat_reads > 0 that share of the reads come from a block
    that has a copy, and the copy's matching region is one of the decoys: for
    an on-target read a near-duplicate of its true locus, for an off-target
    read a near-duplicate of where its signal came from (the cases where the
    decision can go wrong).  Returns (pore, ref2bit, ref_len, [ServingRead])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pore = pore_table(seed ^ 0xA5A5)
    ref = hashed_reference(seed, ref_len)
    span = int(math.ceil(max_events * 1000 / 1045)) + 2 * band + K
    pairs = []
    if dup_frac > 0:
        n_blocks = ref_len // block
        n_dup = max(1, int(dup_frac * n_blocks))
        dst = rng.choice(n_blocks, size=n_dup, replace=False)
        srcs = rng.integers(0, n_blocks, size=n_dup)
        is_dst = np.zeros(n_blocks, bool)
        is_dst[dst] = True
        for d, sb in zip(dst.tolist(), srcs.tolist()):
            # a source block is never itself overwritten, so every copy
            # stays a near-duplicate of its source
            while is_dst[sb]:
                sb = int(rng.integers(0, n_blocks))
            codes = unpack_bases(ref, sb * block, block).copy()
            mut = rng.random(block) < (1.0 - ident)
            codes[mut] = (codes[mut] + rng.integers(1, 4, size=int(mut.sum()))).astype(np.uint8) & 3
            write_bases_fast(ref, d * block, codes)
            pairs.append((sb, d))
    # a read from a copied block walks 2 * max_events + K bases from its start
    walk_len = 2 * max_events + K
    fits = block - max(span, walk_len)
    if repeat_reads > 0 and dup_frac > 0 and fits <= 0:
        raise ValueError("repeat_reads needs blocks longer than a read's walk (%d bases) and its "
                         "candidate span (%d)" % (walk_len, span))
    out = []
    t = 0.0
    for q in range(n_reads):
        t += rng.exponential(1.0 / rate_per_s)
        rep = None
        if pairs and fits > 0 and rng.random() < repeat_reads:
            sb, d = pairs[int(rng.integers(0, len(pairs)))]
            o = int(rng.integers(0, fits))
            rep = (sb * block + o, d * block + o)
        loc = rep[0] if rep else int(rng.integers(0, ref_len - 3 * max_events - span))
        walk = unpack_bases(ref, loc, walk_len)
        ev = simulate_events(rng, walk, pore, max_events, noise_sd, 0.05)
        on = bool(rng.random() >= off_target)
        if not on:  # events from somewhere else than every candidate
            loc2 = int(rng.integers(0, ref_len - 3 * max_events - span))
            walk = unpack_bases(ref, loc2, walk_len)
            ev_off = simulate_events(rng, walk, pore, max_events, noise_sd, 0.05)
            if rep is None:
                ev = ev_off
            # else: the signal stays that of the copied block's source, which is
            # not a candidate; its near-duplicate (the copy) is
        nc = int(rng.integers(1, cmax + 1))
        if rep and nc < 2:
            nc = 2
        c = np.zeros(nc, CANDIDATE_DTYPE)
        true_slot = int(rng.integers(0, nc))
        copy_slot = (true_slot + 1 + int(rng.integers(0, nc - 1))) % nc if rep else -1
        for s_ in range(nc):
            if on and s_ == true_slot:
                off = loc
            elif s_ == copy_slot:
                off = rep[1]
            elif pairs and dup_frac > 0 and rng.random() < 0.5:
                d = pairs[int(rng.integers(0, len(pairs)))][1]
                off = min(d * block + int(rng.integers(0, max(1, block - span))), ref_len - span)
            else:
                off = int(rng.integers(0, ref_len - span))
            c[s_] = (q, off, span, 0, 0, band, 0, 1000, 1045)
        out.append(ServingRead(q, ev, c, on, t, true_cand=true_slot if on else -1))
    return pore, ref, ref_len, out


def scaled(name: str, scale: str = "full", seed: int | None = None) -> Workload:
    """Workload by config name at 'full' or 'small' (oracle-sized) scale."""
    kw = {} if seed is None else {"seed": seed}
    if name == "plain":
        return config_plain(**kw) if scale == "full" else config_plain(n_reads=8, **kw)
    if name == "batched":
        if scale == "full":
            return config_batched(**kw)
        return config_batched(n_reads=48, ref_len=2_000_000, median=400, lo=60, hi=1500, **kw)
    if name == "readuntil":
        if scale == "full":
            return config_readuntil(**kw)
        return config_readuntil(n_reads=24, ref_len=4_000_000, cmin=4, cmax=12, **kw)
    if name == "anchored":
        if scale == "full":
            return config_anchored(**kw)
        return config_anchored(n_reads=40, ref_len=2_000_000, median=400, lo=60, hi=1500, **kw)
    if name == "longread":
        if scale == "full":
            return config_longread(**kw)
        return config_longread(n_reads=3, ref_len=2_000_000, nmin=2000, nmax=4000, **kw)
    raise KeyError(name)
