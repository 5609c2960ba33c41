"""Autotuner for the striped DTW kernel and its planner.

Slot costs: each variant (lanes per alignment G, rows per lane HR) is timed on
a batch made for it: alignments whose band is just wide enough that the
variant's lanes never wait between stripes, about four stripes long, and
enough of them to keep every resident group busy several times over.  The
measured lane-cell slots per second of each variant give its relative slot
cost (1.0 = the fastest); the planner picks, per alignment, the variant with
the fewest cost-weighted slots.

Bin edges: the planner cuts a batch into launch classes of one variant and
one ring size (the ring holds the bottom row of a stripe for the next one, so
its size follows the band width), and moves an alignment that would outlast
the batch to a 32-lane variant.  tune_plan() times a sample batch under each
choice of ring-size bins (powers of 4 or of 2) and of that latency split and
keeps the fastest.

    costs = tune()                                  # {(G, HR): cost}
    plan = tune_plan(sample_workload, costs)[0]     # {"ring_bins": s, "latency_split": x}
    write_table("tune.txt", costs, plan)            # "G HR cost" lines + knobs
    Aligner(..., autotune_path="tune.txt")
"""
from __future__ import annotations

import os
import tempfile

import numpy as np

from . import binding as B
from . import synth as S


def calibration_batch(G, HR, n_align, seed=0):
    """n_align alignments shaped for variant (G, HR), random signal."""
    H = G * HR
    w = (H - HR + 1 + G + 4 + 1) // 2
    n = 4 * H
    m = n
    k = S.K
    rng = np.random.default_rng(seed)
    pore = S.pore_table(seed + 1)
    ref_len = max(4 * (m + k), 1 << 16)
    ref = S.hashed_reference(seed + 2, ref_len)
    events = rng.normal(size=n_align * n).astype(np.float32)
    offs = (np.arange(n_align + 1, dtype=np.uint64) * n).astype(np.uint64)
    cands = np.zeros(n_align, S.CANDIDATE_DTYPE)
    cands["read_id"] = np.arange(n_align)
    cands["ref_offset"] = rng.integers(0, ref_len - (m + k), size=n_align)
    cands["ref_len_bases"] = m + k - 1
    cands["band_w"] = w
    return pore, ref, ref_len, events, offs, cands


def tune(device="cuda:0", runs=3, sm_count=None, groups_factor=4, verbose=False, variants=None):
    """Returns {(G, HR): relative slot cost} measured on this GPU."""
    import torch

    if sm_count is None:
        sm_count = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
    theta = {}
    for v, (G, HR) in enumerate(B.VARIANTS):
        if variants is not None and (G, HR) not in variants:
            continue
        # resident groups: about 5 blocks of 128 threads per SM
        n_align = max(64, sm_count * 5 * (128 // G) * groups_factor // 4)
        pore, ref, ref_len, ev, offs, cands = calibration_batch(G, HR, n_align, seed=v)
        need = B.rawalign_dtw_batch_bytes(len(ev), len(offs) - 1, len(cands),
                                          int(np.sum(cands["ref_len_bases"].astype(np.int64) - S.K + 1)))
        al = B.Aligner(pore, ref, ref_len, arena_bytes=need + len(ref) + (64 << 20), kernel=B.RA_KERNEL_STRIPE[(G, HR)],
                       device=device)
        try:
            b = al.prepare(ev, offs, cands)
            al.poll(al.run(b), 0)
            best = None
            for _ in range(runs):
                al.poll(al.run(b), 0)
                st = al.stats(b)
                rate = st.slots / (st.dtw_ms / 1e3)
                best = rate if best is None else max(best, rate)
            theta[(G, HR)] = best
            if verbose:
                print("variant G=%d HR=%d: %.3g slots/s (%d alignments)" % (G, HR, best, n_align))
            al.release(b)
        finally:
            al.close()
    top = max(theta.values())
    return {gh: top / t for gh, t in theta.items()}


def tune_plan(workload, costs=None, device="cuda:0", runs=3, ring_bins=(2, 1), latency_splits=(0.0, 0.5, 1.0, 2.0),
              block_splits=(None,), arena_bytes=None):
    """Chooses the planner's bin edges on a sample batch (a synth.Workload):
    every (ring_bins, latency_split, block_split) choice is timed (best of
    `runs` replays of the DTW part; block_split None = the library's default);
    returns (best {"ring_bins", "latency_split"[, "block_split"]}, {choice: ms})."""
    w = workload
    if arena_bytes is None:
        m_total = int(np.sum(w.cands["ref_len_bases"].astype(np.int64) - w.k + 1))
        arena_bytes = 2 * B.rawalign_dtw_batch_bytes(len(w.events), w.n_reads, w.n_cands, m_total) + \
            len(w.ref2bit) + (512 << 20)
    times = {}
    with tempfile.TemporaryDirectory() as d:
        for rb, ls, bs in [(rb, ls, bs) for rb in ring_bins for ls in latency_splits for bs in block_splits]:
            path = os.path.join(d, "t_%d_%g_%s.txt" % (rb, ls, bs))
            knobs = {"ring_bins": rb, "latency_split": ls}
            if bs is not None:
                knobs["block_split"] = bs
            write_table(path, costs or {}, knobs)
            al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena_bytes, k=w.k, device=device,
                           autotune_path=path)
            try:
                b = al.prepare(w.events, w.read_offsets, w.cands)
                al.poll(al.run(b), 0)
                best = None
                for _ in range(runs):
                    al.poll(al.run(b), 0)
                    ms = al.stats(b).dtw_ms
                    best = ms if best is None else min(best, ms)
                times[(rb, ls) if bs is None else (rb, ls, bs)] = best
                al.release(b)
            finally:
                al.close()
    best = min(times, key=times.get)
    plan = {"ring_bins": best[0], "latency_split": best[1]}
    if len(best) > 2:
        plan["block_split"] = best[2]
    return plan, times


def write_table(path, costs, plan=None):
    """The tuning file: "G HR cost" lines, then the planner knobs."""
    with open(path, "w") as f:
        for (G, HR), c in costs.items():
            f.write("%d %d %.6f\n" % (G, HR, c))
        if plan:
            if "ring_bins" in plan:
                f.write("ring_bins %d\n" % int(plan["ring_bins"]))
            if "latency_split" in plan:
                f.write("latency_split %.6f\n" % float(plan["latency_split"]))
            if "block_split" in plan:
                f.write("block_split %.6f\n" % float(plan["block_split"]))


def read_table(path):
    """(costs {(G, HR): cost}, plan knobs {name: value}) from a tuning file."""
    costs, plan = {}, {}
    for line in open(path):
        parts = line.split()
        if len(parts) == 3:
            costs[(int(parts[0]), int(parts[1]))] = float(parts[2])
        elif len(parts) == 2 and parts[0] == "ring_bins":
            plan["ring_bins"] = int(parts[1])
        elif len(parts) == 2 and parts[0] in ("latency_split", "block_split"):
            plan[parts[0]] = float(parts[1])
    return costs, plan


def apply(aligner, costs):
    """Sets the measured slot costs on an open Aligner (the planner knobs
    come only from a tuning file given at creation)."""
    B.rawalign_dtw_set_variant_costs(aligner.h, [costs.get(gh, 1.0) for gh in B.VARIANTS])
