"""Autotuner for the striped DTW kernel's variants.

Each variant (lanes per alignment G, rows per lane HR) is timed on a batch
made for it: alignments whose band is just wide enough that the variant's
lanes never wait between stripes (2w >= (G*HR - HR + 1) + G + 4 columns at
slope 1), about four stripes long, and enough of them to keep every resident
group busy several times over.  The measured lane-cell slots per second of
each variant give its relative slot cost (1.0 = the fastest); the planner
picks, per alignment, the variant with the fewest cost-weighted slots.

    costs = tune()                      # {(G, HR): cost}
    write_table("tune.txt", costs)      # "G HR cost" lines
    Aligner(..., autotune_path="tune.txt")
"""
from __future__ import annotations

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


def tune(device="cuda:0", runs=3, sm_count=None, groups_factor=4, verbose=False):
    """Returns {(G, HR): relative slot cost} measured on this GPU."""
    import torch

    if sm_count is None:
        sm_count = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
    theta = {}
    for v, (G, HR) in enumerate(B.VARIANTS):
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


def write_table(path, costs):
    with open(path, "w") as f:
        for (G, HR), c in costs.items():
            f.write("%d %d %.6f\n" % (G, HR, c))


def read_table(path):
    costs = {}
    for line in open(path):
        parts = line.split()
        if len(parts) == 3:
            costs[(int(parts[0]), int(parts[1]))] = float(parts[2])
    return costs


def apply(aligner, costs):
    """Sets the measured costs on an open Aligner."""
    B.rawalign_dtw_set_variant_costs(aligner.h, [costs.get(gh, 1.0) for gh in B.VARIANTS])
