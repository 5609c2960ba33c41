"""The FP32 oracle over all host cores, for full-size parity.

The oracle itself stays the plain single-threaded C of ``oracle/``; this
helper only cuts a workload into groups of whole reads (so that each read's
best candidate and decision come out of one oracle call) and runs
``oracle.map_batch`` / ``oracle.map_anchored`` on the groups from a thread
pool.  ctypes releases the GIL for the duration of each foreign call, so the
groups run in parallel on the host cores.  Results come back in the
workload's candidate order with ``read_id`` and ``cand_idx`` restored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import time

import numpy as np

import oracle as O


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _groups(w, cand_idx, n_groups):
    """Whole reads of the selected candidates, dealt into n_groups groups of
    about equal table area (n*m, what the oracle's loop visits)."""
    cand_idx = np.asarray(cand_idx, np.int64)
    rid = w.cands["read_id"][cand_idx].astype(np.int64)
    n = w.read_lengths()[rid]
    m = w.cands["ref_len_bases"][cand_idx].astype(np.int64) - w.k + 1
    reads, inv = np.unique(rid, return_inverse=True)
    area = np.bincount(inv, weights=(n * m).astype(np.float64), minlength=len(reads))
    n_groups = max(1, min(n_groups, len(reads)))
    # largest reads first, each to the lightest group so far
    load = np.zeros(n_groups)
    owner = np.empty(len(reads), np.int64)
    for q in np.argsort(-area, kind="stable"):
        g = int(np.argmin(load))
        owner[q] = g
        load[g] += area[q]
    return [cand_idx[owner[inv] == g] for g in range(n_groups)]


def map_parallel(w, cand_idx=None, use_f64=False, workers=None, anchored=False):
    """Oracle results (RESULT_DTYPE) for w.cands[cand_idx] (all by default),
    in that order, and a dict with the wall time and the threads used."""
    if cand_idx is None:
        cand_idx = np.arange(w.n_cands)
    cand_idx = np.asarray(cand_idx, np.int64)
    workers = workers or cores()
    O.lib()  # build and load once, before the threads start
    groups = [g for g in _groups(w, cand_idx, 4 * workers) if len(g)]

    def run(g):
        g = np.sort(g)
        sub = w.subset(g)
        if anchored:
            res = O.map_anchored(sub.k, sub.b_match, sub.score_threshold, sub.pore, sub.ref2bit, sub.ref_len,
                                 sub.events, sub.read_offsets, sub.cands, sub.anchors, sub.anchor_offsets,
                                 use_f64=use_f64)
        else:
            res = O.map_batch(sub.k, sub.b_match, sub.score_threshold, sub.end_mode, sub.pore, sub.ref2bit,
                              sub.ref_len, sub.events, sub.read_offsets, sub.cands, use_f64=use_f64)
        res["read_id"] = w.cands["read_id"][g]
        res["cand_idx"] = g.astype(np.uint32)
        return g, res

    t0 = time.perf_counter()
    out = np.zeros(len(cand_idx), O.RESULT_DTYPE)
    pos = np.full(w.n_cands, -1, np.int64)
    pos[cand_idx] = np.arange(len(cand_idx))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for g, res in ex.map(run, groups):
            out[pos[g]] = res
    info = {"seconds": time.perf_counter() - t0, "threads": workers, "alignments": len(cand_idx)}
    return out, info
