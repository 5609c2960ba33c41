"""Read-Until request loop over the C ABI (submit_chunk / flush / poll).

Reads deliver their signal in chunks of events; after every chunk the library
reports, per candidate, the cost and score of the prefix aligned so far and
the read's decision (Sec. 2.3).  The loop stops a read when it is mapped
(accept), when no candidate can reach Score_Threshold any more even if every
remaining event matched perfectly (reject: B_Match * max_events - cost <
threshold, the cost can only grow), or at max_events.  Stopped reads are
closed, which returns their slot and device memory to the library.

Two modes:
  closed loop: a fixed number of reads in flight; a read's next chunk is
               submitted as soon as its previous result is back (sustained
               throughput).
  real time:   reads arrive as a Poisson stream and every chunk becomes
               available chunk_s seconds after the previous one (latency at the
               sequencer's pace).
Every flush launches all chunks queued since the previous flush as one batch
(continuous batching).  Chunk latency = time from submit to result visible.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class ServeStats:
    chunks: int = 0
    cells: int = 0
    reads_done: int = 0
    accepted: int = 0
    rejected: int = 0
    exhausted: int = 0
    wall_s: float = 0.0
    latencies_ms: list = dataclasses.field(default_factory=list)

    def summary(self):
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {
            "chunks": self.chunks, "reads_decided": self.reads_done, "accepted": self.accepted,
            "rejected": self.rejected, "max_events": self.exhausted, "wall_s": round(self.wall_s, 3),
            "gcups": round(self.cells / max(self.wall_s, 1e-9) / 1e9, 3),
            "reads_per_s": round(self.reads_done / max(self.wall_s, 1e-9), 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
        }


class _Live:
    __slots__ = ("rd", "pos", "ticket", "t_submit", "next_ready")

    def __init__(self, rd, next_ready):
        self.rd = rd
        self.pos = 0
        self.ticket = None
        self.t_submit = 0.0
        self.next_ready = next_ready


class ServingLoop:
    def __init__(self, aligner, reads, chunk=180, max_events=4000, b_match=0.4, threshold=20.0):
        self.al = aligner
        self.reads = list(reads)
        self.chunk = chunk
        self.max_events = max_events
        self.b_match = b_match
        self.threshold = threshold

    def _decide(self, live, res, st):
        """True when the read stops after this result."""
        n = live.pos
        if len(res) and np.any(res["decision"] == B.RA_MAPPED):
            st.accepted += 1
            return True
        best_possible = self.b_match * self.max_events - res["cost"].astype(np.float64)
        if len(res) == 0 or np.all(best_possible < self.threshold):
            st.rejected += 1
            return True
        if n >= min(self.max_events, len(live.rd.events)):
            st.exhausted += 1
            return True
        return False

    def _submit(self, live, now):
        rd = live.rd
        p = live.pos
        q = min(p + self.chunk, len(rd.events), self.max_events)
        last = q >= min(self.max_events, len(rd.events))
        live.ticket = B.rawalign_dtw_submit_chunk(self.al.h, rd.read_id, rd.events[p:q],
                                                  rd.cands if p == 0 else None, last)
        live.t_submit = now
        live.pos = q
        return last

    def run(self, max_chunks=10_000, in_flight=512, realtime=False, chunk_s=0.4, duration_s=None,
            arrival_rate=None):
        st = ServeStats()
        pending_reads = list(self.reads)
        live = {}
        closed = []
        t0 = time.perf_counter()
        rng = np.random.default_rng(1)
        next_arrival = t0
        while True:
            now = time.perf_counter()
            if duration_s is not None and now - t0 > duration_s:
                break
            if st.chunks >= max_chunks or (not pending_reads and not live):
                break
            # admit new reads (closed loop: keep in_flight busy; real time: Poisson arrivals)
            while pending_reads and len(live) < in_flight and (not realtime or now >= next_arrival):
                rd = pending_reads.pop(0)
                lv = _Live(rd, now)
                try:
                    self._submit(lv, now)
                except B.RawAlignError as e:
                    if e.code == B.RA_EAGAIN:  # admission refused: retry later
                        pending_reads.insert(0, rd)
                        break
                    raise
                live[rd.read_id] = lv
                if realtime:
                    next_arrival += rng.exponential(1.0 / arrival_rate)
            # closed loop / real time: submit next chunks of reads whose result came back
            for lv in live.values():
                if lv.ticket is None and (not realtime or now >= lv.next_ready):
                    self._submit(lv, now)
            B.rawalign_dtw_flush(self.al.h)
            # collect results
            done_ids = []
            for rid, lv in live.items():
                if lv.ticket is None:
                    continue
                res = B.rawalign_dtw_poll(self.al.h, lv.ticket, 64, timeout_us=-1)
                t = time.perf_counter()
                st.latencies_ms.append((t - lv.t_submit) * 1e3)
                st.chunks += 1
                st.cells += int(res["cells"].sum()) if len(res) else 0
                lv.ticket = None
                lv.next_ready = lv.t_submit + chunk_s
                if self._decide(lv, res, st):
                    done_ids.append(rid)
            for rid in done_ids:
                lv = live.pop(rid)
                st.reads_done += 1
                if lv.pos < min(self.max_events, len(lv.rd.events)):
                    closed.append(B.rawalign_dtw_submit_chunk(self.al.h, rid, np.zeros(0, np.float32), None, True))
            if closed:
                B.rawalign_dtw_flush(self.al.h)
                for t in closed:
                    B.rawalign_dtw_poll(self.al.h, t, 0, timeout_us=-1)
                closed = []
            if realtime:
                waits = [lv.next_ready for lv in live.values() if lv.ticket is None]
                nxt = min(waits + ([next_arrival] if pending_reads else []), default=now)
                dt = nxt - time.perf_counter()
                if dt > 0:
                    time.sleep(min(dt, 0.005))
        st.wall_s = time.perf_counter() - t0
        # close whatever is still open so the library frees it
        for rid, lv in live.items():
            if lv.ticket is not None:
                B.rawalign_dtw_poll(self.al.h, lv.ticket, 64, timeout_us=-1)
            if lv.pos < min(self.max_events, len(lv.rd.events)):
                t = B.rawalign_dtw_submit_chunk(self.al.h, rid, np.zeros(0, np.float32), None, True)
                B.rawalign_dtw_flush(self.al.h)
                B.rawalign_dtw_poll(self.al.h, t, 0, timeout_us=-1)
        return st


@dataclasses.dataclass
class Trajectory:
    """One read's results after each chunk: events aligned so far, the best
    candidate's score and index, and the smallest cost over its candidates."""
    read_id: int
    on_target: bool
    true_cand: int
    events: list = dataclasses.field(default_factory=list)
    best_score: list = dataclasses.field(default_factory=list)
    best_cand: list = dataclasses.field(default_factory=list)
    min_cost: list = dataclasses.field(default_factory=list)
    mapped: list = dataclasses.field(default_factory=list)  # the library's decision at its own threshold


def collect_trajectories(aligner, reads, chunk=180, max_events=4000, in_flight=512):
    """Feeds every read chunk by chunk up to max_events (or its end) through
    submit_chunk / flush / poll, keeping in_flight reads admitted, and
    records each read's trajectory.  Reads are not stopped early, so every
    threshold can be studied on the same trajectories."""
    pending = list(reads)
    live = {}
    out = {}
    while pending or live:
        while pending and len(live) < in_flight:
            rd = pending[0]
            q = min(chunk, len(rd.events), max_events)
            last = q >= min(max_events, len(rd.events))
            try:
                t = B.rawalign_dtw_submit_chunk(aligner.h, rd.read_id, rd.events[:q], rd.cands, last)
            except B.RawAlignError as e:
                if e.code == B.RA_EAGAIN:
                    break
                raise
            pending.pop(0)
            live[rd.read_id] = [rd, q, t]
            out[rd.read_id] = Trajectory(rd.read_id, rd.on_target, getattr(rd, "true_cand", -1))
        B.rawalign_dtw_flush(aligner.h)
        done = []
        for rid, st in live.items():
            rd, q, t = st
            res = B.rawalign_dtw_poll(aligner.h, t, 64, timeout_us=-1)
            tr = out[rid]
            sc = res["score"].astype(np.float64)
            b = int(np.argmax(sc)) if len(sc) else -1
            tr.events.append(q)
            tr.best_score.append(float(sc[b]) if b >= 0 else -np.inf)
            tr.best_cand.append(b)
            tr.min_cost.append(float(res["cost"].min()) if len(res) else np.inf)
            tr.mapped.append(bool(len(res) and np.any(res["decision"] == B.RA_MAPPED)))
            end = min(max_events, len(rd.events))
            if q >= end:
                done.append(rid)
                continue
            q2 = min(q + chunk, end)
            st[1] = q2
            st[2] = B.rawalign_dtw_submit_chunk(aligner.h, rid, rd.events[q:q2], None, q2 >= end)
        for rid in done:
            live.pop(rid)
    return [out[rd.read_id] for rd in reads if rd.read_id in out]


def decision_study(trajectories, thresholds, b_match=0.4, max_events=4000):
    """Read-Until decision policy (Sec. 1, Sec. 3.1) replayed on recorded
    trajectories for several Score_Threshold values.  After each chunk a read
    is accepted when its best score reaches the threshold, rejected when no
    candidate can reach it any more even if every remaining event matched
    exactly (B_Match * max_events - smallest cost < threshold; costs only
    grow), else it continues; at max_events it is undecided.  Per threshold:
    counts, the share of accepted reads whose best candidate is the true
    locus (precision), the share of on-target reads accepted at their true
    locus (recall), and the events consumed before the decision."""
    out = {}
    for thr in thresholds:
        acc = rej = und = tp = 0
        ev_acc, ev_rej, ev_all = [], [], []
        on_total = sum(tr.on_target for tr in trajectories)
        for tr in trajectories:
            decided = None
            for k, n_ev in enumerate(tr.events):
                if tr.best_score[k] >= thr:
                    decided = ("accept", n_ev, tr.best_cand[k])
                    break
                if b_match * max_events - tr.min_cost[k] < thr:
                    decided = ("reject", n_ev, -1)
                    break
            if decided is None:
                und += 1
                ev_all.append(tr.events[-1] if tr.events else 0)
                continue
            kind, n_ev, cand = decided
            ev_all.append(n_ev)
            if kind == "accept":
                acc += 1
                ev_acc.append(n_ev)
                tp += int(tr.on_target and cand == tr.true_cand)
            else:
                rej += 1
                ev_rej.append(n_ev)
        out[float(thr)] = {
            "accepted": acc, "rejected": rej, "undecided": und,
            "precision": round(tp / acc, 4) if acc else None,
            "recall": round(tp / on_total, 4) if on_total else None,
            "mean_events_to_accept": round(float(np.mean(ev_acc)), 1) if ev_acc else None,
            "mean_events_to_reject": round(float(np.mean(ev_rej)), 1) if ev_rej else None,
            "median_events_to_decision": float(np.median(ev_all)) if ev_all else None,
        }
    return out
