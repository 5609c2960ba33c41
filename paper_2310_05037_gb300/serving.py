"""Read-Until request loop over the C ABI (submit_chunks / flush / poll_chunks).

Reads deliver their signal in chunks of events; after every chunk the library
reports, per candidate, the cost and score of the prefix aligned so far and
the read's decision (Sec. 2.3): MAPPED (accept), UNMAPPED (reject: with the
handle's serve_early_reject, as soon as no candidate can reach
Score_Threshold any more even if every remaining event up to max_events
matched exactly; the cost only grows), or PENDING.  The loop stops a read at
its decision or at max_events; a read stopped early is closed with an empty
last chunk, which returns its slot and device memory to the library.

Two modes:
  closed loop: a fixed number of reads in flight; a read's next chunk is
               submitted as soon as its previous result is back (sustained
               throughput).
  real time:   reads arrive as a Poisson stream and every chunk becomes
               available chunk_s seconds after the previous one (latency at the
               sequencer's pace).
Every round submits the chunks of every ready read in one call and launches
them as one flush (continuous batching).  In closed loop the reads are split
into two generations: while one generation's flush runs on the GPU, the
other's results are read back, decided and its next chunks submitted, so the
host work of one generation overlaps the device work of the other.  Chunk
latency = time from submit to result visible on the host.
"""
from __future__ import annotations

import collections
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
    flushes: int = 0
    latencies_ms: list = dataclasses.field(default_factory=list)
    host: dict = dataclasses.field(default_factory=dict)

    def summary(self):
        lat = np.concatenate([np.asarray(x, np.float64).ravel() for x in self.latencies_ms]) \
            if self.latencies_ms else np.zeros(1)
        out = {
            "chunks": self.chunks, "reads_decided": self.reads_done, "accepted": self.accepted,
            "rejected": self.rejected, "max_events": self.exhausted, "wall_s": round(self.wall_s, 3),
            "gcups": round(self.cells / max(self.wall_s, 1e-9) / 1e9, 3),
            "reads_per_s": round(self.reads_done / max(self.wall_s, 1e-9), 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "flushes": self.flushes,
        }
        if self.host:
            out["breakdown_ms"] = {k: round(v, 2) for k, v in self.host.items()}
        return out


class ServingLoop:
    def __init__(self, aligner, reads, chunk=180, max_events=4000):
        self.al = aligner
        self.reads = list(reads)
        self.chunk = chunk
        self.max_events = max_events
        n = len(self.reads)
        # every read's events (up to max_events) and candidates back to back:
        # chunks index into these arrays, nothing is copied per chunk
        self.n_ev = np.array([min(len(rd.events), max_events) for rd in self.reads], np.int64)
        self.ev_off = np.zeros(n + 1, np.int64)
        self.ev_off[1:] = np.cumsum(self.n_ev)
        self.events = (np.concatenate([rd.events[:max_events] for rd in self.reads]).astype(np.float32)
                       if n else np.zeros(0, np.float32))
        self.n_cand = np.array([len(rd.cands) for rd in self.reads], np.int64)
        self.cand_off = np.zeros(n + 1, np.int64)
        self.cand_off[1:] = np.cumsum(self.n_cand)
        self.cands = np.concatenate([rd.cands for rd in self.reads]) if n else np.zeros(0, B.CANDIDATE_DTYPE)
        self.read_id = np.array([rd.read_id for rd in self.reads], np.uint64)

    def _chunks(self, q, pos, close):
        """Chunk records for reads q (the next chunk from pos; close: empty
        closing chunks)."""
        ch = np.zeros(len(q), B.CHUNK_DTYPE)
        ch["read_id"] = self.read_id[q]
        if close:
            ch["last"] = 1
            return ch
        end = self.n_ev[q]
        stop = np.minimum(pos + self.chunk, end)
        ch["ev_offset"] = self.ev_off[q] + pos
        ch["n_events"] = stop - pos
        first = pos == 0
        ch["cand_offset"] = np.where(first, self.cand_off[q], 0)
        ch["n_cands"] = np.where(first, self.n_cand[q], 0)
        ch["last"] = (stop >= end).astype(np.int32)
        return ch

    def run(self, max_chunks=10_000, in_flight=512, realtime=False, chunk_s=0.4, duration_s=None,
            arrival_rate=None, generations=2):
        """Closed loop (default) or real time; returns ServeStats."""
        h = self.al.h
        st = ServeStats()
        n = len(self.reads)
        pos = np.zeros(n, np.int64)            # events submitted so far
        ready_at = np.zeros(n, np.float64)     # when the read's next chunk may go
        live = np.zeros(n, bool)               # admitted and not decided
        busy = np.zeros(n, bool)               # a chunk in flight
        idle = np.zeros(n, bool)               # live and not busy (kept with live and busy)
        n_live = 0
        pending = collections.deque(range(n))  # reads not admitted yet
        to_close = []                          # reads decided early, still open in the library
        gens = collections.deque()             # (tickets, reads, t_submit, closing tickets)
        rng = np.random.default_rng(1)
        t_sub = t_flush = t_poll = 0.0
        B.rawalign_dtw_serve_stats(h, reset=True)
        t0 = time.perf_counter()
        next_arrival = t0
        gen_cap = in_flight if realtime else max(1, -(-in_flight // max(1, generations)))
        res_buf = np.zeros(0, B.RESULT_DTYPE)  # poll_chunks writes here (grown on demand, reused)

        while True:
            now = time.perf_counter()
            if duration_s is not None and now - t0 > duration_s:
                break
            if st.chunks >= max_chunks:
                break
            if not pending and n_live == 0 and not gens and not to_close:
                break
            # admission: closed loop keeps in_flight reads live, real time
            # admits Poisson arrivals
            newq = []
            while pending and n_live + len(newq) < in_flight and (not realtime or now >= next_arrival):
                newq.append(pending.popleft())
                if realtime:
                    next_arrival += rng.exponential(1.0 / arrival_rate)
            if newq:
                newq = np.array(newq, np.int64)
                live[newq] = True
                idle[newq] = True
                n_live += len(newq)
                ready_at[newq] = now
            # the reads whose next chunk can go now: in closed loop at most one
            # generation's worth, and only while fewer generations are in flight
            if realtime:
                q = np.flatnonzero(idle & (ready_at <= now))
            elif len(gens) < generations:
                q = np.flatnonzero(idle)[:gen_cap]
            else:
                q = np.zeros(0, np.int64)
            closes = np.array(to_close, np.int64)
            to_close = []
            if len(q) or len(closes):
                t_start = time.perf_counter()  # a chunk's latency runs from here to its result on the host
                ch = self._chunks(q, pos[q], False)
                if len(closes):
                    ch = np.concatenate([ch, self._chunks(closes, pos[closes], True)])
                a = time.perf_counter()
                tickets, status = B.rawalign_dtw_submit_chunks(h, ch, self.events, self.cands)
                t_sub += time.perf_counter() - a
                sq = status[: len(q)]
                ok = sq == B.RA_OK
                if not ok.all() or status[len(q):].any():
                    bad = np.concatenate([sq[~ok & (sq != B.RA_EAGAIN)], status[len(q):][status[len(q):] != 0]])
                    if len(bad):
                        raise B.RawAlignError("rawalign_dtw_submit_chunks", int(bad[0]))
                    # reads refused admission (no slot or arena memory) wait in front
                    refused = q[sq == B.RA_EAGAIN]
                    live[refused] = False
                    n_live -= len(refused)
                    pending.extendleft(reversed(refused.tolist()))
                    qs = q[ok]
                    pos[qs] += ch["n_events"][: len(q)][ok].astype(np.int64)
                else:
                    qs = q
                    pos[qs] += ch["n_events"][: len(q)].astype(np.int64)
                idle[q] = False
                busy[qs] = True
                a = time.perf_counter()
                B.rawalign_dtw_flush(h)
                t_flush += time.perf_counter() - a
                st.flushes += 1
                gens.append((tickets[: len(q)][ok] if len(qs) < len(q) else tickets[: len(q)], qs, t_start,
                             tickets[len(q):]))
            # read back the oldest generation: in closed loop when the others
            # are on the GPU (or nothing else can start), in real time as soon
            # as it has completed
            while gens:
                tk, qs, ts, ctk = gens[0]
                must = (not realtime) and (len(gens) >= generations or not idle.any())
                a = time.perf_counter()
                cap = int(self.n_cand[qs].sum()) + 1
                if len(res_buf) < cap:
                    res_buf = np.zeros(2 * cap, B.RESULT_DTYPE)
                got = B.rawalign_dtw_poll_chunks(h, np.concatenate([tk, ctk]) if len(ctk) else tk, cap,
                                                 timeout_us=-1 if must else 0, out=res_buf)
                t_poll += time.perf_counter() - a
                if got is None:
                    break
                gens.popleft()
                res, counts = got
                tv = time.perf_counter()
                counts = counts[: len(tk)].astype(np.int64)
                st.latencies_ms.append(np.full(len(tk), (tv - ts) * 1e3))
                st.chunks += len(tk)
                st.cells += int(res["cells"].sum())
                # a chunk's results carry its read's decision (every candidate the same)
                starts = np.cumsum(counts) - counts
                has = counts > 0
                if has.all():
                    dec = res["decision"][starts].astype(np.int64)
                else:
                    dec = np.full(len(tk), B.RA_PENDING, np.int64)
                    dec[has] = res["decision"][starts[has]]
                busy[qs] = False
                ready_at[qs] = ts + chunk_s if realtime else tv
                at_end = pos[qs] >= self.n_ev[qs]
                acc = dec == B.RA_MAPPED
                rej = (dec == B.RA_UNMAPPED) & ~at_end
                exh = at_end & ~acc
                done = acc | rej | exh
                st.accepted += int(acc.sum())
                st.rejected += int(rej.sum())
                st.exhausted += int(exh.sum())
                n_done = int(done.sum())
                st.reads_done += n_done
                n_live -= n_done
                live[qs[done]] = False
                idle[qs] = ~done
                # decided before their last chunk: closed in the next round
                to_close.extend(qs[done & ~at_end].tolist())
                if must:
                    break
            if realtime and not gens and not to_close:
                waits = ready_at[live & ~busy]
                cands_t = ([float(waits.min())] if len(waits) else []) + ([next_arrival] if pending else [])
                dt = (min(cands_t) if cands_t else now) - time.perf_counter()
                if dt > 0:
                    time.sleep(min(dt, 0.002))
        st.wall_s = time.perf_counter() - t0
        # drain: results still in flight, then close every read left open
        while gens:
            tk, qs, ts, ctk = gens.popleft()
            B.rawalign_dtw_poll_chunks(h, np.concatenate([tk, ctk]), int(self.n_cand[qs].sum()) + 1)
            busy[qs] = False
        open_q = sorted(set(to_close) | set(np.nonzero(live & (pos > 0) & (pos < self.n_ev))[0].tolist()))
        if open_q:
            open_q = np.array(open_q, np.int64)
            tickets, status = B.rawalign_dtw_submit_chunks(h, self._chunks(open_q, pos[open_q], True),
                                                           self.events, self.cands)
            B.rawalign_dtw_flush(h)
            B.rawalign_dtw_poll_chunks(h, tickets[status == B.RA_OK], 1)
        lib = B.rawalign_dtw_serve_stats(h, reset=True)
        st.host = {"python_submit": t_sub * 1e3, "python_flush": t_flush * 1e3, "python_poll_wait": t_poll * 1e3,
                   "python_other": (st.wall_s - t_sub - t_flush - t_poll) * 1e3,
                   "library_submit": lib.host_submit_ms, "library_flush_plan_launch": lib.host_flush_ms,
                   "library_flush_cuda_calls": lib.host_launch_ms, "library_flush_planning": lib.host_plan_ms,
                   "library_reap": lib.host_reap_ms,
                   "device_h2d": lib.h2d_ms, "device_kernels": lib.device_ms, "device_d2h": lib.d2h_ms,
                   "flushes": float(lib.flushes)}
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
    """Feeds every read chunk by chunk up to max_events (or its end) and
    records each read's trajectory.  Up to in_flight reads are admitted at a
    time and advance together: one submit_chunks, one flush and one
    poll_chunks per round.  Reads are not stopped early, so every threshold
    can be studied on the same trajectories."""
    loop = ServingLoop(aligner, reads, chunk=chunk, max_events=max_events)
    h = aligner.h
    n = len(loop.reads)
    out = [Trajectory(rd.read_id, rd.on_target, getattr(rd, "true_cand", -1)) for rd in loop.reads]
    pos = np.zeros(n, np.int64)
    todo = list(range(n))
    live = []
    while todo or live:
        while todo and len(live) < in_flight:
            live.append(todo.pop(0))
        q = np.array(live, np.int64)
        ch = loop._chunks(q, pos[q], False)
        tickets, status = B.rawalign_dtw_submit_chunks(h, ch, loop.events, loop.cands)
        if np.any((status != B.RA_OK) & (status != B.RA_EAGAIN)):
            raise B.RawAlignError("rawalign_dtw_submit_chunks", int(status[status != B.RA_OK][0]))
        ok = status == B.RA_OK
        if not ok.any():
            raise RuntimeError("no read admitted: too few serving slots or too little arena memory")
        B.rawalign_dtw_flush(h)
        res, counts = B.rawalign_dtw_poll_chunks(h, tickets[ok], int(loop.n_cand[q[ok]].sum()))
        at = 0
        qs = q[ok]
        pos[qs] += ch["n_events"][ok].astype(np.int64)
        for x, k in zip(qs.tolist(), counts.tolist()):
            r = res[at:at + k]
            at += k
            tr = out[x]
            sc = r["score"].astype(np.float64)
            b = int(np.argmax(sc)) if len(sc) else -1
            tr.events.append(int(pos[x]))
            tr.best_score.append(float(sc[b]) if b >= 0 else -np.inf)
            tr.best_cand.append(b)
            tr.min_cost.append(float(r["cost"].min()) if len(r) else np.inf)
            tr.mapped.append(bool(len(r) and np.any(r["decision"] == B.RA_MAPPED)))
        # finished reads leave; refused ones stay and retry their first chunk
        done = set(qs[pos[qs] >= loop.n_ev[qs]].tolist())
        live = [x for x in live if x not in done]
    return out


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
