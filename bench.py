"""Benchmark of the RawAlign DTW alignment path on GB300.

One step = one pass of the whole path over one batch: by default the
batched-uneven workload (20k reads with lognormal event counts, 1-8
candidate regions each on a 100 Mb reference, band 10 % of the span);
--workload readuntil | longread | plain picks another full-size batch.  The
path is expected signal, band, DTW, end cell, score and per-read decision,
all in the library's kernels (replays of the captured CUDA graphs).  Inputs are resident in HBM when the timed region starts and
are larger than L2; L2 is also flushed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload batched|readuntil|longread|plain]

Prints one JSON line (rank 0).  value = in-band DTW cells / device time
(GCUPS, whole job over all ranks).  e2e = the same metric through the public
submit/poll calls from pinned host buffers (copies included).  Extra keys:
reads_per_s, the plain one-alignment-per-launch kernel on a sample of the same
workload, the batched/plain speed-up, the Read-Until serving loop, and
"workloads": the Read-Until prefix, long-read and anchor-guided batches at
full size, each with device GCUPS, its fraction of the roofline and its
end-to-end rate (--extra picks them).  --impl reference times the CPU oracle
(the only reference this path has) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "batched": ("batched_uneven: %d reads, lognormal event counts (median 1500, 200-8000), 1-8 candidates "
                "per read (1 true + decoys) on a 100 Mb uniform-ACGT reference, span = events x U(0.9,1.3), "
                "band 10%% of span, 6-mer pore table N(0,1), noise sd 0.3, 5%% skips, FP32 global DTW"),
    "readuntil": ("readuntil_prefix: 100000 reads x first 450 events, 16-64 candidates per read on a 3 Gb "
                  "uniform-ACGT reference with 2% of its 5 kb blocks duplicated at 90% identity, band 64, "
                  "FP32 global DTW"),
    "longread": ("longread_banded: 2000 reads of 20k-100k events (uniform), 2 candidates each on a 100 Mb "
                 "reference, band 5% of span, 5% skips + 5% stays, noise sd 0.4, FP32 global DTW"),
    "batched_et": ("batched_uneven_early_termination: the batched-uneven workload (%d reads) with each read's "
                   "true locus first among its candidates (as chaining-score order puts it) and branch-and-bound "
                   "early termination on: the others stop once they cannot beat the read's best score; GCUPS "
                   "counts the cells computed"),
    "anchored": ("anchored_batched: the batched-uneven shapes (20000 reads, 1-8 candidates, band 10% of span) "
                 "with anchor-guided alignment: each candidate's chain (true locus: runs of one event per k-mer "
                 "from the simulated read, 8-16 events; decoys: 0-6 random anchors), gaps aligned by banded DTW"),
    "plain": ("plain: 64 reads x 500 events, 1 candidate each (true 550-value segment of a 20 kb reference), "
              "unbanded FP32 DTW"),
}
METRIC = "DTW GCUPS and reads/s (batched and served vs plain per-alignment kernel); p50/p99 chunk latency"
OPS_PER_CELL = 4  # sub, min, min, add per DP cell
# ALU-pipe lane-slots per in-band cell of the striped kernel's hot loop: the
# 3-input min (issued at half rate: 2 slots), the select of the row's event
# by the band mask with its share of the mask-to-predicate moves (1.15), the
# per-column work spread over the lane's 24 rows (about 0.35) and the stripe
# changes (about 0.1); the subtraction and the addition go to the FMA pipe.
ALU_SLOTS_PER_CELL = 3.6
# DRAM bytes (read + write) of the DTW part of one step of a workload, from an
# ncu capture of the current kernel (None: not captured for this kernel).
TRAFFIC = {"batched": 907394816}
TRAFFIC_BASIS = ("dram__bytes_read.sum + dram__bytes_write.sum of the striped kernel's 8 launches of one step of "
                 "the full 20k-read batch (ncu, one pass per launch, averaged over 5 replays); algorithmic bytes "
                 "per step are about 190 MB (events once, 2-bit reference once, 32 B per alignment)")


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.p = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="rawalign_clocks_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()
        self.rows = self._read()
        if self.path:
            try:
                os.unlink(self.path)
            except OSError:
                pass

    def _read(self):
        rows = []
        if not self.p or not self.path:
            return rows
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[4], f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        return rows

    def summary(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in load:
            for nm, v in zip(names, r[4:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(load), "power_w_max": pmax}


def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if n_gpus > 0 else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _all_reduce(x, world, op_name):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x, world):
    return _all_reduce(x, world, "MAX")


def sum_over_ranks(x, world):
    return _all_reduce(x, world, "SUM")


def cpu_baseline(w, seconds=15.0, seed=1):
    """The oracle, as it stands, single-threaded on the host: a random sample
    of the workload's alignments, about `seconds` of CPU work."""
    import oracle as O

    rng = np.random.default_rng(seed)
    order = rng.permutation(w.n_cands)
    cells = 0
    done = 0
    t0 = time.perf_counter()
    chunk = 16
    pos = 0
    while time.perf_counter() - t0 < seconds and pos < len(order):
        sub = w.subset(np.sort(order[pos : pos + chunk]))
        pos += chunk
        if sub.anchor_offsets is not None:
            res = O.map_anchored(sub.k, sub.b_match, sub.score_threshold, sub.pore, sub.ref2bit, sub.ref_len,
                                 sub.events, sub.read_offsets, sub.cands, sub.anchors, sub.anchor_offsets)
        else:
            res = O.map_batch(sub.k, sub.b_match, sub.score_threshold, sub.end_mode, sub.pore, sub.ref2bit,
                              sub.ref_len, sub.events, sub.read_offsets, sub.cands)
        cells += int(res["cells"].sum())
        done += len(res)
    el = time.perf_counter() - t0
    return {"value": cells / el / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": "%d random alignments of the workload (%.3g in-band cells) in %.1f s, single thread"
                      % (done, cells, el), "seconds": el}


def host_cpu():
    """Model name and online cores of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"cpu_model": model or platform.processor() or platform.machine(), "machine": platform.machine(),
            "nproc": os.cpu_count()}


def workload_name(args, name=None):
    name = name or args.workload
    d = WORKLOADS[name]
    return d % args.reads if name in ("batched", "batched_et") else d


def make_workload(S, args, rank, name=None):
    """The step's batch; every rank draws its own (weak scaling, replicas)."""
    name = name or args.workload
    if name in ("batched", "batched_et"):
        return S.config_batched(n_reads=args.reads, seed=0x5EED0002 + rank, true_first=name == "batched_et")
    if name == "longread" and args.longread_reads != 2000:
        return S.config_longread(n_reads=args.longread_reads, seed=0x5EED0005 + rank)
    return S.scaled(name, "full", seed=None if rank == 0 else 0x5EED1000 + rank)


def arena_bytes(B, w):
    """The prepared batch and two submissions in flight, plus ring scratch
    for bands too wide for shared-memory rings."""
    m_total = int(np.sum(w.cands["ref_len_bases"].astype(np.int64) - w.k + 1))
    need = B.rawalign_dtw_batch_bytes(len(w.events), w.n_reads, w.n_cands, m_total)
    arena = 3 * need + len(w.ref2bit) + (256 << 20)
    if w.anchor_offsets is not None:  # per-gap work items and results, pieces
        arena += 3 * (len(w.anchors) + w.n_cands) * 512
    m_c = w.cands["ref_len_bases"].astype(np.int64) - w.k + 1
    w_c = np.where(w.cands["band_w"] < 0, m_c, w.cands["band_w"].astype(np.int64))
    if w.n_cands and int(np.max(2 * w_c + 1)) > 2000:
        arena += 3 * (2 << 30)
    return arena, m_total


def prepare(al, w):
    if w.anchor_offsets is not None:
        return al.prepare_anchored(w.events, w.read_offsets, w.cands, w.anchors, w.anchor_offsets)
    return al.prepare(w.events, w.read_offsets, w.cands)


def time_resident(torch, al, batch, w, steps, warmup, flush, clk_ctx=None):
    """Replays of the prepared batch (inputs resident in HBM), CUDA events on
    the library's stream around each step, L2 flushed before each step.
    Returns per-step results, device times and the DTW part's times."""
    stream = al.stream
    res = None
    for _ in range(warmup):
        res = al.poll(al.run(batch), w.n_cands)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    dtw_ms, tot_ms = [], []
    torch.cuda.synchronize()
    with (clk_ctx if clk_ctx is not None else _Null()):
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                ev0[i].record(stream)
            t = al.run(batch)
            with torch.cuda.stream(stream):
                ev1[i].record(stream)
            al.poll(t, 0)
            dtw_ms.append(al.stats(batch).dtw_ms)
            tot_ms.append(ev0[i].elapsed_time(ev1[i]))
        torch.cuda.synchronize()
    return res, tot_ms, dtw_ms


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def time_e2e(B, torch, al, w, steps, world):
    """The same cells through the public submit/poll calls from pinned host
    buffers: inputs copied in and results copied out (into one pinned buffer)
    every step, two submissions in flight (step i+1 planned and uploaded while
    step i runs)."""
    from paper_2310_05037_gb300 import synth as S

    anchored = w.anchor_offsets is not None
    ev_np = torch.from_numpy(w.events).pin_memory().numpy()
    off_np = torch.from_numpy(w.read_offsets.view(np.int64)).pin_memory().numpy().view(np.uint64)
    cand_np = torch.from_numpy(w.cands.view(np.uint8)).pin_memory().numpy().view(S.CANDIDATE_DTYPE)
    # results come back into one pinned buffer, reused every step
    res_np = torch.empty(w.n_cands * B.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory().numpy().view(
        B.RESULT_DTYPE)

    def submit():
        if anchored:
            return B.rawalign_dtw_submit_anchored(al.h, ev_np, off_np, cand_np, w.anchors, w.anchor_offsets)
        return B.rawalign_dtw_submit_batch(al.h, ev_np, off_np, cand_np)

    def pipelined(k):
        t = submit()
        r = None
        for i in range(k):
            t_next = submit() if i + 1 < k else None
            r = B.rawalign_dtw_poll(al.h, t, w.n_cands, out=res_np)
            t = t_next
        return r

    # the host part of one submission, from a batch prepared the same way
    # (after the handle's first prepare, which also allocates its staging)
    bp = (al.prepare_anchored(ev_np, off_np, cand_np, w.anchors, w.anchor_offsets) if anchored
          else al.prepare(ev_np, off_np, cand_np))
    al.poll(al.run(bp), 0)
    host = prepare_split(al.stats(bp))
    al.release(bp)
    pipelined(2)
    barrier(world)
    t0 = time.perf_counter()
    r = pipelined(steps)
    el = max_over_ranks(time.perf_counter() - t0, world)
    cells = sum_over_ranks(float(r["cells"].sum()) * steps, world)
    return {"value": round(cells / el / 1e9, 2), "unit": "GCUPS",
            "h2d_bytes_per_step": int(w.events.nbytes + w.read_offsets.nbytes + w.cands.nbytes +
                                      (w.anchors.nbytes + w.anchor_offsets.nbytes if anchored else 0)),
            "d2h_bytes_per_step": int(w.n_cands * B.RESULT_DTYPE.itemsize),
            "ms_per_step": round(el / steps * 1e3, 2),
            "pipelining": "two submissions in flight (submit i+1, then poll i)",
            "host_buffers": "pinned inputs and one pinned result buffer reused every step",
            "host_prepare_ms": host}


def prepare_split(st):
    """Host time of one prepare of a step's batch (the work each end-to-end
    submission repeats): planning on the library's threads, then the uploads."""
    return {"plan": round(st.host_plan_ms, 2), "upload": round(st.host_upload_ms, 2)}


def peak_gcups(torch, local):
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    return sms, f_max, sms * 128 * f_max * 1e6 / OPS_PER_CELL / 1e9


def pipe_bound_gcups(sms, f_mhz):
    """Bound of the ALU pipe for the striped kernel's instruction mix:
    SMs x 64 ALU lanes per clock x f / ALU lane-slots per cell."""
    return sms * 64 * f_mhz * 1e6 / ALU_SLOTS_PER_CELL / 1e9


def measure_extra(B, S, torch, args, name, local, flush, peak):
    """One more full-size workload: device GCUPS of resident replays, the DTW
    part's fraction of the roofline, and end to end through submit/poll."""
    t0 = time.perf_counter()
    w = make_workload(S, args, 0, name)
    gen_s = time.perf_counter() - t0
    arena, m_total = arena_bytes(B, w)
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena, device="cuda:%d" % local)
    try:
        batch = prepare(al, w)
        steps = max(3, min(args.steps, 5))
        res, tot_ms, dtw_ms = time_resident(torch, al, batch, w, steps, 3, flush)
        cells = int(res["cells"].sum())
        step_ms = sum(tot_ms) / len(tot_ms)
        dtw_avg = sum(dtw_ms) / len(dtw_ms)
        launches = al.stats(batch).launches
        al.release(batch)
        e2e = time_e2e(B, torch, al, w, max(3, args.steps), 1) if not args.no_e2e else None
    finally:
        al.close()
        del al
        torch.cuda.empty_cache()
    dtw_gcups = cells / (dtw_avg / 1e3) / 1e9
    out = {"workload": workload_name(args, name), "alignments": w.n_cands, "reads": w.n_reads,
           "cells_per_step": cells, "value": round(cells / (step_ms / 1e3) / 1e9, 2), "unit": "GCUPS",
           "ms_per_step": round(step_ms, 3), "dtw_kernel_ms": round(dtw_avg, 3),
           "dtw_gcups": round(dtw_gcups, 2), "frac": round(dtw_gcups / peak, 4),
           "steps": steps, "warmup": 3, "gpu_launches_per_step": int(launches),
           "reads_per_s": round(w.n_reads / (step_ms / 1e3), 1), "generate_s": round(gen_s, 1)}
    if e2e:
        out["e2e"] = e2e
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(WORKLOADS))
    ap.add_argument("--reads", type=int, default=20000, help="reads of the batched workload")
    ap.add_argument("--longread-reads", type=int, default=2000, help="reads of the long-read workload")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--extra", default="readuntil,longread,anchored",
                    help="other full-size workloads measured after the headline one (comma list, or none)")
    ap.add_argument("--serve-chunks", type=int, default=30000)
    ap.add_argument("--serve-realtime-s", type=float, default=6.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    from paper_2310_05037_gb300 import synth as S

    if args.impl == "reference":
        return run_reference(args, S)

    world, rank, local = dist_init(args.gpus)
    import torch

    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2310_05037_gb300 import binding as B

    w = make_workload(S, args, rank)
    arena, m_total = arena_bytes(B, w)
    al = B.Aligner(w.pore, w.ref2bit, w.ref_len, arena_bytes=arena, device="cuda:%d" % local,
                   early_termination=args.workload == "batched_et")
    anchored = w.anchor_offsets is not None
    batch = prepare(al, w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda:%d" % local)

    barrier(world)
    clk = ClockSampler(local)
    res, tot_ms, dtw_ms = time_resident(torch, al, batch, w, args.steps, args.warmup, flush, clk)
    barrier(world)
    cells_step = int(res["cells"].sum())
    pruned_step = int(np.sum(res["status"] == B.RA_RESULT_PRUNED))
    reads_step = w.n_reads
    launches_step = al.stats(batch).launches
    clocks = clk.summary()
    step_ms = sum(tot_ms) / len(tot_ms)
    total_s = max_over_ranks(sum(tot_ms) / 1e3, world)
    total_cells = sum_over_ranks(cells_step * args.steps, world)
    value = total_cells / total_s / 1e9
    dtw_avg_ms = sum(dtw_ms) / len(dtw_ms)

    sms, f_max, peak = peak_gcups(torch, local)
    achieved = cells_step / (dtw_avg_ms / 1e3) / 1e9
    pipe = pipe_bound_gcups(sms, f_max)
    roofline = {
        "bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "GCUPS",
        "frac": round(achieved / peak, 4), "traffic": TRAFFIC.get(args.workload) if args.reads == 20000 else None,
        "kernel": "dtw_stripe_kernel", "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz / %d ops per cell "
        "(derived, MEASURED_PEAKS sm_max_mhz)" % (sms, f_max, OPS_PER_CELL),
        "pipe_bound": {"gcups": round(pipe, 1), "frac": round(achieved / pipe, 4),
                       "alu_slots_per_cell": ALU_SLOTS_PER_CELL,
                       "basis": "%d SMs x 64 ALU lanes per clock x %.0f MHz / ALU lane-slots per cell of the "
                                "kernel's instruction mix (3-input min at half rate)" % (sms, f_max)},
    }
    if roofline["traffic"] is not None:
        roofline["traffic_per_cell_bytes"] = round(roofline["traffic"] / cells_step, 5)
        roofline["traffic_basis"] = TRAFFIC_BASIS
    if clocks.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = round(achieved / (peak * clocks["sm_mhz"] / f_max), 4)

    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args), "reads": w.n_reads, "alignments": w.n_cands,
                   "cells_per_step": cells_step,
                   "l2": "inputs larger than L2 (expected signal %.0f MB, events %.0f MB) and a 256 MB L2 flush "
                         "between timed steps" % (m_total * 4 / 1e6, len(w.events) * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "reads_per_s": round(sum_over_ranks(reads_step * args.steps, world) / total_s, 1),
        "pruned_alignments_per_step": pruned_step,
        "dtw_kernel_ms": round(dtw_avg_ms, 3),
        "gpu_launches": int(launches_step * args.steps),
        "roofline": roofline, "clocks": clocks,
    }

    # plain one-alignment-per-launch kernel on a sample of the same workload
    if not args.no_plain and rank == 0:
        # a random sample of the workload's alignments: at most 300, and no
        # more than about 1e9 table cells (seconds for the plain kernel)
        rng = np.random.default_rng(5)
        perm = rng.permutation(w.n_cands)[:300]
        nn = w.read_lengths()[w.cands["read_id"][perm].astype(np.int64)]
        mm = w.cands["ref_len_bases"][perm].astype(np.int64) - w.k + 1
        keep = max(1, int(np.searchsorted(np.cumsum(nn * mm), 1e9)))
        sub = w.subset(np.sort(perm[:keep]))
        alp = B.Aligner(sub.pore, sub.ref2bit, sub.ref_len, arena_bytes=1 << 30, kernel=B.RA_KERNEL_PLAIN,
                        device="cuda:%d" % local)
        if anchored:
            bp = alp.prepare_anchored(sub.events, sub.read_offsets, sub.cands, sub.anchors, sub.anchor_offsets)
        else:
            bp = alp.prepare(sub.events, sub.read_offsets, sub.cands)
        tp = alp.run(bp)
        rp = alp.poll(tp, sub.n_cands)
        tp = alp.run(bp)
        alp.poll(tp, 0)
        stp = alp.stats(bp)
        plain_gcups = float(rp["cells"].sum()) / (stp.dtw_ms / 1e3) / 1e9
        alp.release(bp)
        alp.close()
        out["plain_kernel"] = {"gcups": round(plain_gcups, 3), "sample_alignments": sub.n_cands,
                               "launches": int(stp.launches)}
        out["speedup_vs_plain"] = round(achieved / plain_gcups, 1)

    # end to end through submit/poll with pinned host buffers
    if not args.no_e2e:
        out["e2e"] = time_e2e(B, torch, al, w, max(3, args.steps), world)
    al.release(batch)
    al.close()
    del al
    torch.cuda.empty_cache()

    # Read-Until serving: 512 reads in flight, 180-event chunks, <= 4000 events
    if not args.no_serve and rank == 0:
        from paper_2310_05037_gb300.serving import ServingLoop

        # 4 disjoint sets of 4096 reads from one generator: a full-size
        # warm-up loop, then three measured loops (median by GCUPS; all three
        # are reported)
        pore_s, ref_s, rl_s, sreads_all = S.config_serving(n_reads=4 * 4096)
        sets = [sreads_all[i * 4096:(i + 1) * 4096] for i in range(4)]
        sreads = sets[0]
        als = B.Aligner(pore_s, ref_s, rl_s, arena_bytes=(len(ref_s) + (1536 << 20)), serve_slots=1024,
                        serve_max_events=4000, max_candidates=32, device="cuda:%d" % local,
                        serve_early_reject=True)
        ServingLoop(als, sets[3]).run(max_chunks=args.serve_chunks, in_flight=512)  # warm-up
        reps = [ServingLoop(als, sets[i]).run(max_chunks=args.serve_chunks, in_flight=512).summary()
                for i in range(3)]
        closed = dict(sorted(reps, key=lambda x: x["gcups"])[1])
        closed["repeats_gcups"] = [round(x["gcups"], 1) for x in reps]
        rt = ServingLoop(als, sreads[::-1]).run(max_chunks=10 ** 9, in_flight=512, realtime=True, chunk_s=0.4,
                                                 duration_s=args.serve_realtime_s, arrival_rate=1280.0).summary()
        from paper_2310_05037_gb300.serving import collect_trajectories, decision_study

        als.close()
        # decision policy (Sec. 3.1) on reads whose loci have near-duplicates:
        # 2 % of the reference's 20 kb blocks copied at 98 % identity (as
        # segmental duplications), 25 % of the reads from a copied block with
        # the copy among their candidates; event noise sd 0.3 to 0.5
        study = {}
        for sd in (0.3, 0.4, 0.5):
            pore_d, ref_d, rl_d, dreads = S.config_serving(seed=0x5EED0040, n_reads=512, noise_sd=sd, dup_frac=0.02,
                                                           repeat_reads=0.25, ident=0.98, block=20000)
            ald = B.Aligner(pore_d, ref_d, rl_d, arena_bytes=len(ref_d) + (1 << 30), serve_slots=512,
                            serve_max_events=4000, max_candidates=32, device="cuda:%d" % local)
            try:
                trs = collect_trajectories(ald, dreads, chunk=180, max_events=4000, in_flight=512)
            finally:
                ald.close()
            study["noise_sd_%.2f" % sd] = decision_study(trs, [10.0, 20.0, 30.0, 40.0, 60.0], max_events=4000)
        out["served"] = {"closed_loop": closed, "realtime": rt,
                         "decision_study": {"reads": 512, "by_noise_and_threshold": study,
                                            "workload": "512 reads per noise level, 2% of 20 kb blocks copied at 98% "
                                                        "identity, 25% of reads from a copied block with its copy "
                                                        "among the candidates, 50% off-target"},
                         "workload": "Read-Until serving: Poisson stream, 512 reads in flight, 180-event chunks, "
                                     "<= 4000 events, 1-32 candidates, band 64, FREE end, 50% off-target reads",
                         "loop": "closed loop, median of 3 runs on disjoint 4096-read sets after a full warm-up run: "
                                 "two generations of 256 reads, one submit_chunks + flush + "
                                 "poll_chunks per generation; reads stop at the library's decision (MAPPED, or "
                                 "UNMAPPED once no candidate can reach the threshold within 4000 events)"}
        out["speedup_served_vs_plain"] = (round(closed["gcups"] / out["plain_kernel"]["gcups"], 1)
                                          if "plain_kernel" in out else None)

    # the other full-size batch workloads, each measured the same way
    extra = [x for x in args.extra.split(",") if x and x != "none" and x != args.workload]
    if extra and rank == 0:
        out["workloads"] = {}
        for name in extra:
            out["workloads"][name] = measure_extra(B, S, torch, args, name, local, flush, peak)

    if not args.no_cpu and rank == 0 and world >= 1:
        cb = cpu_baseline(w, seconds=args.cpu_seconds)
        cb["cores"] = 1
        cb.update(host_cpu())
        out["cpu_baseline"] = {k: v for k, v in cb.items() if k != "seconds"}

    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def run_reference(args, S):
    """The reference arm: the CPU oracle on bounded samples of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = make_workload(S, args, 0)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup):
        cpu_baseline(w, seconds=per_step, seed=100 + i)
    vals, secs, samples = [], [], []
    for i in range(args.steps):
        cb = cpu_baseline(w, seconds=per_step, seed=200 + i)
        vals.append(cb["value"])
        secs.append(cb["seconds"])
        samples.append(cb["sample"])
    value = statistics.mean(vals)
    config = {"workload": workload_name(args), "reads": w.n_reads, "alignments": w.n_cands}
    if w.anchor_offsets is None:
        # the in-band cells of the whole workload: the oracle's band (slope
        # num/den, half-width w_eff) gives each row the columns j with
        # |j den - i num| <= w_eff den, clipped to the table
        import oracle as O

        lens = w.read_lengths()
        rid = w.cands["read_id"].astype(np.int64)
        total = 0
        for c in range(w.n_cands):
            n, m = int(lens[rid[c]]), int(w.cands["ref_len_bases"][c]) - w.k + 1
            b = O.band_params(n, m, int(w.cands["band_w"][c]), int(w.cands["slope_num"][c]),
                              int(w.cands["slope_den"][c]))
            if b.unbanded:
                total += n * m
                continue
            i = np.arange(n, dtype=np.int64)
            lo = np.maximum(-((b.w_eff * b.den - i * b.num) // b.den), 0)
            hi = np.minimum((i * b.num + b.w_eff * b.den) // b.den, m - 1)
            total += int(np.maximum(hi - lo + 1, 0).sum())
        config["cells_per_step"] = total
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(secs), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {**host_cpu(), "value": round(value, 5), "unit": "GCUPS", "cores": 1, "kind": "oracle",
                         "sample": "each step: random alignments of the workload for %.1f s, single thread; "
                                   "last: %s" % (per_step, samples[-1])},
        "e2e": {"value": round(value, 5), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
