"""ctypes binding of librawalign_dtw (include/rawalign_dtw.h).

Argument marshalling only: every step of the alignment path runs in the
library's CUDA kernels.  PyTorch supplies the device arena and the stream.
The binding fails loudly if the shared library is missing; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .synth import ANCHOR_DTYPE, CANDIDATE_DTYPE

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librawalign_dtw.so")

RA_OK, RA_EINVAL, RA_ENOMEM, RA_EAGAIN, RA_ENOTREADY, RA_ETIMEDOUT, RA_EDEVICE = 0, -1, -2, -3, -4, -5, -6
RA_END_GLOBAL, RA_END_FREE = 0, 1
RA_UNMAPPED, RA_MAPPED, RA_PENDING = 0, 1, 2
RA_RESULT_PRUNED = 1
RA_KERNEL_AUTO, RA_KERNEL_PLAIN, RA_KERNEL_SPLIT = 0, 1, 2
RA_KERNEL_VARIANT0 = 16
VARIANTS = [(32, 16), (16, 16), (32, 8), (16, 8), (8, 8), (4, 8), (16, 24), (8, 24), (32, 24), (4, 24)]
RA_KERNEL_STRIPE = {gh: RA_KERNEL_VARIANT0 + v for v, gh in enumerate(VARIANTS)}

STATUS_NAMES = {0: "RA_OK", -1: "RA_EINVAL", -2: "RA_ENOMEM", -3: "RA_EAGAIN", -4: "RA_ENOTREADY",
                -5: "RA_ETIMEDOUT", -6: "RA_EDEVICE"}


class RawAlignError(RuntimeError):
    def __init__(self, call, code):
        super().__init__("%s failed: %s (%d)" % (call, STATUS_NAMES.get(code, "?"), code))
        self.code = code


class Config(C.Structure):
    _fields_ = [
        ("k", C.c_int32),
        ("b_match", C.c_float),
        ("score_threshold", C.c_float),
        ("end_mode", C.c_int32),
        ("arena_dev", C.c_void_p),
        ("arena_bytes", C.c_uint64),
        ("cuda_stream", C.c_void_p),
        ("max_candidates", C.c_int32),
        ("kernel", C.c_int32),
        ("serve_slots", C.c_int32),
        ("serve_max_events", C.c_int32),
        ("autotune_path", C.c_char_p),
        ("early_termination", C.c_int32),
        ("serve_early_reject", C.c_int32),
        ("test_stall_handoff", C.c_int32),
        ("pad", C.c_int32),
    ]


class Candidate(C.Structure):
    _fields_ = [
        ("read_id", C.c_uint64),
        ("ref_offset", C.c_uint64),
        ("ref_len_bases", C.c_uint32),
        ("strand", C.c_uint8),
        ("pad0", C.c_uint8 * 3),
        ("band_w", C.c_int32),
        ("pad1", C.c_int32),
        ("slope_num", C.c_int64),
        ("slope_den", C.c_int64),
    ]


class Result(C.Structure):
    _fields_ = [
        ("read_id", C.c_uint64),
        ("cand_idx", C.c_uint32),
        ("cost", C.c_float),
        ("score", C.c_float),
        ("end_i", C.c_int32),
        ("end_j", C.c_int32),
        ("w_eff", C.c_int32),
        ("cells", C.c_uint64),
        ("status", C.c_int32),
        ("is_best", C.c_int32),
        ("decision", C.c_int32),
        ("pad", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("dtw_ms", C.c_double),
        ("total_ms", C.c_double),
        ("cells", C.c_uint64),
        ("slots", C.c_uint64),
        ("launches", C.c_uint32),
        ("split", C.c_uint32),
        ("host_plan_ms", C.c_double),
        ("host_upload_ms", C.c_double),
    ]


class ServeStats(C.Structure):
    _fields_ = [
        ("flushes", C.c_uint64),
        ("chunks", C.c_uint64),
        ("pieces", C.c_uint64),
        ("cells", C.c_uint64),
        ("host_submit_ms", C.c_double),
        ("host_flush_ms", C.c_double),
        ("h2d_ms", C.c_double),
        ("device_ms", C.c_double),
        ("d2h_ms", C.c_double),
        ("host_launch_ms", C.c_double),
        ("host_plan_ms", C.c_double),
        ("host_reap_ms", C.c_double),
    ]


CHUNK_DTYPE = np.dtype(
    {
        "names": ["read_id", "ev_offset", "n_events", "cand_offset", "n_cands", "last"],
        "formats": ["<u8", "<u8", "<u4", "<u4", "<u4", "<i4"],
        "offsets": [0, 8, 16, 20, 24, 28],
        "itemsize": 32,
    }
)

RESULT_DTYPE = np.dtype(
    {
        "names": [f[0] for f in Result._fields_],
        "formats": ["<u8", "<u4", "<f4", "<f4", "<i4", "<i4", "<i4", "<u8", "<i4", "<i4", "<i4", "<i4"],
        "offsets": [getattr(Result, f[0]).offset for f in Result._fields_],
        "itemsize": C.sizeof(Result),
    }
)

# symbol -> (restype, argtypes)
_u64p = C.POINTER(C.c_uint64)
SIGNATURES = {
    "rawalign_dtw_create": (C.c_int, [C.POINTER(Config), C.c_void_p, C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p)]),
    "rawalign_dtw_submit_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, _u64p]),
    "rawalign_dtw_submit_chunk": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_int, _u64p]),
    "rawalign_dtw_flush": (C.c_int, [C.c_void_p]),
    "rawalign_dtw_submit_chunks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]),
    "rawalign_dtw_poll_chunks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p,
                                           C.c_int64]),
    "rawalign_dtw_serve_stats": (C.c_int, [C.c_void_p, C.POINTER(ServeStats), C.c_int]),
    "rawalign_dtw_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.c_int64]),
    "rawalign_dtw_prepare_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, _u64p]),
    "rawalign_dtw_prepare_anchored": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                                C.c_uint32, C.c_void_p, C.c_void_p, _u64p]),
    "rawalign_dtw_submit_anchored": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                               C.c_uint32, C.c_void_p, C.c_void_p, _u64p]),
    "rawalign_dtw_traceback": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_int32, C.c_void_p,
                                         C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.c_void_p]),
    "rawalign_dtw_run_batch": (C.c_int, [C.c_void_p, C.c_uint64, _u64p]),
    "rawalign_dtw_release_batch": (C.c_int, [C.c_void_p, C.c_uint64]),
    "rawalign_dtw_destroy": (C.c_int, [C.c_void_p]),
    "rawalign_dtw_batch_stats": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Stats)]),
    "rawalign_dtw_batch_bytes": (C.c_uint64, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64]),
    "rawalign_dtw_set_variant_costs": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_uint32]),
    "rawalign_dtw_align_noalloc": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_int32, C.c_int64,
                                             C.c_int64, C.c_int32, C.c_float, C.c_void_p, C.c_void_p]),
}

_lib = None


def load(path: str | None = None):
    """Loads the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("librawalign_dtw.so is missing (%s): run __graft_entry__.build()" % p)
        L = C.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(call, code):
    if code != RA_OK:
        raise RawAlignError(call, code)


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else C.c_void_p(0)


# ---- the ABI, one Python function per entry point (same names) -------------

def rawalign_dtw_create(config: Config, pore: np.ndarray, ref2bit: np.ndarray, ref_len: int) -> C.c_void_p:
    pore = np.ascontiguousarray(pore, np.float32)
    ref = np.ascontiguousarray(ref2bit, np.uint8)
    h = C.c_void_p()
    _check("rawalign_dtw_create", load().rawalign_dtw_create(C.byref(config), _ptr(pore), _ptr(ref), int(ref_len), C.byref(h)))
    return h


def _batch_args(events, read_offsets, cands):
    ev = np.ascontiguousarray(events, np.float32)
    offs = np.ascontiguousarray(read_offsets, np.uint64)
    cands = np.ascontiguousarray(cands)
    if cands.dtype != CANDIDATE_DTYPE:
        raise TypeError("candidates must use CANDIDATE_DTYPE")
    return ev, offs, cands


def rawalign_dtw_submit_batch(h, events, read_offsets, cands) -> int:
    ev, offs, cands = _batch_args(events, read_offsets, cands)
    t = C.c_uint64()
    _check("rawalign_dtw_submit_batch", load().rawalign_dtw_submit_batch(
        h, _ptr(ev), _ptr(offs), len(offs) - 1, _ptr(cands), len(cands), C.byref(t)))
    return t.value


def rawalign_dtw_prepare_batch(h, events, read_offsets, cands) -> int:
    ev, offs, cands = _batch_args(events, read_offsets, cands)
    b = C.c_uint64()
    _check("rawalign_dtw_prepare_batch", load().rawalign_dtw_prepare_batch(
        h, _ptr(ev), _ptr(offs), len(offs) - 1, _ptr(cands), len(cands), C.byref(b)))
    return b.value


def _anchor_args(anchors, anchor_offsets, n_cands):
    aoffs = np.ascontiguousarray(anchor_offsets, np.uint64)
    if len(aoffs) != n_cands + 1:
        raise ValueError("anchor_offsets needs n_cands + 1 entries")
    a = np.ascontiguousarray(anchors if anchors is not None else np.zeros(0, ANCHOR_DTYPE))
    if a.dtype != ANCHOR_DTYPE:
        a = np.ascontiguousarray(np.asarray(a, dtype=ANCHOR_DTYPE))
    return a, aoffs


def rawalign_dtw_prepare_anchored(h, events, read_offsets, cands, anchors, anchor_offsets) -> int:
    ev, offs, cands = _batch_args(events, read_offsets, cands)
    a, aoffs = _anchor_args(anchors, anchor_offsets, len(cands))
    b = C.c_uint64()
    _check("rawalign_dtw_prepare_anchored", load().rawalign_dtw_prepare_anchored(
        h, _ptr(ev), _ptr(offs), len(offs) - 1, _ptr(cands), len(cands), _ptr(a) if len(a) else None, _ptr(aoffs),
        C.byref(b)))
    return b.value


def rawalign_dtw_submit_anchored(h, events, read_offsets, cands, anchors, anchor_offsets) -> int:
    ev, offs, cands = _batch_args(events, read_offsets, cands)
    a, aoffs = _anchor_args(anchors, anchor_offsets, len(cands))
    t = C.c_uint64()
    _check("rawalign_dtw_submit_anchored", load().rawalign_dtw_submit_anchored(
        h, _ptr(ev), _ptr(offs), len(offs) - 1, _ptr(cands), len(cands), _ptr(a) if len(a) else None, _ptr(aoffs),
        C.byref(t)))
    return t.value


def rawalign_dtw_traceback(h, events, cand, end_mode=RA_END_GLOBAL, k=6):
    """(result record, path as an (L, 2) int32 array of (i, j) from (0,0))."""
    ev = np.ascontiguousarray(events, np.float32)
    cd = np.ascontiguousarray(np.asarray(cand).reshape(1))
    if cd.dtype != CANDIDATE_DTYPE:
        raise TypeError("the candidate must use CANDIDATE_DTYPE")
    m = int(cd["ref_len_bases"][0]) - k + 1
    cap = max(len(ev) + max(m, 1) - 1, 1)
    pi = np.zeros(cap, np.int32)
    pj = np.zeros(cap, np.int32)
    ln = C.c_uint32()
    res = np.zeros(1, RESULT_DTYPE)
    _check("rawalign_dtw_traceback", load().rawalign_dtw_traceback(
        h, _ptr(ev), len(ev), _ptr(cd), int(end_mode), _ptr(pi), _ptr(pj), cap, C.byref(ln), _ptr(res)))
    return res[0], np.stack([pi[: ln.value], pj[: ln.value]], axis=1)


def rawalign_dtw_run_batch(h, batch: int) -> int:
    t = C.c_uint64()
    _check("rawalign_dtw_run_batch", load().rawalign_dtw_run_batch(h, batch, C.byref(t)))
    return t.value


def rawalign_dtw_release_batch(h, batch: int) -> None:
    _check("rawalign_dtw_release_batch", load().rawalign_dtw_release_batch(h, batch))


def rawalign_dtw_submit_chunk(h, read_id: int, events, cands=None, last: bool = False) -> int:
    ev = np.ascontiguousarray(events, np.float32)
    t = C.c_uint64()
    if cands is not None:
        cands = np.ascontiguousarray(cands)
        cp, nc = _ptr(cands), len(cands)
    else:
        cp, nc = C.c_void_p(0), 0
    code = load().rawalign_dtw_submit_chunk(h, int(read_id), _ptr(ev), len(ev), cp, nc, 1 if last else 0, C.byref(t))
    _check("rawalign_dtw_submit_chunk", code)
    return t.value


def rawalign_dtw_flush(h) -> None:
    _check("rawalign_dtw_flush", load().rawalign_dtw_flush(h))


def rawalign_dtw_submit_chunks(h, chunks, events, cands):
    """chunks: CHUNK_DTYPE array; events / cands: the arrays the chunks index.
    Returns (tickets uint64 array, status int32 array)."""
    ch = np.ascontiguousarray(chunks)
    if ch.dtype != CHUNK_DTYPE:
        raise TypeError("chunks must use CHUNK_DTYPE")
    ev = np.ascontiguousarray(events, np.float32)
    cd = np.ascontiguousarray(cands)
    if cd.dtype != CANDIDATE_DTYPE:
        raise TypeError("candidates must use CANDIDATE_DTYPE")
    tickets = np.zeros(len(ch), np.uint64)
    status = np.zeros(len(ch), np.int32)
    _check("rawalign_dtw_submit_chunks", load().rawalign_dtw_submit_chunks(
        h, _ptr(ch), len(ch), _ptr(ev), _ptr(cd), _ptr(tickets), _ptr(status)))
    return tickets, status


def rawalign_dtw_poll_chunks(h, tickets, cap: int, timeout_us: int = -1, out=None):
    """Results of every ticket, back to back, and the count per ticket; None
    while RA_ENOTREADY.  out: optional contiguous RESULT_DTYPE array of at
    least cap records, reused across calls; the results are then a view of it."""
    t = np.ascontiguousarray(tickets, np.uint64)
    if out is None:
        out = np.zeros(max(int(cap), 1), RESULT_DTYPE)
    elif out.dtype != RESULT_DTYPE or not out.flags.c_contiguous or len(out) < cap:
        raise TypeError("out must be a contiguous RESULT_DTYPE array of at least cap records")
    counts = np.zeros(len(t), np.uint32)
    code = load().rawalign_dtw_poll_chunks(h, _ptr(t), len(t), _ptr(out), int(cap), _ptr(counts), int(timeout_us))
    if code == RA_ENOTREADY:
        return None
    _check("rawalign_dtw_poll_chunks", code)
    return out[: int(counts.sum())], counts


def rawalign_dtw_serve_stats(h, reset: bool = False) -> ServeStats:
    s = ServeStats()
    _check("rawalign_dtw_serve_stats", load().rawalign_dtw_serve_stats(h, C.byref(s), 1 if reset else 0))
    return s


def rawalign_dtw_poll(h, ticket: int, cap: int, timeout_us: int = -1, out=None):
    """Returns a structured array of results, or None while RA_ENOTREADY.
    out: optional RESULT_DTYPE array of at least cap records to write into
    (e.g. a view of pinned memory reused across calls, so that the results
    come back in one fast copy); the return value is then a view of it."""
    if out is None:
        out = np.zeros(max(cap, 1), RESULT_DTYPE)
    elif out.dtype != RESULT_DTYPE or not out.flags.c_contiguous or len(out) < cap:
        raise TypeError("out must be a contiguous RESULT_DTYPE array of at least cap records")
    n = C.c_uint32()
    code = load().rawalign_dtw_poll(h, int(ticket), _ptr(out), cap, C.byref(n), int(timeout_us))
    if code == RA_ENOTREADY:
        return None
    _check("rawalign_dtw_poll", code)
    return out[: n.value]


def rawalign_dtw_batch_stats(h, batch: int) -> Stats:
    s = Stats()
    _check("rawalign_dtw_batch_stats", load().rawalign_dtw_batch_stats(h, batch, C.byref(s)))
    return s


def rawalign_dtw_set_variant_costs(h, costs) -> None:
    arr = (C.c_double * len(costs))(*[float(c) for c in costs])
    _check("rawalign_dtw_set_variant_costs", load().rawalign_dtw_set_variant_costs(h, arr, len(costs)))


def rawalign_dtw_batch_bytes(n_events, n_reads, n_cands, total_ref_values) -> int:
    return int(load().rawalign_dtw_batch_bytes(int(n_events), int(n_reads), int(n_cands), int(total_ref_values)))


def rawalign_dtw_align_noalloc(d_events: int, n_events: int, d_ref_signal: int, m: int, band_w: int, slope_num: int,
                               slope_den: int, end_mode: int, b_match: float, d_result: int, stream: int) -> int:
    """Device pointers in (ints); returns the status code (RA_OK when queued)."""
    return int(load().rawalign_dtw_align_noalloc(C.c_void_p(d_events), n_events, C.c_void_p(d_ref_signal), m, band_w,
                                                 slope_num, slope_den, end_mode, b_match, C.c_void_p(d_result),
                                                 C.c_void_p(stream)))


def rawalign_dtw_destroy(h) -> None:
    _check("rawalign_dtw_destroy", load().rawalign_dtw_destroy(h))


# ---- convenience wrapper: arena and stream from torch ------------------------

class Aligner:
    """Owns a handle, its torch-allocated arena and stream.

    >>> al = Aligner(pore, ref2bit, ref_len, arena_bytes=1 << 30)
    >>> res = al.align(events, read_offsets, cands)
    """

    def __init__(self, pore, ref2bit, ref_len, arena_bytes=1 << 30, k=6, b_match=0.4, score_threshold=20.0,
                 end_mode=RA_END_GLOBAL, kernel=RA_KERNEL_AUTO, stream=None, serve_slots=0,
                 serve_max_events=0, max_candidates=64, device="cuda:0", autotune_path=None,
                 early_termination=False, serve_early_reject=False, test_stall_handoff=False):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        cfg = Config()
        cfg.k = k
        cfg.b_match = b_match
        cfg.score_threshold = score_threshold
        cfg.end_mode = end_mode
        cfg.arena_dev = self.arena.data_ptr()
        cfg.arena_bytes = int(arena_bytes)
        cfg.cuda_stream = self.stream.cuda_stream
        cfg.max_candidates = max_candidates
        cfg.kernel = kernel
        cfg.serve_slots = serve_slots
        cfg.serve_max_events = serve_max_events
        cfg.early_termination = 1 if early_termination else 0
        cfg.serve_early_reject = 1 if serve_early_reject else 0
        cfg.test_stall_handoff = 1 if test_stall_handoff else 0
        self._tune_path = autotune_path.encode() if autotune_path else None
        cfg.autotune_path = self._tune_path
        self.cfg = cfg
        self.h = rawalign_dtw_create(cfg, pore, ref2bit, ref_len)

    def align(self, events, read_offsets, cands, timeout_us=-1):
        t = rawalign_dtw_submit_batch(self.h, events, read_offsets, cands)
        return rawalign_dtw_poll(self.h, t, len(cands), timeout_us)

    def prepare(self, events, read_offsets, cands):
        return rawalign_dtw_prepare_batch(self.h, events, read_offsets, cands)

    def align_anchored(self, events, read_offsets, cands, anchors, anchor_offsets, timeout_us=-1):
        t = rawalign_dtw_submit_anchored(self.h, events, read_offsets, cands, anchors, anchor_offsets)
        return rawalign_dtw_poll(self.h, t, len(cands), timeout_us)

    def prepare_anchored(self, events, read_offsets, cands, anchors, anchor_offsets):
        return rawalign_dtw_prepare_anchored(self.h, events, read_offsets, cands, anchors, anchor_offsets)

    def traceback(self, events, cand, end_mode=RA_END_GLOBAL):
        return rawalign_dtw_traceback(self.h, events, cand, end_mode, k=self.cfg.k)

    def run(self, batch):
        return rawalign_dtw_run_batch(self.h, batch)

    def poll(self, ticket, cap, timeout_us=-1, out=None):
        return rawalign_dtw_poll(self.h, ticket, cap, timeout_us, out)

    def stats(self, batch):
        return rawalign_dtw_batch_stats(self.h, batch)

    def release(self, batch):
        rawalign_dtw_release_batch(self.h, batch)

    def close(self):
        if self.h:
            rawalign_dtw_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
