"""CPU oracle for the RawAlign DTW path (arXiv 2310.05037) -- test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and shares no code with it.

The arithmetic lives in ``rawalign_oracle.c`` (plain C, single-threaded,
``-O2 -ffp-contract=off``, no fast-math); this module only compiles it and
marshals numpy arrays through ctypes.

Functions and the passages they follow:
  expected_signal     Sup. A.1.1 (k-mer model -> expected event values)
  band_params/in_band Sec. 2.4.3 (band around a line of slope read/ref length)
  dtw_f32/dtw_f64     Sec. 2.2  (DTW recurrence over N, NW, W; corner cell)
  brute_f32/brute_f64 Sec. 2.2  (same cost as a minimum over warping paths)
  score_f32/score_f64 Sec. 2.3  (Score = B_Match * N_Read - C_DTW)
  map_batch           Sec. 2.3 + Sec. 3.1 (best candidate, threshold decision)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rawalign_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

END_GLOBAL = 0
END_FREE = 1
UNMAPPED, MAPPED, PENDING = 0, 1, 2

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rawalign_oracle.h"))
    ):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Band(C.Structure):
    _fields_ = [("unbanded", C.c_int), ("num", C.c_int64), ("den", C.c_int64), ("w_eff", C.c_int64)]


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
        ("cost64", C.c_double),
        ("score64", C.c_double),
    ]


class Anchor(C.Structure):
    _fields_ = [("q", C.c_uint32), ("t", C.c_uint32), ("len", C.c_uint32)]


ANCHOR_DTYPE = np.dtype([("q", "<u4"), ("t", "<u4"), ("len", "<u4")])


RESULT_DTYPE = np.dtype(
    {
        "names": [f[0] for f in Result._fields_],
        "formats": ["<u8", "<u4", "<f4", "<f4", "<i4", "<i4", "<i4", "<u8", "<i4", "<i4", "<i4", "<i4", "<f8", "<f8"],
        "offsets": [getattr(Result, f[0]).offset for f in Result._fields_],
        "itemsize": C.sizeof(Result),
    }
)


def _P(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            i64, u64, f32, f64 = C.c_int64, C.c_uint64, C.c_float, C.c_double
            pf, pd, pu8 = C.POINTER(C.c_float), C.POINTER(C.c_double), C.POINTER(C.c_uint8)
            L.ora_kmer_index.restype = i64
            L.ora_kmer_index.argtypes = [pu8, C.c_int]
            L.ora_expected_signal.restype = i64
            L.ora_expected_signal.argtypes = [pu8, i64, C.c_int, pf, pf]
            L.ora_segment_codes.restype = C.c_int
            L.ora_segment_codes.argtypes = [pu8, u64, u64, u64, C.c_int, pu8]
            L.ora_band_params.restype = C.c_int
            L.ora_band_params.argtypes = [i64, i64, i64, i64, i64, C.POINTER(Band)]
            L.ora_in_band.restype = C.c_int
            L.ora_in_band.argtypes = [C.POINTER(Band), i64, i64]
            L.ora_band_cells.restype = u64
            L.ora_band_cells.argtypes = [C.POINTER(Band), i64, i64]
            pi64, pu64 = C.POINTER(i64), C.POINTER(u64)
            L.ora_dtw_f32.restype = C.c_int
            L.ora_dtw_f32.argtypes = [pf, i64, pf, i64, i64, i64, i64, C.c_int, pf, pi64, pi64, pu64, pi64, pf]
            L.ora_dtw_f64.restype = C.c_int
            L.ora_dtw_f64.argtypes = [pd, i64, pd, i64, i64, i64, i64, C.c_int, pd, pi64, pi64, pu64, pi64, pd]
            L.ora_brute_f32.restype = C.c_int
            L.ora_brute_f32.argtypes = [pf, i64, pf, i64, i64, i64, i64, C.c_int, pf, pi64, pu64]
            L.ora_brute_f64.restype = C.c_int
            L.ora_brute_f64.argtypes = [pd, i64, pd, i64, i64, i64, i64, C.c_int, pd, pi64, pu64]
            L.ora_score_f32.restype = f32
            L.ora_score_f32.argtypes = [f32, i64, f32]
            L.ora_score_f64.restype = f64
            L.ora_score_f64.argtypes = [f64, i64, f64]
            pa = C.POINTER(Anchor)
            L.ora_anchored_f32.restype = C.c_int
            L.ora_anchored_f32.argtypes = [pf, i64, pf, i64, pa, i64, i64, pf, pu64]
            L.ora_anchored_f64.restype = C.c_int
            L.ora_anchored_f64.argtypes = [pd, i64, pd, i64, pa, i64, i64, pd, pu64]
            L.ora_anchored_brute.restype = C.c_int
            L.ora_anchored_brute.argtypes = [pd, i64, pd, i64, pa, i64, pd]
            L.ora_map_anchored.restype = C.c_int
            L.ora_map_anchored.argtypes = [
                C.c_int, f32, f32, pf, pu8, u64, pf, pu64, C.c_uint32,
                C.POINTER(Candidate), C.c_uint32, pa, pu64, C.POINTER(Result), C.c_int,
            ]
            pi32 = C.POINTER(C.c_int32)
            L.ora_traceback_f32.restype = C.c_int
            L.ora_traceback_f32.argtypes = [pf, i64, pf, i64, i64, i64, i64, C.c_int, pi32, pi32, i64, pi64, pf]
            L.ora_map_batch.restype = C.c_int
            L.ora_map_batch.argtypes = [
                C.c_int, f32, f32, C.c_int, pf, pu8, u64, pf, pu64, C.c_uint32,
                C.POINTER(Candidate), C.c_uint32, C.POINTER(Result), C.c_int,
            ]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def kmer_index(codes, k):
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    return int(lib().ora_kmer_index(_P(c, C.c_uint8), k))


def expected_signal(codes, k, pore):
    """r[j] = pore[idx(codes[j..j+k-1])] (Sup. A.1.1)."""
    c = np.ascontiguousarray(codes, dtype=np.uint8)
    p = _f32(pore)
    m = max(len(c) - k + 1, 0)
    out = np.empty(max(m, 1), np.float32)
    got = lib().ora_expected_signal(_P(c, C.c_uint8), len(c), k, _P(p, C.c_float), _P(out, C.c_float))
    return out[:got]


def segment_codes(ref2bit, ref_len, off, length, strand):
    ref = np.ascontiguousarray(ref2bit, dtype=np.uint8)
    out = np.empty(max(int(length), 1), np.uint8)
    rc = lib().ora_segment_codes(_P(ref, C.c_uint8), int(ref_len), int(off), int(length), int(strand), _P(out, C.c_uint8))
    if rc != 0:
        raise ValueError("segment outside the reference")
    return out[: int(length)]


def band_params(n, m, band_w, num=0, den=0):
    b = Band()
    rc = lib().ora_band_params(n, m, band_w, num, den, C.byref(b))
    if rc != 0:
        raise ValueError("invalid band parameters")
    return b


def in_band(b, i, j):
    return bool(lib().ora_in_band(C.byref(b), i, j))


def band_cells(b, n, m):
    return int(lib().ora_band_cells(C.byref(b), n, m))


def dtw_f32(e, r, band_w=-1, num=0, den=0, end_mode=END_GLOBAL, full=False):
    """Returns (cost, end_i, end_j, cells, w_eff[, D matrix])."""
    e = _f32(e)
    r = _f32(r)
    n, m = len(e), len(r)
    cost = C.c_float()
    ei, ej, we = C.c_int64(), C.c_int64(), C.c_int64()
    cells = C.c_uint64()
    D = np.empty((n, m), np.float32) if full else None
    rc = lib().ora_dtw_f32(
        _P(e, C.c_float), n, _P(r, C.c_float), m, band_w, num, den, end_mode,
        C.byref(cost), C.byref(ei), C.byref(ej), C.byref(cells), C.byref(we),
        _P(D, C.c_float) if full else None,
    )
    if rc != 0:
        raise ValueError("oracle rejected the input (%d)" % rc)
    out = (np.float32(cost.value), ei.value, ej.value, cells.value, we.value)
    return out + (D,) if full else out


def dtw_f64(e, r, band_w=-1, num=0, den=0, end_mode=END_GLOBAL, full=False):
    e = _f64(e)
    r = _f64(r)
    n, m = len(e), len(r)
    cost = C.c_double()
    ei, ej, we = C.c_int64(), C.c_int64(), C.c_int64()
    cells = C.c_uint64()
    D = np.empty((n, m), np.float64) if full else None
    rc = lib().ora_dtw_f64(
        _P(e, C.c_double), n, _P(r, C.c_double), m, band_w, num, den, end_mode,
        C.byref(cost), C.byref(ei), C.byref(ej), C.byref(cells), C.byref(we),
        _P(D, C.c_double) if full else None,
    )
    if rc != 0:
        raise ValueError("oracle rejected the input (%d)" % rc)
    out = (cost.value, ei.value, ej.value, cells.value, we.value)
    return out + (D,) if full else out


def brute_f32(e, r, band_w=-1, num=0, den=0, end_mode=END_GLOBAL):
    """Minimum over warping paths, FP32 accumulation from the start: (cost, end_j, paths)."""
    e = _f32(e)
    r = _f32(r)
    cost = C.c_float()
    ej = C.c_int64()
    paths = C.c_uint64()
    rc = lib().ora_brute_f32(_P(e, C.c_float), len(e), _P(r, C.c_float), len(r), band_w, num, den, end_mode,
                             C.byref(cost), C.byref(ej), C.byref(paths))
    if rc != 0:
        raise ValueError("brute force is limited to tiny inputs")
    return np.float32(cost.value), ej.value, paths.value


def brute_f64(e, r, band_w=-1, num=0, den=0, end_mode=END_GLOBAL):
    e = _f64(e)
    r = _f64(r)
    cost = C.c_double()
    ej = C.c_int64()
    paths = C.c_uint64()
    rc = lib().ora_brute_f64(_P(e, C.c_double), len(e), _P(r, C.c_double), len(r), band_w, num, den, end_mode,
                             C.byref(cost), C.byref(ej), C.byref(paths))
    if rc != 0:
        raise ValueError("brute force is limited to tiny inputs")
    return cost.value, ej.value, paths.value


def score_f32(b_match, n_read, cost):
    return np.float32(lib().ora_score_f32(float(np.float32(b_match)), int(n_read), float(np.float32(cost))))


def score_f64(b_match, n_read, cost):
    return lib().ora_score_f64(float(b_match), int(n_read), float(cost))


def map_batch(k, b_match, score_threshold, end_mode, pore, ref2bit, ref_len, events, read_offsets, cands,
              use_f64=False):
    """Whole-path oracle for a batch (same record layout as the library).

    ``cands`` is a numpy structured array with the candidate layout; returns a
    structured array of results (RESULT_DTYPE).  Raises ValueError on inputs
    the path must reject.
    """
    pore = _f32(pore)
    ref = np.ascontiguousarray(ref2bit, dtype=np.uint8)
    ev = _f32(events)
    offs = np.ascontiguousarray(read_offsets, dtype=np.uint64)
    cands = np.ascontiguousarray(cands)
    assert cands.dtype.itemsize == C.sizeof(Candidate)
    n_reads = len(offs) - 1
    out = np.zeros(len(cands), RESULT_DTYPE)
    rc = lib().ora_map_batch(
        int(k), float(np.float32(b_match)), float(np.float32(score_threshold)), int(end_mode),
        _P(pore, C.c_float), _P(ref, C.c_uint8), int(ref_len), _P(ev, C.c_float), _P(offs, C.c_uint64),
        n_reads, cands.ctypes.data_as(C.POINTER(Candidate)), len(cands),
        out.ctypes.data_as(C.POINTER(Result)), 1 if use_f64 else 0,
    )
    if rc != 0:
        raise ValueError("oracle rejected the batch (%d)" % rc)
    return out


def _anchors(anchors):
    a = np.ascontiguousarray(np.asarray(anchors, dtype=ANCHOR_DTYPE) if not isinstance(anchors, np.ndarray)
                             or anchors.dtype != ANCHOR_DTYPE else anchors)
    return a


def anchored_f32(e, r, anchors, band_w=-1):
    """Anchor-guided cost (Sec. 2.4.2), FP32: (cost, cells).  anchors: sequence
    of (q, t, len) or an ANCHOR_DTYPE array."""
    e, r, a = _f32(e), _f32(r), _anchors(anchors)
    cost = C.c_float()
    cells = C.c_uint64()
    rc = lib().ora_anchored_f32(_P(e, C.c_float), len(e), _P(r, C.c_float), len(r),
                                a.ctypes.data_as(C.POINTER(Anchor)), len(a), band_w, C.byref(cost), C.byref(cells))
    if rc != 0:
        raise ValueError("oracle rejected the anchors (%d)" % rc)
    return np.float32(cost.value), cells.value


def anchored_f64(e, r, anchors, band_w=-1):
    e, r, a = _f64(e), _f64(r), _anchors(anchors)
    cost = C.c_double()
    cells = C.c_uint64()
    rc = lib().ora_anchored_f64(_P(e, C.c_double), len(e), _P(r, C.c_double), len(r),
                                a.ctypes.data_as(C.POINTER(Anchor)), len(a), band_w, C.byref(cost), C.byref(cells))
    if rc != 0:
        raise ValueError("oracle rejected the anchors (%d)" % rc)
    return cost.value, cells.value


def anchored_brute(e, r, anchors):
    """Minimum path sum (FP64) over N/W/NW paths that stay in the gap rectangles,
    one-sided gap lines and anchor diagonals; tiny tables only."""
    e, r, a = _f64(e), _f64(r), _anchors(anchors)
    cost = C.c_double()
    rc = lib().ora_anchored_brute(_P(e, C.c_double), len(e), _P(r, C.c_double), len(r),
                                  a.ctypes.data_as(C.POINTER(Anchor)), len(a), C.byref(cost))
    if rc != 0:
        raise ValueError("brute force is limited to tiny inputs with valid anchors")
    return cost.value


def map_anchored(k, b_match, score_threshold, pore, ref2bit, ref_len, events, read_offsets, cands, anchors,
                 anchor_offsets, use_f64=False):
    """Whole-path oracle for a batch in anchor-guided mode (GLOBAL ends)."""
    pore = _f32(pore)
    ref = np.ascontiguousarray(ref2bit, dtype=np.uint8)
    ev = _f32(events)
    offs = np.ascontiguousarray(read_offsets, dtype=np.uint64)
    cands = np.ascontiguousarray(cands)
    a = _anchors(anchors)
    aoffs = np.ascontiguousarray(anchor_offsets, dtype=np.uint64)
    assert len(aoffs) == len(cands) + 1
    out = np.zeros(len(cands), RESULT_DTYPE)
    rc = lib().ora_map_anchored(
        int(k), float(np.float32(b_match)), float(np.float32(score_threshold)),
        _P(pore, C.c_float), _P(ref, C.c_uint8), int(ref_len), _P(ev, C.c_float), _P(offs, C.c_uint64),
        len(offs) - 1, cands.ctypes.data_as(C.POINTER(Candidate)), len(cands),
        a.ctypes.data_as(C.POINTER(Anchor)), _P(aoffs, C.c_uint64),
        out.ctypes.data_as(C.POINTER(Result)), 1 if use_f64 else 0,
    )
    if rc != 0:
        raise ValueError("oracle rejected the batch (%d)" % rc)
    return out


def traceback_f32(e, r, band_w=-1, num=0, den=0, end_mode=END_GLOBAL):
    """Optimal warping path (ties: NW, then N, then W) from (0,0) to the end
    cell: (cost, path as an (L, 2) int array of (i, j)); empty when no
    in-band path reaches the end."""
    e, r = _f32(e), _f32(r)
    n, m = len(e), len(r)
    cap = n + m - 1
    pi = np.zeros(cap, np.int32)
    pj = np.zeros(cap, np.int32)
    ln = C.c_int64()
    cost = C.c_float()
    rc = lib().ora_traceback_f32(_P(e, C.c_float), n, _P(r, C.c_float), m, band_w, num, den, end_mode,
                                 _P(pi, C.c_int32), _P(pj, C.c_int32), cap, C.byref(ln), C.byref(cost))
    if rc != 0:
        raise ValueError("oracle rejected the input (%d)" % rc)
    return np.float32(cost.value), np.stack([pi[: ln.value], pj[: ln.value]], axis=1)
