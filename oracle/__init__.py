"""FP64 CPU oracle for the elastic distances of arXiv 2102.05221 (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s cpu_baseline / reference legs, never by the product path.
It shares no code with the CUDA library: its C source (``eap_oracle.c``) is
compiled here with the host C compiler, and this wrapper passes it numpy
arrays through ctypes.

Functions mirror the plain definitions (see ``eap_oracle.c`` for citations):
``distance`` (Eq. Common + each distance's equations), ``eapruned``
(Algorithm 5 with its cell counter), ``nn1`` (Algorithm 1), ``nn1_eapruned``
(Algorithm 1 calling Algorithm 5 with the best-so-far as cut-off), ``pairwise``
(full matrix) and ``lb_keogh`` (textbook LB_Keogh).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eap_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

KINDS = {"dtw": 0, "cdtw": 1, "wdtw": 2, "erp": 3, "msm": 4, "twe": 5}
COST_SQ, COST_ABS = 0, 1
DEFAULT_COST = {"dtw": COST_SQ, "cdtw": COST_SQ, "wdtw": COST_SQ,
                "erp": COST_ABS, "msm": COST_ABS, "twe": COST_ABS}


class OrcParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cost", ctypes.c_int32),
                ("window", ctypes.c_int32), ("derivative", ctypes.c_int32),
                ("window_ratio", ctypes.c_double),
                ("wdtw_g", ctypes.c_double), ("wdtw_wmax", ctypes.c_double),
                ("erp_gap", ctypes.c_double), ("msm_c", ctypes.c_double),
                ("twe_nu", ctypes.c_double), ("twe_lambda", ctypes.c_double)]


def make_params(kind: str, cost=None, window: int = -1, window_ratio: float = -1.0,
                wdtw_g: float = 0.05, wdtw_wmax: float = 1.0, erp_gap: float = 0.0,
                msm_c: float = 0.5, twe_nu: float = 0.001, twe_lambda: float = 1.0,
                derivative: int = 0) -> OrcParams:
    """Oracle parameter block.  ``window_ratio`` is widened from float32 so that
    w = floor(r * max(L_S, L_T)) sees the same r as a float32 caller."""
    k = kind.lower()
    return OrcParams(KINDS[k], DEFAULT_COST[k] if cost is None else int(cost), int(window), int(derivative),
                     float(np.float32(window_ratio)) if window_ratio >= 0 else -1.0,
                     float(np.float32(wdtw_g)), float(np.float32(wdtw_wmax)),
                     float(np.float32(erp_gap)), float(np.float32(msm_c)),
                     float(np.float32(twe_nu)), float(np.float32(twe_lambda)))


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no CUDA involved)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            f32p, f64p = P(ctypes.c_float), P(ctypes.c_double)
            i64p, i32p = P(ctypes.c_int64), P(ctypes.c_int32)
            lib.orc_distance.restype = ctypes.c_double
            lib.orc_distance.argtypes = [P(OrcParams), f32p, ctypes.c_int, f32p, ctypes.c_int]
            lib.orc_eapruned.restype = ctypes.c_double
            lib.orc_eapruned.argtypes = [P(OrcParams), f32p, ctypes.c_int, f32p, ctypes.c_int,
                                         ctypes.c_double, i64p]
            lib.orc_eabase.restype = ctypes.c_double
            lib.orc_eabase.argtypes = [P(OrcParams), f32p, ctypes.c_int, f32p, ctypes.c_int,
                                       ctypes.c_double, i64p]
            lib.orc_subseq.restype = ctypes.c_int
            lib.orc_subseq.argtypes = [P(OrcParams), f32p, ctypes.c_int64, f32p, ctypes.c_int, i64p, f64p,
                                       ctypes.c_int]
            lib.orc_nn1.restype = ctypes.c_int
            lib.orc_nn1.argtypes = [P(OrcParams), f32p, i64p, i32p, ctypes.c_int,
                                    f32p, i64p, i32p, ctypes.c_int, i32p, f64p, ctypes.c_int]
            lib.orc_nn1_eapruned.restype = ctypes.c_int
            lib.orc_nn1_eapruned.argtypes = [P(OrcParams), f32p, i64p, i32p, ctypes.c_int,
                                             f32p, i64p, i32p, ctypes.c_int, i32p, f64p, i64p]
            lib.orc_pairwise.restype = ctypes.c_int
            lib.orc_pairwise.argtypes = [P(OrcParams), f32p, i64p, i32p, ctypes.c_int, f64p, ctypes.c_int]
            lib.orc_cross.restype = ctypes.c_int
            lib.orc_cross.argtypes = [P(OrcParams), f32p, i64p, i32p, ctypes.c_int,
                                      f32p, i64p, i32p, ctypes.c_int, f64p, ctypes.c_int]
            lib.orc_envelope.restype = None
            lib.orc_envelope.argtypes = [f32p, ctypes.c_int, ctypes.c_long, f64p, f64p]
            lib.orc_lb_keogh.restype = ctypes.c_double
            lib.orc_lb_keogh.argtypes = [f32p, f32p, ctypes.c_int, ctypes.c_long, ctypes.c_int]
            _lib = lib
    return _lib


def _f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def distance(params: OrcParams, s, t) -> float:
    """D(S,T) by the full cost-matrix definition (FP64)."""
    s, t = _f32(s), _f32(t)
    return _load().orc_distance(ctypes.byref(params), _ptr(s, ctypes.c_float), len(s),
                                _ptr(t, ctypes.c_float), len(t))


def eapruned(params: OrcParams, s, t, cutoff: float):
    """Algorithm 5: returns (D or +inf, number of computed cells)."""
    s, t = _f32(s), _f32(t)
    cells = ctypes.c_int64(0)
    d = _load().orc_eapruned(ctypes.byref(params), _ptr(s, ctypes.c_float), len(s),
                             _ptr(t, ctypes.c_float), len(t), float(cutoff), ctypes.byref(cells))
    return d, int(cells.value)


def eabase(params: OrcParams, s, t, cutoff: float):
    """Algorithm 4 (EABase): returns (D, or +inf if abandoned on a row
    minimum above the cut-off; number of computed cells)."""
    s, t = _f32(s), _f32(t)
    cells = ctypes.c_int64(0)
    d = _load().orc_eabase(ctypes.byref(params), _ptr(s, ctypes.c_float), len(s),
                           _ptr(t, ctypes.c_float), len(t), float(cutoff), ctypes.byref(cells))
    return d, int(cells.value)


def subseq(params: OrcParams, T, q, nthreads: int | None = None):
    """Sub-sequence search (Section 5.3): (position, distance) of the window
    of T closest to q, both z-normalised; (-1, inf) if q is longer than T."""
    T, q = _f32(T), _f32(q)
    pos = ctypes.c_int64(-1)
    dist = ctypes.c_double(0.0)
    rc = _load().orc_subseq(ctypes.byref(params), _ptr(T, ctypes.c_float), len(T), _ptr(q, ctypes.c_float),
                            len(q), ctypes.byref(pos), ctypes.byref(dist), nthreads or os.cpu_count() or 1)
    if rc != 0:
        raise ValueError("orc_subseq: invalid arguments")
    return int(pos.value), float(dist.value)


def _packed_args(p):
    data = _f32(p.data)
    off = np.ascontiguousarray(p.offsets, dtype=np.int64)
    ln = np.ascontiguousarray(p.lengths, dtype=np.int32)
    return data, off, ln


def nn1(params: OrcParams, queries, refs, nthreads: int | None = None):
    """Algorithm 1 for every query of a packed set: (idx int32[nq], dist float64[nq])."""
    qd, qo, ql = _packed_args(queries)
    rd, ro, rl = _packed_args(refs)
    nq = len(ql)
    idx = np.zeros(nq, dtype=np.int32)
    dist = np.zeros(nq, dtype=np.float64)
    nt = nthreads or os.cpu_count() or 1
    _load().orc_nn1(ctypes.byref(params), _ptr(qd, ctypes.c_float), _ptr(qo, ctypes.c_int64),
                    _ptr(ql, ctypes.c_int32), nq, _ptr(rd, ctypes.c_float), _ptr(ro, ctypes.c_int64),
                    _ptr(rl, ctypes.c_int32), len(rl), _ptr(idx, ctypes.c_int32),
                    _ptr(dist, ctypes.c_double), int(nt))
    return idx, dist


def nn1_eapruned(params: OrcParams, queries, refs):
    """Algorithm 1 with Algorithm 5 as the distance (cut-off = best so far),
    one thread, candidates in index order: (idx int32[nq], dist float64[nq],
    computed cells)."""
    qd, qo, ql = _packed_args(queries)
    rd, ro, rl = _packed_args(refs)
    nq = len(ql)
    idx = np.zeros(nq, dtype=np.int32)
    dist = np.zeros(nq, dtype=np.float64)
    cells = ctypes.c_int64(0)
    _load().orc_nn1_eapruned(ctypes.byref(params), _ptr(qd, ctypes.c_float), _ptr(qo, ctypes.c_int64),
                             _ptr(ql, ctypes.c_int32), nq, _ptr(rd, ctypes.c_float), _ptr(ro, ctypes.c_int64),
                             _ptr(rl, ctypes.c_int32), len(rl), _ptr(idx, ctypes.c_int32),
                             _ptr(dist, ctypes.c_double), ctypes.byref(cells))
    return idx, dist, int(cells.value)


def pairwise(params: OrcParams, series, nthreads: int | None = None) -> np.ndarray:
    """Full n x n matrix of D(set_i, set_j) (FP64)."""
    d, o, l = _packed_args(series)
    n = len(l)
    out = np.zeros((n, n), dtype=np.float64)
    nt = nthreads or os.cpu_count() or 1
    _load().orc_pairwise(ctypes.byref(params), _ptr(d, ctypes.c_float), _ptr(o, ctypes.c_int64),
                         _ptr(l, ctypes.c_int32), n, _ptr(out, ctypes.c_double), int(nt))
    return out


def cross(params: OrcParams, a, b, nthreads: int | None = None) -> np.ndarray:
    """Matrix of D(a_i, b_j) for packed sets a (rows) and b (columns), FP64."""
    ad, ao, al = _packed_args(a)
    bd, bo, bl = _packed_args(b)
    out = np.zeros((len(al), len(bl)), dtype=np.float64)
    nt = nthreads or os.cpu_count() or 1
    _load().orc_cross(ctypes.byref(params), _ptr(ad, ctypes.c_float), _ptr(ao, ctypes.c_int64),
                      _ptr(al, ctypes.c_int32), len(al), _ptr(bd, ctypes.c_float), _ptr(bo, ctypes.c_int64),
                      _ptr(bl, ctypes.c_int32), len(bl), _ptr(out, ctypes.c_double), int(nt))
    return out


def envelope(q, w: int):
    q = _f32(q)
    U = np.zeros(len(q)); Lo = np.zeros(len(q))
    _load().orc_envelope(_ptr(q, ctypes.c_float), len(q), int(w), _ptr(U, ctypes.c_double),
                         _ptr(Lo, ctypes.c_double))
    return U, Lo


def lb_keogh(q, c, w: int, cost: int = COST_SQ) -> float:
    q, c = _f32(q), _f32(c)
    assert len(q) == len(c)
    return _load().orc_lb_keogh(_ptr(q, ctypes.c_float), _ptr(c, ctypes.c_float), len(q), int(w), int(cost))
