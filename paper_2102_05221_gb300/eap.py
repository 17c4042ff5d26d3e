"""Thin ctypes binding of libeap's C ABI (include/eap.h), same names.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides device memory and streams.  If libeap.so is not
built, or there is no CUDA device, calls raise instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

EAP_OK, EAP_EINVAL, EAP_ENOMEM, EAP_EAGAIN, EAP_ETIMEOUT, EAP_EDEVICE, EAP_EINTERNAL = 0, -1, -2, -3, -4, -5, -6
KINDS = {"dtw": 0, "cdtw": 1, "wdtw": 2, "erp": 3, "msm": 4, "twe": 5}
KIND_NAMES = {v: k for k, v in KINDS.items()}
EAP_COST_DEFAULT, EAP_COST_SQ, EAP_COST_ABS = -1, 0, 1
EAP_LB_NONE, EAP_LB_KEOGH, EAP_LB_KEOGH2 = 0, 1, 2
EAP_PRUNE_ONLY, EAP_BASE = 0, 1


class EapError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class eap_params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cost", ctypes.c_int32), ("window_ratio", ctypes.c_float),
                ("window", ctypes.c_int32), ("wdtw_g", ctypes.c_float), ("wdtw_wmax", ctypes.c_float),
                ("erp_gap", ctypes.c_float), ("msm_c", ctypes.c_float), ("twe_nu", ctypes.c_float),
                ("twe_lambda", ctypes.c_float), ("lb", ctypes.c_int32), ("prune", ctypes.c_int32),
                ("derivative", ctypes.c_int32)]


class eap_series_set(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("lengths", ctypes.c_void_p),
                ("h_offsets", ctypes.c_void_p), ("h_lengths", ctypes.c_void_p), ("data_len", ctypes.c_int64),
                ("count", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class eap_plan(ctypes.Structure):
    _fields_ = [("mapping", ctypes.c_int32), ("strip_width", ctypes.c_int32), ("lanes_per_pair", ctypes.c_int32),
                ("band_exact", ctypes.c_int32)]


PLAN_MAPPINGS = {1: "band", 2: "group", 3: "warp", 4: "cta"}


class eap_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("pairs_lb_pruned", ctypes.c_uint64),
                ("pairs_abandoned", ctypes.c_uint64), ("cells_effective", ctypes.c_uint64),
                ("cells_computed", ctypes.c_uint64), ("dp_ms", ctypes.c_double), ("lb_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if k.endswith("_ms") else int(getattr(self, k))) for k, _ in self._fields_}


class eap_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_query_len", ctypes.c_int32), ("device", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libeap.so (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libeap.so is not built ({path}); run paper_2102_05221_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
        lib.eap_params_default.argtypes = [P(eap_params), i32]
        lib.eap_params_default.restype = None
        lib.eap_strerror.argtypes = [ctypes.c_int]
        lib.eap_strerror.restype = ctypes.c_char_p
        lib.eap_version.restype = i32
        lib.eap_nn1.argtypes = [P(eap_params), P(eap_series_set), P(eap_series_set), vp, vp, vp, P(eap_stats)]
        lib.eap_nn1_host.argtypes = [P(eap_params), vp, vp, vp, i32, vp, vp, vp, i32, vp, vp, P(eap_stats)]
        lib.eap_pairwise.argtypes = [P(eap_params), P(eap_series_set), vp, i32, vp, P(eap_stats)]
        lib.eap_pairs.argtypes = [P(eap_params), P(eap_series_set), P(eap_series_set), vp, vp, vp, vp, i32, vp,
                                  P(eap_stats)]
        lib.eap_lb_keogh.argtypes = [P(eap_params), P(eap_series_set), P(eap_series_set), vp, vp, vp, i32, vp]
        lib.eap_nn1_keys.argtypes = [P(eap_params), P(eap_series_set), P(eap_series_set), ctypes.c_int64, vp, vp,
                                     P(eap_stats)]
        lib.eap_keys_unpack.argtypes = [vp, i32, vp, vp, vp]
        lib.eap_lb_matrix.argtypes = [P(eap_params), P(eap_series_set), P(eap_series_set), i32, vp, vp]
        lib.eap_nn1_plan.argtypes = [P(eap_params), i32, i32, i32, i32, P(eap_plan)]
        if hasattr(lib, "eap_serve_create"):
            lib.eap_serve_create.argtypes = [P(eap_serve_config), P(ctypes.c_int)]
            lib.eap_serve_create.restype = vp
            lib.eap_serve_add_refset.argtypes = [vp, vp, vp, vp, i32, P(i32)]
            lib.eap_serve_submit.argtypes = [vp, i32, P(eap_params), vp, i32, P(u64)]
            lib.eap_serve_poll.argtypes = [vp, u64, P(i32), P(ctypes.c_float)]
            lib.eap_serve_drain.argtypes = [vp, i32]
            lib.eap_serve_destroy.argtypes = [vp]
        lib.eap_subseq.argtypes = [P(eap_params), vp, ctypes.c_int64, P(eap_series_set), vp, vp, vp, P(eap_stats)]
        for name in ("eap_nn1", "eap_nn1_host", "eap_pairwise", "eap_pairs", "eap_lb_keogh", "eap_subseq",
                     "eap_nn1_keys", "eap_keys_unpack", "eap_lb_matrix"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load(build_if_missing=False).eap_strerror(int(code)).decode()
    except Exception:
        return f"error {code}"


def _check(rc: int, where: str):
    if rc != EAP_OK:
        raise EapError(rc, where)


def params(kind, **kw) -> eap_params:
    """Parameter block with the distance's defaults, overridden by keywords
    (cost, window_ratio, window, wdtw_g, wdtw_wmax, erp_gap, msm_c, twe_nu,
    twe_lambda, lb, prune, derivative)."""
    k = KINDS[kind] if isinstance(kind, str) else int(kind)
    p = eap_params()
    load().eap_params_default(ctypes.byref(p), k)
    for key, val in kw.items():
        if not hasattr(p, key):
            raise TypeError(f"unknown parameter {key}")
        setattr(p, key, val)
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libeap needs a CUDA device; none is available")
    return torch


class SeriesSet:
    """A packed series set resident on the GPU, with the host mirrors of its
    offsets and lengths that the C ABI asks for."""

    def __init__(self, data, offsets, lengths, device=None):
        torch = _torch()
        dev = torch.device(device or "cuda")
        self.h_offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.h_lengths = np.ascontiguousarray(np.asarray(lengths, dtype=np.int32))
        if isinstance(data, torch.Tensor):
            self.data = data.to(device=dev, dtype=torch.float32).contiguous()
        else:
            self.data = torch.from_numpy(np.ascontiguousarray(np.asarray(data, dtype=np.float32))).to(dev)
        self.offsets = torch.from_numpy(self.h_offsets.copy()).to(dev)
        self.lengths = torch.from_numpy(self.h_lengths.copy()).to(dev)
        self.count = int(self.h_lengths.shape[0])

    @classmethod
    def from_packed(cls, packed, device=None):
        return cls(packed.data, packed.offsets, packed.lengths, device)

    @classmethod
    def from_matrix(cls, x, device=None):
        x = np.asarray(x, dtype=np.float32)
        n, L = x.shape
        return cls(x.reshape(-1), np.arange(n, dtype=np.int64) * L, np.full(n, L, np.int32), device)

    def struct(self) -> eap_series_set:
        s = eap_series_set()
        s.data = self.data.data_ptr() if self.data.numel() else None
        s.offsets = self.offsets.data_ptr() if self.count else None
        s.lengths = self.lengths.data_ptr() if self.count else None
        s.h_offsets = self.h_offsets.ctypes.data if self.count else None
        s.h_lengths = self.h_lengths.ctypes.data if self.count else None
        s.data_len = int(self.data.numel())
        s.count = self.count
        return s


def _stream_ptr(stream):
    torch = _torch()
    st = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(st.cuda_stream)


def eap_nn1(p: eap_params, queries: SeriesSet, refs: SeriesSet, stream=None, with_stats: bool = False,
            out_idx=None, out_dist=None):
    """1-NN of every query among refs: (idx int32 tensor, dist float32 tensor[, stats dict])."""
    torch = _torch()
    lib = load()
    dev = queries.data.device
    idx = out_idx if out_idx is not None else torch.empty(queries.count, dtype=torch.int32, device=dev)
    dist = out_dist if out_dist is not None else torch.empty(queries.count, dtype=torch.float32, device=dev)
    qs, rs = queries.struct(), refs.struct()
    st = eap_stats()
    rc = lib.eap_nn1(ctypes.byref(p), ctypes.byref(qs), ctypes.byref(rs),
                     ctypes.c_void_p(idx.data_ptr() if queries.count else 0),
                     ctypes.c_void_p(dist.data_ptr() if queries.count else 0),
                     _stream_ptr(stream), ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_nn1")
    return (idx, dist, st.as_dict()) if with_stats else (idx, dist)


def eap_nn1_keys(p: eap_params, queries: SeriesSet, refs: SeriesSet, index_offset: int = 0, stream=None,
                 with_stats: bool = False, out_keys=None):
    """1-NN against one candidate shard as packed keys (int64 tensor on the
    device): (D bits << 32) | (local index + index_offset); the element-wise
    minimum over the shards is the 1-NN over their union."""
    torch = _torch()
    lib = load()
    dev = queries.data.device
    keys = out_keys if out_keys is not None else torch.empty(queries.count, dtype=torch.int64, device=dev)
    qs, rs = queries.struct(), refs.struct()
    st = eap_stats()
    rc = lib.eap_nn1_keys(ctypes.byref(p), ctypes.byref(qs), ctypes.byref(rs), int(index_offset),
                          ctypes.c_void_p(keys.data_ptr() if queries.count else 0), _stream_ptr(stream),
                          ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_nn1_keys")
    return (keys, st.as_dict()) if with_stats else keys


def eap_lb_matrix(p: eap_params, queries: SeriesSet, refs: SeriesSet, two_way: bool = True, stream=None):
    """The 1-NN search's lower-bound pass: [queries x refs] float32 tensor of
    max(LB_Keogh(Q, C), LB_Keogh(C, Q)) (first term only without two_way)."""
    torch = _torch()
    lib = load()
    out = torch.empty((queries.count, refs.count), dtype=torch.float32, device=queries.data.device)
    qs, rs = queries.struct(), refs.struct()
    rc = lib.eap_lb_matrix(ctypes.byref(p), ctypes.byref(qs), ctypes.byref(rs), int(bool(two_way)),
                           ctypes.c_void_p(out.data_ptr() if out.numel() else 0), _stream_ptr(stream))
    _check(rc, "eap_lb_matrix")
    return out


def eap_nn1_plan(p: eap_params, n_queries: int, min_len: int, max_query_len: int, max_ref_len: int) -> dict:
    """The kernel mapping and strip width eap_nn1 runs for these sizes: a dict
    with mapping ("band", "group", "warp" or "cta"), strip_width,
    lanes_per_pair and band_exact.  Host only: needs no GPU."""
    lib = load()
    out = eap_plan()
    rc = lib.eap_nn1_plan(ctypes.byref(p), int(n_queries), int(min_len), int(max_query_len), int(max_ref_len),
                          ctypes.byref(out))
    _check(rc, "eap_nn1_plan")
    return {"mapping": PLAN_MAPPINGS[out.mapping], "strip_width": int(out.strip_width),
            "lanes_per_pair": int(out.lanes_per_pair), "band_exact": bool(out.band_exact)}


def eap_keys_unpack(keys, stream=None, out_idx=None, out_dist=None):
    """Keys of eap_nn1_keys to (idx int32, dist float32) device tensors."""
    torch = _torch()
    lib = load()
    n = int(keys.numel())
    idx = out_idx if out_idx is not None else torch.empty(n, dtype=torch.int32, device=keys.device)
    dist = out_dist if out_dist is not None else torch.empty(n, dtype=torch.float32, device=keys.device)
    rc = lib.eap_keys_unpack(ctypes.c_void_p(keys.data_ptr() if n else 0), n,
                             ctypes.c_void_p(idx.data_ptr() if n else 0), ctypes.c_void_p(dist.data_ptr() if n else 0),
                             _stream_ptr(stream))
    _check(rc, "eap_keys_unpack")
    return idx, dist


def eap_nn1_host(p: eap_params, queries, refs, with_stats: bool = False, out_idx=None, out_dist=None):
    """1-NN with host (numpy) packed sets in and host arrays out."""
    lib = load()
    _torch()

    def arrs(x):
        return (np.ascontiguousarray(x.data, dtype=np.float32), np.ascontiguousarray(x.offsets, dtype=np.int64),
                np.ascontiguousarray(x.lengths, dtype=np.int32))

    qd, qo, ql = arrs(queries)
    rd, ro, rl = arrs(refs)
    nq = len(ql)
    idx = out_idx if out_idx is not None else np.empty(nq, dtype=np.int32)
    dist = out_dist if out_dist is not None else np.empty(nq, dtype=np.float32)
    st = eap_stats()

    def ptr(a):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr())
        return ctypes.c_void_p(a.ctypes.data)

    rc = lib.eap_nn1_host(ctypes.byref(p), ptr(qd), ptr(qo), ptr(ql), nq, ptr(rd), ptr(ro), ptr(rl), len(rl),
                          ptr(idx), ptr(dist), ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_nn1_host")
    return (idx, dist, st.as_dict()) if with_stats else (idx, dist)


def eap_pairwise(p: eap_params, series: SeriesSet, mode: int = EAP_PRUNE_ONLY, stream=None, with_stats=False,
                 out=None):
    """Symmetric n x n distance matrix (float32 tensor)."""
    torch = _torch()
    lib = load()
    n = series.count
    m = out if out is not None else torch.empty((n, n), dtype=torch.float32, device=series.data.device)
    s = series.struct()
    st = eap_stats()
    rc = lib.eap_pairwise(ctypes.byref(p), ctypes.byref(s), ctypes.c_void_p(m.data_ptr() if n else 0), int(mode),
                          _stream_ptr(stream), ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_pairwise")
    return (m, st.as_dict()) if with_stats else m


def eap_pairs(p: eap_params, a: SeriesSet, b: SeriesSet, ia, ib, cutoff=None, stream=None, with_stats=False):
    """out[k] = D(a[ia[k]], b[ib[k]]) if <= cutoff[k] else +inf (float32 tensor)."""
    torch = _torch()
    lib = load()
    dev = a.data.device
    ia = torch.as_tensor(ia, dtype=torch.int32, device=dev).contiguous()
    ib = torch.as_tensor(ib, dtype=torch.int32, device=dev).contiguous()
    n = int(ia.numel())
    if cutoff is None:
        cut = torch.full((n,), float("inf"), dtype=torch.float32, device=dev)
    else:
        cut = torch.as_tensor(cutoff, dtype=torch.float32, device=dev).contiguous()
    out = torch.empty(n, dtype=torch.float32, device=dev)
    sa, sb = a.struct(), b.struct()
    st = eap_stats()
    rc = lib.eap_pairs(ctypes.byref(p), ctypes.byref(sa), ctypes.byref(sb), ctypes.c_void_p(ia.data_ptr()),
                       ctypes.c_void_p(ib.data_ptr()), ctypes.c_void_p(cut.data_ptr()),
                       ctypes.c_void_p(out.data_ptr()), n, _stream_ptr(stream),
                       ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_pairs")
    return (out, st.as_dict()) if with_stats else out


def eap_lb_keogh(p: eap_params, a: SeriesSet, b: SeriesSet, ia, ib, stream=None):
    """LB_Keogh(a[ia[k]], b[ib[k]]) for equal-length pairs (float32 tensor)."""
    torch = _torch()
    lib = load()
    dev = a.data.device
    ia = torch.as_tensor(ia, dtype=torch.int32, device=dev).contiguous()
    ib = torch.as_tensor(ib, dtype=torch.int32, device=dev).contiguous()
    n = int(ia.numel())
    out = torch.empty(n, dtype=torch.float32, device=dev)
    sa, sb = a.struct(), b.struct()
    rc = lib.eap_lb_keogh(ctypes.byref(p), ctypes.byref(sa), ctypes.byref(sb), ctypes.c_void_p(ia.data_ptr()),
                          ctypes.c_void_p(ib.data_ptr()), ctypes.c_void_p(out.data_ptr()), n, _stream_ptr(stream))
    _check(rc, "eap_lb_keogh")
    return out


def eap_subseq(p: eap_params, ref, queries: SeriesSet, stream=None, with_stats: bool = False):
    """Sub-sequence search (Section 5.3): for every query, the start position
    of the window of the long series `ref` (a 1-D float32 array or device
    tensor) closest to it under z-normalised DTW / CDTW.  Returns device
    tensors (pos int64, dist float32) [and the stats]."""
    torch = _torch()
    lib = load()
    dev = queries.data.device
    r = ref if isinstance(ref, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32))
    r = r.to(device=dev, dtype=torch.float32).contiguous()
    pos = torch.empty(queries.count, dtype=torch.int64, device=dev)
    dist = torch.empty(queries.count, dtype=torch.float32, device=dev)
    sq = queries.struct()
    st = eap_stats()
    rc = lib.eap_subseq(ctypes.byref(p), ctypes.c_void_p(r.data_ptr() if r.numel() else None), int(r.numel()),
                        ctypes.byref(sq), ctypes.c_void_p(pos.data_ptr() if pos.numel() else None),
                        ctypes.c_void_p(dist.data_ptr() if dist.numel() else None), _stream_ptr(stream),
                        ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_subseq")
    return (pos, dist, st.as_dict()) if with_stats else (pos, dist)


def eap_pairs_noalloc(p: eap_params, a: SeriesSet, b: SeriesSet, ia, ib, cutoff=None, stream=None,
                      with_stats=False, out=None):
    """eap_pairs for callers that cannot allocate device memory during the
    call: the library takes its scratch from a fixed 4 MiB device array
    instead of allocating.  `ia`, `ib`, `cutoff` and `out` must already be
    device tensors (int32, int32, float32, float32) when the caller itself
    cannot allocate; host lists are converted here for convenience."""
    torch = _torch()
    lib = load()
    if not hasattr(lib, "_noalloc_ready"):
        lib.eap_pairs_noalloc.argtypes = [ctypes.POINTER(eap_params), ctypes.POINTER(eap_series_set),
                                          ctypes.POINTER(eap_series_set), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.POINTER(eap_stats)]
        lib.eap_pairs_noalloc.restype = ctypes.c_int
        lib._noalloc_ready = True
    dev = a.data.device
    ia = torch.as_tensor(ia, dtype=torch.int32, device=dev).contiguous()
    ib = torch.as_tensor(ib, dtype=torch.int32, device=dev).contiguous()
    n = int(ia.numel())
    if cutoff is None:
        cutoff = torch.full((n,), float("inf"), dtype=torch.float32, device=dev)
    cut = torch.as_tensor(cutoff, dtype=torch.float32, device=dev).contiguous()
    res = out if out is not None else torch.empty(n, dtype=torch.float32, device=dev)
    sa, sb = a.struct(), b.struct()
    st = eap_stats()
    rc = lib.eap_pairs_noalloc(ctypes.byref(p), ctypes.byref(sa), ctypes.byref(sb), ctypes.c_void_p(ia.data_ptr()),
                               ctypes.c_void_p(ib.data_ptr()), ctypes.c_void_p(cut.data_ptr()),
                               ctypes.c_void_p(res.data_ptr()), n, _stream_ptr(stream),
                               ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_pairs_noalloc")
    return (res, st.as_dict()) if with_stats else res


class eap_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("lat_p50_ms", ctypes.c_double), ("lat_p99_ms", ctypes.c_double),
                ("lat_max_ms", ctypes.c_double), ("inflight_bytes", ctypes.c_int64), ("inflight", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved_"}


class Server:
    """eap_serve_*: resident reference sets, footprint admission, continuous
    batching of single 1-NN queries submitted from host memory."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=0, max_query_len=0, device=0):
        _torch()
        lib = load()
        if not hasattr(lib, "_serve_ready"):
            P = ctypes.POINTER
            lib.eap_serve_stats_get.argtypes = [ctypes.c_void_p, P(eap_serve_stats), ctypes.c_int32]
            for n in ("eap_serve_add_refset", "eap_serve_submit", "eap_serve_poll", "eap_serve_drain",
                      "eap_serve_destroy", "eap_serve_stats_get"):
                getattr(lib, n).restype = ctypes.c_int
            lib._serve_ready = True
        self._lib = lib
        cfg = eap_serve_config(int(hbm_budget_bytes), int(max_inflight), int(max_query_len), int(device), 0)
        status = ctypes.c_int(0)
        self._h = lib.eap_serve_create(ctypes.byref(cfg), ctypes.byref(status))
        if not self._h:
            raise EapError(status.value, "eap_serve_create")
        self._keep = []

    def add_refset(self, packed) -> int:
        data = np.ascontiguousarray(packed.data, dtype=np.float32)
        off = np.ascontiguousarray(packed.offsets, dtype=np.int64)
        ln = np.ascontiguousarray(packed.lengths, dtype=np.int32)
        sid = ctypes.c_int32(-1)
        rc = self._lib.eap_serve_add_refset(self._h, ctypes.c_void_p(data.ctypes.data), ctypes.c_void_p(off.ctypes.data),
                                            ctypes.c_void_p(ln.ctypes.data), len(ln), ctypes.byref(sid))
        _check(rc, "eap_serve_add_refset")
        return sid.value

    def submit(self, set_id: int, p: eap_params, query) -> int | None:
        """Ticket, or None when the query is not admitted now (EAP_EAGAIN)."""
        q = np.ascontiguousarray(query, dtype=np.float32)
        t = ctypes.c_uint64(0)
        rc = self._lib.eap_serve_submit(self._h, int(set_id), ctypes.byref(p), ctypes.c_void_p(q.ctypes.data),
                                        len(q), ctypes.byref(t))
        if rc == EAP_EAGAIN:
            return None
        _check(rc, "eap_serve_submit")
        return t.value

    def poll(self, ticket: int):
        """(idx, dist) once done, None before."""
        idx, dist = ctypes.c_int32(0), ctypes.c_float(0)
        rc = self._lib.eap_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(idx), ctypes.byref(dist))
        if rc == EAP_EAGAIN:
            return None
        _check(rc, "eap_serve_poll")
        return idx.value, dist.value

    def drain(self, timeout_ms: int = 60000):
        _check(self._lib.eap_serve_drain(self._h, int(timeout_ms)), "eap_serve_drain")

    def stats(self, reset: bool = False) -> dict:
        st = eap_serve_stats()
        _check(self._lib.eap_serve_stats_get(self._h, ctypes.byref(st), int(reset)), "eap_serve_stats_get")
        return st.as_dict()

    def close(self):
        if self._h:
            self._lib.eap_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class eap_nn1_task(ctypes.Structure):
    _fields_ = [("params", eap_params), ("queries", eap_series_set), ("refs", eap_series_set),
                ("out_idx", ctypes.c_void_p), ("out_dist", ctypes.c_void_p)]


def _batch_lib():
    lib = load()
    if not hasattr(lib, "_batch_ready"):
        P = ctypes.POINTER
        lib.eap_nn1_batch.argtypes = [P(eap_nn1_task), ctypes.c_int32, ctypes.c_void_p, P(eap_stats)]
        lib.eap_nn1_batch.restype = ctypes.c_int
        lib.eap_autotune.argtypes = [P(eap_nn1_task), ctypes.c_int32, ctypes.c_void_p, ctypes.c_char_p]
        lib.eap_autotune.restype = ctypes.c_int
        lib.eap_autotune_load.argtypes = [ctypes.c_char_p]
        lib.eap_autotune_load.restype = ctypes.c_int
        lib.eap_autotune_reset.argtypes = []
        lib.eap_autotune_reset.restype = None
        lib._batch_ready = True
    return lib


class Nn1Task:
    """One 1-NN problem of a batch: parameters, query and reference sets,
    and device output tensors (allocated here unless given)."""

    def __init__(self, p: eap_params, queries: SeriesSet, refs: SeriesSet, out_idx=None, out_dist=None):
        torch = _torch()
        dev = queries.data.device
        self.p, self.queries, self.refs = p, queries, refs
        self.out_idx = out_idx if out_idx is not None else torch.empty(queries.count, dtype=torch.int32, device=dev)
        self.out_dist = out_dist if out_dist is not None else torch.empty(queries.count, dtype=torch.float32,
                                                                          device=dev)

    def struct(self) -> eap_nn1_task:
        t = eap_nn1_task()
        t.params = self.p
        t.queries = self.queries.struct()
        t.refs = self.refs.struct()
        t.out_idx = self.out_idx.data_ptr() if self.queries.count else None
        t.out_dist = self.out_dist.data_ptr() if self.queries.count else None
        return t


def _task_array(tasks):
    arr = (eap_nn1_task * max(1, len(tasks)))()
    for i, t in enumerate(tasks):
        arr[i] = t.struct()
    return arr


def eap_nn1_batch(tasks, stream=None, with_stats=False):
    """All tasks' 1-NN searches in one persistent DP launch (results land in
    each task's out_idx / out_dist)."""
    lib = _batch_lib()
    arr = _task_array(tasks)
    st = eap_stats()
    rc = lib.eap_nn1_batch(arr, len(tasks), _stream_ptr(stream), ctypes.byref(st) if with_stats else None)
    _check(rc, "eap_nn1_batch")
    return st.as_dict() if with_stats else None


def eap_autotune(tasks, stream=None, cache_path=None):
    lib = _batch_lib()
    arr = _task_array(tasks)
    rc = lib.eap_autotune(arr, len(tasks), _stream_ptr(stream), cache_path.encode() if cache_path else None)
    _check(rc, "eap_autotune")


def eap_autotune_load(cache_path):
    _check(_batch_lib().eap_autotune_load(cache_path.encode()), "eap_autotune_load")


def eap_autotune_reset():
    _batch_lib().eap_autotune_reset()
