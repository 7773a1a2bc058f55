"""Python binding of libcdgpu (community detection on one GB300 GPU).

Argument marshalling only: every function below forwards to the C entry point
of the same name in ``libcdgpu.so`` (declared in ``include/cdgpu.h``); all
compute runs in the library's CUDA kernels. PyTorch is used for device memory
and streams. There is no CPU fallback: if the library cannot be loaded the
calls raise.

Method: arXiv 2507.06471 — Label Propagation (Algorithm 1), Louvain local
moving (Algorithm 2, Eq. deltaQ) and aggregation (Algorithm 3), modularity
(Sec. II-C), under the synchronous schedule described in ``cdgpu.h``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

CD_OK, CD_EINVAL, CD_EBOUNDS, CD_ENOMEM, CD_ECUDA, CD_EOVERFLOW, CD_ETIMEOUT, CD_ENOTSYM = (
    0, -1, -2, -3, -4, -5, -6, -7)

EXPORTED = [
    "cd_params_default", "cd_csr_upload", "cd_graph_free", "cd_graph_info", "cd_graph_download",
    "cd_lpa_run", "cd_louvain_local_move", "cd_louvain_aggregate", "cd_modularity",
    "cd_louvain_run", "cd_trace_get", "cd_profile_get", "cd_status_string", "cd_last_cuda_error",
    "cd_launch_count", "cd_modularity_noalloc", "cd_graph_set_batches", "cd_batch_lpa_run",
    "cd_batch_louvain_run", "cd_graph_set_bins", "cd_autotune", "cd_server_create", "cd_server_submit",
    "cd_server_wait", "cd_server_stats", "cd_server_destroy",
]

CD_REQ_LPA, CD_REQ_LOUVAIN = 1, 2


class cd_params(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("threshold", ctypes.c_int64), ("tie_keep_current", ctypes.c_int32),
                ("singleton_rule", ctypes.c_int32), ("use_frontier", ctypes.c_int32),
                ("timing", ctypes.c_int32), ("sched_seed", ctypes.c_uint64),
                ("aggregation", ctypes.c_int32), ("asynchronous", ctypes.c_int32),
                ("device_loop", ctypes.c_int32)]


class cd_round_trace(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("round", ctypes.c_int32), ("active", ctypes.c_int64),
                ("arcs", ctypes.c_int64), ("moved", ctypes.c_int64), ("deferred", ctypes.c_int64),
                ("scan_ms", ctypes.c_float), ("round_ms", ctypes.c_float), ("cands", ctypes.c_int64),
                ("moved_arcs", ctypes.c_int64)]


class cd_kernel_profile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double)]


class cd_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("n", ctypes.c_int64),
                ("q", ctypes.c_double), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("batched_with", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class CDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.cd_status_string(status).decode() if _lib else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


_lib = None
_P = ctypes.c_void_p


def lib():
    """Load libcdgpu.so (building it first if the sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.cd_params_default.argtypes = [ctypes.POINTER(cd_params)]
        L.cd_csr_upload.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, _P, ctypes.POINTER(_P)]
        L.cd_graph_free.argtypes = [_P]
        L.cd_graph_info.argtypes = [_P, _P, _P, _P]
        L.cd_graph_download.argtypes = [_P, _P, _P, _P, ctypes.c_int]
        L.cd_lpa_run.argtypes = [_P, ctypes.POINTER(cd_params), _P, ctypes.c_int, _P]
        L.cd_louvain_local_move.argtypes = [_P, ctypes.POINTER(cd_params), _P, ctypes.c_int,
                                            ctypes.c_int, _P, _P]
        L.cd_louvain_aggregate.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(_P), _P, _P]
        L.cd_modularity.argtypes = [_P, _P, ctypes.c_int, _P]
        L.cd_louvain_run.argtypes = [_P, ctypes.POINTER(cd_params), _P, ctypes.c_int, _P, _P]
        L.cd_trace_get.argtypes = [_P, _P, ctypes.c_int32, _P]
        L.cd_profile_get.argtypes = [_P, _P, ctypes.c_int32, _P]
        L.cd_status_string.restype = ctypes.c_char_p
        L.cd_status_string.argtypes = [ctypes.c_int]
        L.cd_last_cuda_error.argtypes = []
        L.cd_launch_count.restype = ctypes.c_int64
        L.cd_launch_count.argtypes = []
        L.cd_modularity_noalloc.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P]
        L.cd_graph_set_batches.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int]
        L.cd_graph_set_bins.argtypes = [_P, ctypes.c_int32, ctypes.c_int32]
        L.cd_autotune.argtypes = [_P, ctypes.POINTER(cd_params), ctypes.c_int32, _P, _P]
        L.cd_batch_lpa_run.argtypes = [_P, ctypes.POINTER(cd_params), _P, ctypes.c_int, _P]
        L.cd_batch_louvain_run.argtypes = [_P, ctypes.POINTER(cd_params), _P, ctypes.c_int, _P, _P]
        L.cd_server_create.argtypes = [ctypes.POINTER(cd_params), ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_P)]
        L.cd_server_submit.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int, _P, _P, ctypes.c_int64,
                                       ctypes.c_int64, _P]
        L.cd_server_wait.argtypes = [_P, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(cd_request_result), _P]
        L.cd_server_stats.argtypes = [_P, _P, _P, _P, _P]
        L.cd_server_destroy.argtypes = [_P]
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != CD_OK:
        raise CDError(rc, where)


def _ptr(x):
    """(pointer, on_device) of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    return x.ctypes.data_as(ctypes.c_void_p), 0


def _stream_ptr(stream):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ------------------------------------------------------------------ same-name entry points

def cd_params_default(**overrides) -> cd_params:
    p = cd_params()
    _check(lib().cd_params_default(ctypes.byref(p)), "cd_params_default")
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def cd_csr_upload(offsets, cols, w=None, n: Optional[int] = None, stream=None) -> ctypes.c_void_p:
    """Upload a symmetric CSR (torch tensors on one device, or numpy arrays)."""
    n = (len(offsets) - 1) if n is None else n
    nnz = int(len(cols))
    po, dev_o = _ptr(offsets)
    pc, dev_c = _ptr(cols)
    pw, dev_w = _ptr(w)
    if w is not None and dev_w != dev_o:
        raise ValueError("offsets, cols and w must live on the same side (host or device)")
    if dev_o != dev_c:
        raise ValueError("offsets and cols must live on the same side (host or device)")
    is64 = int(str(offsets.dtype).endswith("int64"))
    if not is64 and not str(offsets.dtype).endswith("int32"):
        raise TypeError("offsets must be int32 or int64")
    if not str(cols.dtype).endswith("int32") or (w is not None and not str(w.dtype).endswith("int32")):
        raise TypeError("cols and w must be int32")
    out = ctypes.c_void_p()
    _check(lib().cd_csr_upload(po, is64, pc, pw, n, nnz, dev_o, _stream_ptr(stream), ctypes.byref(out)),
           "cd_csr_upload")
    return out


def cd_graph_free(g) -> None:
    _check(lib().cd_graph_free(g), "cd_graph_free")


def cd_graph_info(g):
    n, nnz, vol = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cd_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(vol)), "cd_graph_info")
    return n.value, nnz.value, vol.value


def cd_graph_download(g):
    """(off int64[n+1], cols int32[nnz], w int64[nnz]) host arrays, loops as L."""
    n, nnz, _ = cd_graph_info(g)
    off = np.zeros(n + 1, dtype=np.int64)
    cols = np.zeros(max(nnz, 1), dtype=np.int32)
    w = np.zeros(max(nnz, 1), dtype=np.int64)
    _check(lib().cd_graph_download(g, _ptr(off)[0], _ptr(cols)[0], _ptr(w)[0], 0), "cd_graph_download")
    return off, cols[:nnz], w[:nnz]


def cd_lpa_run(g, params: cd_params, labels_out):
    p, dev = _ptr(labels_out)
    r = ctypes.c_int32()
    _check(lib().cd_lpa_run(g, ctypes.byref(params), p, dev, ctypes.byref(r)), "cd_lpa_run")
    return r.value


def cd_louvain_local_move(g, params: cd_params, labels_io, init_given: bool = False):
    p, dev = _ptr(labels_io)
    mv, r = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().cd_louvain_local_move(g, ctypes.byref(params), p, int(init_given), dev,
                                       ctypes.byref(mv), ctypes.byref(r)), "cd_louvain_local_move")
    return mv.value, r.value


def cd_louvain_aggregate(g, labels, newid_out=None):
    p, dev = _ptr(labels)
    pn, devn = _ptr(newid_out)
    if newid_out is not None and devn != dev:
        raise ValueError("labels and newid_out must live on the same side")
    out, k = ctypes.c_void_p(), ctypes.c_int64()
    _check(lib().cd_louvain_aggregate(g, p, dev, ctypes.byref(out), pn, ctypes.byref(k)),
           "cd_louvain_aggregate")
    return out, k.value


def cd_modularity(g, labels) -> float:
    p, dev = _ptr(labels)
    q = ctypes.c_double()
    _check(lib().cd_modularity(g, p, dev, ctypes.byref(q)), "cd_modularity")
    return q.value


def cd_louvain_run(g, params: cd_params, labels_out):
    p, dev = _ptr(labels_out)
    lv, q = ctypes.c_int32(), ctypes.c_double()
    _check(lib().cd_louvain_run(g, ctypes.byref(params), p, dev, ctypes.byref(lv), ctypes.byref(q)),
           "cd_louvain_run")
    return lv.value, q.value


def cd_trace_get(g):
    cnt = ctypes.c_int32()
    _check(lib().cd_trace_get(g, None, 0, ctypes.byref(cnt)), "cd_trace_get")
    buf = (cd_round_trace * max(cnt.value, 1))()
    _check(lib().cd_trace_get(g, buf, cnt.value, ctypes.byref(cnt)), "cd_trace_get")
    return [{f: getattr(buf[i], f) for f, _ in cd_round_trace._fields_} for i in range(cnt.value)]


def cd_profile_get(g):
    cnt = ctypes.c_int32()
    buf = (cd_kernel_profile * 64)()
    _check(lib().cd_profile_get(g, buf, 64, ctypes.byref(cnt)), "cd_profile_get")
    return [{"name": buf[i].name.decode(), "launches": buf[i].launches, "total_ms": buf[i].total_ms,
             "alg_bytes": buf[i].alg_bytes} for i in range(min(cnt.value, 64))]


def cd_modularity_noalloc(offsets, cols, w, labels, n: Optional[int] = None, stream=None) -> float:
    """Modularity without device allocation (device tensors: int64 offsets,
    int32 cols/w/labels); see cdgpu.h for the size limit and the rules."""
    n = (len(offsets) - 1) if n is None else n
    ptrs = [_ptr(x) for x in (offsets, cols, w, labels)]
    if any(p is not None and not dev for p, dev in ptrs):
        raise ValueError("cd_modularity_noalloc takes device arrays only")
    if str(offsets.dtype) != "torch.int64":
        raise TypeError("offsets must be int64")
    q = ctypes.c_double()
    _check(lib().cd_modularity_noalloc(ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], n, int(len(cols)),
                                       _stream_ptr(stream), ctypes.byref(q)), "cd_modularity_noalloc")
    return q.value


def cd_graph_set_batches(g, vstart) -> None:
    """vstart: int64 array of n_graphs+1 vertex offsets (host numpy or device tensor)."""
    p, dev = _ptr(vstart)
    _check(lib().cd_graph_set_batches(g, p, int(len(vstart)) - 1, dev), "cd_graph_set_batches")


def cd_batch_lpa_run(g, params: cd_params, labels_out, n_graphs: int):
    p, dev = _ptr(labels_out)
    rounds = np.zeros(n_graphs, dtype=np.int32)
    _check(lib().cd_batch_lpa_run(g, ctypes.byref(params), p, dev, _ptr(rounds)[0]), "cd_batch_lpa_run")
    return rounds


def cd_batch_louvain_run(g, params: cd_params, labels_out, n_graphs: int):
    p, dev = _ptr(labels_out)
    levels = np.zeros(n_graphs, dtype=np.int32)
    q = np.zeros(n_graphs, dtype=np.float64)
    _check(lib().cd_batch_louvain_run(g, ctypes.byref(params), p, dev, _ptr(levels)[0], _ptr(q)[0]),
           "cd_batch_louvain_run")
    return levels, q


def cd_graph_set_bins(g, t_warp: int, t_hub: int) -> None:
    _check(lib().cd_graph_set_bins(g, t_warp, t_hub), "cd_graph_set_bins")


def cd_autotune(g, params: cd_params, rounds: int = 3):
    tw, th = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().cd_autotune(g, ctypes.byref(params), rounds, ctypes.byref(tw), ctypes.byref(th)), "cd_autotune")
    return tw.value, th.value


def cd_launch_count() -> int:
    return int(lib().cd_launch_count())


def cd_status_string(status: int) -> str:
    return lib().cd_status_string(status).decode()


def cd_server_create(params: cd_params, slots: int = 4, mem_budget_bytes: int = 0, small_n: int = 4096,
                     batch_arcs: int = 1 << 24) -> ctypes.c_void_p:
    h = _P()
    _check(lib().cd_server_create(ctypes.byref(params), slots, mem_budget_bytes, small_n, batch_arcs,
                                  ctypes.byref(h)), "cd_server_create")
    return h


def cd_server_submit(s, kind: int, offsets, cols, w=None) -> int:
    """Queue one request; offsets/cols/w are HOST numpy arrays (copied)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
    rid = ctypes.c_int64()
    _check(lib().cd_server_submit(s, kind, _ptr(offsets)[0], 1, _ptr(cols)[0], _ptr(w)[0], len(offsets) - 1,
                                  len(cols), ctypes.byref(rid)), "cd_server_submit")
    return rid.value


def cd_server_wait(s, rid: int, n: int, timeout_ms: int = -1):
    """(labels (numpy int32), cd_request_result) of a finished request."""
    res = cd_request_result()
    labels = np.empty(n, dtype=np.int32)
    _check(lib().cd_server_wait(s, rid, timeout_ms, ctypes.byref(res), _ptr(labels)[0]), "cd_server_wait")
    return labels, res


def cd_server_stats(s):
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib().cd_server_stats(s, *[ctypes.byref(x) for x in v]), "cd_server_stats")
    return {"admitted": v[0].value, "completed": v[1].value, "packed_calls": v[2].value, "in_use": v[3].value}


def cd_server_destroy(s) -> None:
    _check(lib().cd_server_destroy(s), "cd_server_destroy")


# ------------------------------------------------------------------ convenience handle

class Graph:
    """Owns a cd_graph handle; methods forward to the entry points above."""

    def __init__(self, offsets, cols, w=None, stream=None):
        self.h = cd_csr_upload(offsets, cols, w, stream=stream)
        self.n, self.nnz, self.vol = cd_graph_info(self.h)

    @classmethod
    def _adopt(cls, h):
        g = cls.__new__(cls)
        g.h = h
        g.n, g.nnz, g.vol = cd_graph_info(h)
        return g

    def close(self):
        if getattr(self, "h", None):
            cd_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _labels(self, device):
        import torch
        return torch.empty(self.n, dtype=torch.int32, device=device)

    def lpa(self, params=None, device="cuda", **kw):
        params = params or cd_params_default(**kw)
        lab = self._labels(device)
        rounds = cd_lpa_run(self.h, params, lab)
        return lab, rounds

    def local_move(self, params=None, labels=None, device="cuda", **kw):
        params = params or cd_params_default(**kw)
        if labels is None:
            lab = self._labels(device)
            moves, rounds = cd_louvain_local_move(self.h, params, lab, False)
        else:
            lab = labels.clone()
            moves, rounds = cd_louvain_local_move(self.h, params, lab, True)
        return lab, moves, rounds

    def louvain(self, params=None, device="cuda", **kw):
        params = params or cd_params_default(**kw)
        lab = self._labels(device)
        levels, q = cd_louvain_run(self.h, params, lab)
        return lab, levels, q

    def aggregate(self, labels, newid_out=None):
        h, k = cd_louvain_aggregate(self.h, labels, newid_out)
        return Graph._adopt(h), k

    def modularity(self, labels) -> float:
        return cd_modularity(self.h, labels)

    def download(self):
        return cd_graph_download(self.h)

    def set_batches(self, vstart):
        cd_graph_set_batches(self.h, vstart)
        self.n_graphs = int(len(vstart)) - 1

    def batch_lpa(self, params=None, device="cuda", **kw):
        params = params or cd_params_default(**kw)
        lab = self._labels(device)
        rounds = cd_batch_lpa_run(self.h, params, lab, self.n_graphs)
        return lab, rounds

    def batch_louvain(self, params=None, device="cuda", **kw):
        params = params or cd_params_default(**kw)
        lab = self._labels(device)
        levels, q = cd_batch_louvain_run(self.h, params, lab, self.n_graphs)
        return lab, levels, q

    def trace(self):
        return cd_trace_get(self.h)

    def profile(self):
        return cd_profile_get(self.h)


class Server:
    """Owns a cd_server; submit() returns an id, result() waits for it."""

    def __init__(self, params=None, slots=4, mem_budget_bytes=0, small_n=4096, batch_arcs=1 << 24, **kw):
        params = params or cd_params_default(**kw)
        self.h = cd_server_create(params, slots, mem_budget_bytes, small_n, batch_arcs)
        self._n = {}

    def submit(self, kind, offsets, cols, w=None) -> int:
        rid = cd_server_submit(self.h, kind, offsets, cols, w)
        self._n[rid] = len(offsets) - 1
        return rid

    def result(self, rid, timeout_ms=-1):
        try:
            labels, res = cd_server_wait(self.h, rid, self._n[rid], timeout_ms)
        except CDError as e:
            if e.status != CD_ETIMEOUT:  # the request is finished (failed)
                self._n.pop(rid, None)
            raise
        del self._n[rid]
        return labels, res

    def stats(self):
        return cd_server_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            cd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
