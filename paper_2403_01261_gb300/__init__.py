"""GB300 (sm_103a) GSL-LPA: label propagation with split-last, on one GPU.

Thin Python binding over the C ABI of ``include/gsllpa.h`` (libgsllpa.so):
argument marshalling only, every step runs in the library's CUDA kernels.
There is no CPU fallback; if the library cannot be loaded the import of a
function fails with an error.  PyTorch supplies device memory and streams.

    import paper_2403_01261_gb300 as gsl
    labels = gsl.gsllpa(offsets, cols)            # torch CUDA tensors
    q = gsl.modularity(offsets, cols, labels)
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = ["Stats", "Context", "GslError", "lpa", "split", "modularity", "gsllpa", "gsllpa_host", "library_path",
           "load", "kernel_launches", "Server", "MODE_SYNC", "MODE_ASYNC"]

MODE_SYNC = 0
MODE_ASYNC = 1
STATS_SWEEPS = 64

_lock = threading.Lock()
_lib = None


class GslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gsl error {code}: {msg}")
        self.code = code


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("cols", ctypes.c_void_p)]


class ProfileSlot(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("kernels", ctypes.c_int64),
                ("ms", ctypes.c_double), ("vertices", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("bytes", ctypes.c_double)]


class Profile(ctypes.Structure):
    _fields_ = [("nslots", ctypes.c_int32), ("slot", ProfileSlot * 24)]


class BatchStats(ctypes.Structure):
    _fields_ = [("num_graphs", ctypes.c_int32), ("pad", ctypes.c_int32), ("graph_launches", ctypes.c_int64),
                ("ms", ctypes.c_float)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("slot_vertices", ctypes.c_int64),
                ("slot_entries", ctypes.c_int64), ("memory_fraction", ctypes.c_double),
                ("max_batch_graphs", ctypes.c_int32), ("mode", ctypes.c_int32), ("tolerance", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("pad", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("batch_graphs", ctypes.c_int64),
                ("queue_ms", ctypes.c_double), ("service_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("h2d_ms", ctypes.c_double), ("compute_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("batches", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("max_concurrent_batches", ctypes.c_int64)]


class TuneResult(ctypes.Structure):
    _fields_ = [("warp_max", ctypes.c_int32), ("blk_max", ctypes.c_int32), ("pregather", ctypes.c_int32),
                ("candidates", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("best_ms", ctypes.c_float), ("entry_ms", ctypes.c_float),
                ("majority", ctypes.c_int32), ("blk_threads", ctypes.c_int32), ("blk_slots", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("changed", ctypes.c_int64 * STATS_SWEEPS), ("active", ctypes.c_int64 * STATS_SWEEPS),
                ("edges_scanned", ctypes.c_int64), ("communities", ctypes.c_int64),
                ("ms_lpa", ctypes.c_float), ("ms_split", ctypes.c_float)]

    def as_dict(self):
        t = min(self.iterations, STATS_SWEEPS)
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "changed": list(self.changed[:t]), "active": list(self.active[:t]),
                "edges_scanned": self.edges_scanned, "communities": self.communities,
                "ms_lpa": self.ms_lpa, "ms_split": self.ms_split}


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load().gsl_kernel_launches())


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libgsllpa.so, building it with nvcc first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sp = ctypes.POINTER(Stats)
        cp = ctypes.POINTER(Csr)
        lib.gsl_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
        lib.gsl_ctx_destroy.argtypes = [P]
        lib.gsl_ctx_set_tuning.argtypes = [P, i32, i32]
        lib.gsl_autotune.argtypes = [P, cp, P, i32, i32, ctypes.POINTER(TuneResult), P]
        lib.gsl_autotune_batch.argtypes = [P, cp, i32, P, P, dbl, i32, i32, P, ctypes.POINTER(TuneResult), P]
        lib.gsl_ctx_set_pregather.argtypes = [P, i32]
        lib.gsl_ctx_set_block_config.argtypes = [P, i32, i32]
        lib.gsl_ctx_set_majority.argtypes = [P, i32]
        lib.gsl_ctx_set_hub_cluster.argtypes = [P, i64]
        lib.gsl_ctx_set_f32_fixed.argtypes = [P, i32]
        lib.gsl_ctx_set_retry_bounds.argtypes = [P, i32, i32]
        lib.gsl_ctx_set_host_overlap.argtypes = [P, i64]
        lib.gsl_lpa_f32.argtypes = [P, cp, P, P, dbl, i32, i32, P, sp, P]
        lib.gsl_gsllpa_f32.argtypes = [P, cp, P, dbl, i32, i32, P, sp, P]
        lib.gsl_modularity_f32.argtypes = [P, cp, P, P, ctypes.POINTER(dbl), P]
        lib.gsl_split_lp.argtypes = [P, cp, P, P, i32, ctypes.POINTER(i32), P]
        lib.gsl_disconnected.argtypes = [P, cp, P, P, ctypes.POINTER(i64), P]
        lib.gsl_lpa.argtypes = [P, cp, P, P, dbl, i32, i32, P, sp, P]
        lib.gsl_split.argtypes = [P, cp, P, P, i32, ctypes.POINTER(i64), P]
        lib.gsl_modularity.argtypes = [P, cp, P, P, ctypes.POINTER(dbl), P]
        lib.gsl_gsllpa.argtypes = [P, cp, P, dbl, i32, i32, P, sp, P]
        lib.gsl_gsllpa_host.argtypes = [P, i64, i64, P, P, P, dbl, i32, i32, P, sp, P]
        lib.gsl_gsllpa_batch.argtypes = [P, cp, i32, P, P, dbl, i32, i32, P, P, ctypes.POINTER(BatchStats), P]
        lib.gsl_ctx_set_batch_mode.argtypes = [P, i32]
        lib.gsl_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ServerConfig)]
        lib.gsl_server_capacity.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.gsl_server_submit.argtypes = [P, i64, i64, P, P, ctypes.POINTER(i64)]
        lib.gsl_server_wait.argtypes = [P, i64, P, ctypes.POINTER(RequestInfo)]
        lib.gsl_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        lib.gsl_server_destroy.argtypes = [P]
        lib.gsl_strerror.restype = ctypes.c_char_p
        lib.gsl_strerror.argtypes = [ctypes.c_int]
        lib.gsl_ctx_last_error.restype = ctypes.c_char_p
        lib.gsl_ctx_last_error.argtypes = [P]
        lib.gsl_version.restype = ctypes.c_int
        lib.gsl_ctx_set_profiling.argtypes = [P, i32]
        lib.gsl_ctx_get_profile.argtypes = [P, ctypes.POINTER(Profile)]
        lib.gsl_kernel_launches.restype = i64
        lib.gsl_kernel_launches.argtypes = []
        for name in ("gsl_ctx_create", "gsl_ctx_destroy", "gsl_ctx_set_tuning", "gsl_lpa", "gsl_split",
                     "gsl_ctx_set_profiling", "gsl_ctx_get_profile",
                     "gsl_modularity", "gsl_gsllpa", "gsl_gsllpa_host", "gsl_gsllpa_batch", "gsl_ctx_set_batch_mode",
                     "gsl_server_create", "gsl_server_capacity", "gsl_server_submit", "gsl_server_wait",
                     "gsl_server_get_stats", "gsl_server_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_graph(offsets, cols, weights=None):
    import torch
    if not (offsets.is_cuda and cols.is_cuda):
        raise ValueError("offsets and cols must be CUDA tensors")
    if offsets.dtype != torch.int64 or cols.dtype != torch.int32:
        raise TypeError("offsets must be int64 and cols int32")
    if not (offsets.is_contiguous() and cols.is_contiguous()):
        raise ValueError("offsets and cols must be contiguous")
    if weights is not None and (weights.dtype != torch.int32 or not weights.is_cuda or not weights.is_contiguous()
                                or weights.numel() != cols.numel()):
        raise TypeError("weights must be a contiguous int32 CUDA tensor with one entry per column")
    c = Csr()
    c.n = offsets.numel() - 1
    c.nnz = cols.numel()
    c.offsets = offsets.data_ptr()
    c.cols = cols.data_ptr() if cols.numel() else None
    return c


class Context:
    """One library context (scratch memory) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self.device = device
        rc = self._lib.gsl_ctx_create(ctypes.byref(self._h), device)
        if rc != 0:
            raise GslError(rc, self._lib.gsl_strerror(rc).decode())

    def close(self):
        if self._h:
            self._lib.gsl_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass

    def _raise(self, rc):
        if rc != 0:
            raise GslError(rc, f"{self._lib.gsl_strerror(rc).decode()}: {self._lib.gsl_ctx_last_error(self._h).decode()}")

    def set_tuning(self, warp_max: int, blk_max: int):
        self._raise(self._lib.gsl_ctx_set_tuning(self._h, warp_max, blk_max))

    def autotune(self, offsets, cols, weights=None, mode=MODE_SYNC, sweeps=4, stream=None):
        """Times the first `sweeps` sweeps under each candidate threshold pair
        and sets the fastest on this context; returns the choice and times."""
        g = _check_graph(offsets, cols, weights)
        r = TuneResult()
        self._raise(self._lib.gsl_autotune(self._h, ctypes.byref(g), _ptr(weights), int(mode), int(sweeps),
                                           ctypes.byref(r), _stream(stream)))
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def autotune_batch(self, offsets, cols, vptr, weights=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC,
                       out=None, stream=None):
        """Times the batched path (gsl_gsllpa_batch) under each candidate
        setting on these packed graphs and sets the fastest on this context;
        returns (labels, the choice and times)."""
        import numpy as np
        import torch
        g = _check_graph(offsets, cols, weights)
        vp = np.ascontiguousarray(vptr, dtype=np.int64)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        r = TuneResult()
        self._raise(self._lib.gsl_autotune_batch(self._h, ctypes.byref(g), int(vp.shape[0] - 1),
                                                 vp.ctypes.data_as(ctypes.c_void_p), _ptr(weights), float(tolerance),
                                                 int(max_iters), int(mode), _ptr(out), ctypes.byref(r),
                                                 _stream(stream)))
        return out, {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def set_block_config(self, threads: int, table_slots: int):
        self._raise(self._lib.gsl_ctx_set_block_config(self._h, int(threads), int(table_slots)))

    def set_majority(self, mode: int):
        """0: never, 1: once labels settle (default), 2: every sweep after the first."""
        self._raise(self._lib.gsl_ctx_set_majority(self._h, int(mode)))

    def set_f32_fixed(self, mode: int):
        """1 (default): float weights with an exact fixed-point form run on
        the integer sweeps; 0: always float64 sums."""
        self._raise(self._lib.gsl_ctx_set_f32_fixed(self._h, int(mode)))

    def set_hub_cluster(self, max_degree: int):
        """Hubs up to this degree are aggregated by one 8-CTA thread-block
        cluster each (default: every hub); 0 turns the clusters off."""
        self._raise(self._lib.gsl_ctx_set_hub_cluster(self._h, int(max_degree)))

    def set_pregather(self, mode: int):
        """0: never (default), 1: when the frontier is large, 2: every eligible sweep."""
        self._raise(self._lib.gsl_ctx_set_pregather(self._h, int(mode)))

    def set_retry_bounds(self, probe_bound: int = 0, unionfind_bound: int = 0):
        """Bounds of the device retry loops (hash probes, union-find steps);
        0 restores the defaults.  A loop that reaches its bound makes the call
        fail with GSL_ERR_TIMEOUT."""
        self._raise(self._lib.gsl_ctx_set_retry_bounds(self._h, int(probe_bound), int(unionfind_bound)))

    def set_host_overlap(self, min_entries: int):
        """Entries from which gsllpa_host overlaps its column copy with the
        first two sweeps (pinned columns, unit weights, synchronous mode);
        0: never."""
        self._raise(self._lib.gsl_ctx_set_host_overlap(self._h, int(min_entries)))

    def set_batch_mode(self, use_cuda_graph: bool):
        self._raise(self._lib.gsl_ctx_set_batch_mode(self._h, int(bool(use_cuda_graph))))

    def set_profiling(self, enable: bool):
        """Enables (and zeroes) or disables per-slot CUDA-event profiling."""
        self._raise(self._lib.gsl_ctx_set_profiling(self._h, int(bool(enable))))

    def profile(self):
        """Per-slot device time, counts and algorithmic bytes since profiling was enabled."""
        p = Profile()
        self._raise(self._lib.gsl_ctx_get_profile(self._h, ctypes.byref(p)))
        out = []
        for k in range(p.nslots):
            sl = p.slot[k]
            out.append({"name": sl.name.decode(), "launches": sl.launches, "kernels": sl.kernels, "ms": sl.ms,
                        "vertices": sl.vertices, "entries": sl.entries, "bytes": sl.bytes})
        return out

    def lpa(self, offsets, cols, weights=None, labels_init=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC,
            out=None, stream=None, stats=False):
        import torch
        g = _check_graph(offsets, cols, weights)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        st = Stats()
        rc = self._lib.gsl_lpa(self._h, ctypes.byref(g), _ptr(weights), _ptr(labels_init), float(tolerance),
                               int(max_iters), int(mode), _ptr(out), ctypes.byref(st), _stream(stream))
        self._raise(rc)
        return (out, st.as_dict()) if stats else out

    def _check_f32(self, cols, weights):
        import torch
        if (weights is None or weights.dtype != torch.float32 or not weights.is_cuda or not weights.is_contiguous()
                or weights.numel() != cols.numel()):
            raise TypeError("weights must be a contiguous float32 CUDA tensor with one entry per column")

    def lpa_f32(self, offsets, cols, weights, labels_init=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC,
                out=None, stream=None, stats=False):
        """LPA with float32 weights and float64 sums (the paper's precision)."""
        import torch
        g = _check_graph(offsets, cols)
        self._check_f32(cols, weights)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        st = Stats()
        self._raise(self._lib.gsl_lpa_f32(self._h, ctypes.byref(g), _ptr(weights), _ptr(labels_init),
                                          float(tolerance), int(max_iters), int(mode), _ptr(out), ctypes.byref(st),
                                          _stream(stream)))
        return (out, st.as_dict()) if stats else out

    def gsllpa_f32(self, offsets, cols, weights, tolerance=0.05, max_iters=20, mode=MODE_SYNC, out=None,
                   stream=None, stats=False):
        import torch
        g = _check_graph(offsets, cols)
        self._check_f32(cols, weights)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        st = Stats()
        self._raise(self._lib.gsl_gsllpa_f32(self._h, ctypes.byref(g), _ptr(weights), float(tolerance),
                                             int(max_iters), int(mode), _ptr(out), ctypes.byref(st), _stream(stream)))
        return (out, st.as_dict()) if stats else out

    def modularity_f32(self, offsets, cols, labels, weights, stream=None):
        g = _check_graph(offsets, cols)
        self._check_f32(cols, weights)
        q = ctypes.c_double()
        self._raise(self._lib.gsl_modularity_f32(self._h, ctypes.byref(g), _ptr(weights), _ptr(labels),
                                                 ctypes.byref(q), _stream(stream)))
        return q.value

    def split(self, offsets, cols, labels, renumber=False, out=None, stream=None):
        import torch
        g = _check_graph(offsets, cols)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        k = ctypes.c_int64()
        rc = self._lib.gsl_split(self._h, ctypes.byref(g), _ptr(labels), _ptr(out), int(bool(renumber)),
                                 ctypes.byref(k), _stream(stream))
        self._raise(rc)
        return out, int(k.value)

    def split_lp(self, offsets, cols, labels, pruning=False, out=None, stream=None):
        """Algorithm 1 (SL-LP, or SL-LPP with pruning) -> (labels, sweeps)."""
        import torch
        g = _check_graph(offsets, cols)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        t = ctypes.c_int32()
        rc = self._lib.gsl_split_lp(self._h, ctypes.byref(g), _ptr(labels), _ptr(out), int(bool(pruning)),
                                    ctypes.byref(t), _stream(stream))
        self._raise(rc)
        return out, int(t.value)

    def disconnected(self, offsets, cols, labels, flags=False, stream=None):
        """Algorithm 4 -> number of disconnected communities (and, with
        flags=True, a uint8 tensor flagging them)."""
        import torch
        g = _check_graph(offsets, cols)
        f = torch.zeros(g.n, dtype=torch.uint8, device=offsets.device) if flags else None
        k = ctypes.c_int64()
        rc = self._lib.gsl_disconnected(self._h, ctypes.byref(g), _ptr(labels), _ptr(f), ctypes.byref(k),
                                        _stream(stream))
        self._raise(rc)
        return (int(k.value), f) if flags else int(k.value)

    def modularity(self, offsets, cols, labels, weights=None, stream=None):
        g = _check_graph(offsets, cols, weights)
        q = ctypes.c_double()
        rc = self._lib.gsl_modularity(self._h, ctypes.byref(g), _ptr(weights), _ptr(labels), ctypes.byref(q),
                                      _stream(stream))
        self._raise(rc)
        return q.value

    def gsllpa(self, offsets, cols, weights=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC, out=None,
               stream=None, stats=False):
        import torch
        g = _check_graph(offsets, cols, weights)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        st = Stats()
        rc = self._lib.gsl_gsllpa(self._h, ctypes.byref(g), _ptr(weights), float(tolerance), int(max_iters),
                                  int(mode), _ptr(out), ctypes.byref(st), _stream(stream))
        self._raise(rc)
        return (out, st.as_dict()) if stats else out

    def gsllpa_batch(self, offsets, cols, vptr, weights=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC,
                     out=None, stream=None, stats=False):
        """Batched GSL-LPA over graphs packed in one CSR (graph k owns vertices
        vptr[k]..vptr[k+1]-1).  Returns local labels (and per-graph sweeps)."""
        import numpy as np
        import torch
        g = _check_graph(offsets, cols, weights)
        vp = np.ascontiguousarray(np.asarray(vptr, dtype=np.int64))
        ng = int(vp.shape[0] - 1)
        if out is None:
            out = torch.empty(g.n, dtype=torch.int32, device=offsets.device)
        iters = np.zeros(max(ng, 1), dtype=np.int32)
        bs = BatchStats()
        rc = self._lib.gsl_gsllpa_batch(self._h, ctypes.byref(g), ng, vp.ctypes.data_as(ctypes.c_void_p), _ptr(weights),
                                        float(tolerance), int(max_iters), int(mode), _ptr(out),
                                        iters.ctypes.data_as(ctypes.c_void_p), ctypes.byref(bs), _stream(stream))
        self._raise(rc)
        if stats:
            return out, iters[:ng].copy(), {"ms": bs.ms, "graph_launches": bs.graph_launches}
        return out, iters[:ng].copy()

    def gsllpa_host(self, offsets, cols, weights=None, tolerance=0.05, max_iters=20, mode=MODE_SYNC, out=None,
                    stream=None, stats=False):
        """GSL-LPA on host tensors/arrays (CPU torch tensors, pinned preferred);
        the copies to and from the device happen inside the call."""
        import torch
        offsets = torch.as_tensor(offsets)
        cols = torch.as_tensor(cols)
        if offsets.dtype != torch.int64 or cols.dtype != torch.int32 or offsets.is_cuda or cols.is_cuda:
            raise TypeError("host offsets int64 and cols int32 expected")
        n = offsets.numel() - 1
        if out is None:
            out = torch.empty(n, dtype=torch.int32)
        if weights is not None:
            weights = torch.as_tensor(weights)
        st = Stats()
        rc = self._lib.gsl_gsllpa_host(self._h, n, cols.numel(), _ptr(offsets), _ptr(cols), _ptr(weights),
                                       float(tolerance), int(max_iters), int(mode), _ptr(out), ctypes.byref(st),
                                       _stream(stream))
        self._raise(rc)
        return (out, st.as_dict()) if stats else out


class Server:
    """Continuous-batching request server (see gsl_server_* in include/gsllpa.h).
    Graphs are host arrays (numpy int64 offsets, int32 cols) that must stay
    alive until their wait() returns; the server keeps a reference."""

    def __init__(self, device=0, slots=2, slot_vertices=0, slot_entries=0, memory_fraction=0.5,
                 max_batch_graphs=0, tolerance=0.05, max_iters=20, mode=MODE_SYNC):
        import threading as _th
        self._lib = load()
        cfg = ServerConfig(device=device, slots=slots, slot_vertices=slot_vertices, slot_entries=slot_entries,
                           memory_fraction=memory_fraction, max_batch_graphs=max_batch_graphs, mode=mode,
                           tolerance=tolerance, max_iters=max_iters)
        self._h = ctypes.c_void_p()
        rc = self._lib.gsl_server_create(ctypes.byref(self._h), ctypes.byref(cfg))
        if rc != 0:
            raise GslError(rc, self._lib.gsl_strerror(rc).decode())
        self._keep = {}
        self._keep_lock = _th.Lock()

    def capacity(self):
        v, e = ctypes.c_int64(), ctypes.c_int64()
        self._lib.gsl_server_capacity(self._h, ctypes.byref(v), ctypes.byref(e))
        return v.value, e.value

    def submit(self, offsets, cols):
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        col = np.ascontiguousarray(cols, dtype=np.int32)
        rid = ctypes.c_int64()
        rc = self._lib.gsl_server_submit(self._h, off.shape[0] - 1, col.shape[0], off.ctypes.data_as(ctypes.c_void_p),
                                         col.ctypes.data_as(ctypes.c_void_p) if col.shape[0] else None,
                                         ctypes.byref(rid))
        if rc != 0:
            raise GslError(rc, self._lib.gsl_strerror(rc).decode())
        with self._keep_lock:
            self._keep[rid.value] = (off, col)
        return rid.value

    def wait(self, rid, info=False):
        import numpy as np
        with self._keep_lock:
            off, _ = self._keep[rid]
        n = off.shape[0] - 1
        out = np.empty(max(n, 1), dtype=np.int32)
        ri = RequestInfo()
        rc = self._lib.gsl_server_wait(self._h, rid, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ri))
        with self._keep_lock:
            self._keep.pop(rid, None)
        if rc != 0:
            raise GslError(rc, self._lib.gsl_strerror(rc).decode())
        lab = out[:n]
        if info:
            return lab, {"sweeps": ri.sweeps, "batch_graphs": ri.batch_graphs, "queue_ms": ri.queue_ms,
                         "service_ms": ri.service_ms, "latency_ms": ri.latency_ms, "h2d_ms": ri.h2d_ms,
                         "compute_ms": ri.compute_ms, "d2h_ms": ri.d2h_ms}
        return lab

    def stats(self):
        st = ServerStats()
        self._lib.gsl_server_get_stats(self._h, ctypes.byref(st))
        return {"completed": st.completed, "batches": st.batches, "queued": st.queued,
                "max_concurrent_batches": st.max_concurrent_batches}

    def close(self):
        if self._h:
            self._lib.gsl_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass


_default = {}


def _ctx(device=None) -> Context:
    import torch
    d = torch.cuda.current_device() if device is None else int(device)
    with _lock:
        if d not in _default:
            _default[d] = None
    if _default[d] is None:
        _default[d] = Context(d)
    return _default[d]


def lpa(offsets, cols, weights=None, **kw):
    return _ctx(offsets.device.index).lpa(offsets, cols, weights, **kw)


def split(offsets, cols, labels, **kw):
    return _ctx(offsets.device.index).split(offsets, cols, labels, **kw)


def modularity(offsets, cols, labels, weights=None, **kw):
    return _ctx(offsets.device.index).modularity(offsets, cols, labels, weights, **kw)


def gsllpa(offsets, cols, weights=None, **kw):
    return _ctx(offsets.device.index).gsllpa(offsets, cols, weights, **kw)


def gsllpa_host(offsets, cols, weights=None, device=0, **kw):
    return _ctx(device).gsllpa_host(offsets, cols, weights, **kw)
