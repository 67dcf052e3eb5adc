"""Python binding of librambo (include/rambo.h): argument marshalling only.

Every step of insertion and query runs in the library's CUDA kernels.  Inputs
are numpy arrays (host memory) or CUDA torch tensors (device memory); PyTorch
is used only to hold device buffers and to name the current stream.  There is
no CPU fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

from . import build as _build

OK, EINVAL, ERANGE, EBADSEQ, ENOMEM, ENOSPC, ECUDA, ETIMEOUT, EIO, ESTATE, E2BIG = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10

_u64, _u32, _u16, _i32, _p = C.c_uint64, C.c_uint32, C.c_uint16, C.c_int, C.c_void_p


class RamboInfo(C.Structure):
    _fields_ = [("K", _u64), ("B", _u32), ("R", _u32), ("eta", _u32), ("L", _u32), ("m", _u64), ("seed", _u64),
                ("row_words", _u32), ("row_stride", _u32), ("index_bytes", _u64), ("n_registered", _u64),
                ("nodes", _u32), ("cells_per_node", _u32), ("tau_seed", _u64)]


class QueryStats(C.Structure):
    _fields_ = [("n_queries", _u64), ("keys_submitted", _u64), ("keys_probed", _u64), ("rows_read", _u64),
                ("n_results", _u64), ("kernel_launches", _u64), ("query_kernel_ms", C.c_float),
                ("device_ms", C.c_float), ("stage_queries", _u64 * 4), ("staged_words", _u64)]


class ServerConfig(C.Structure):
    _fields_ = [("slots", _u32), ("max_batch_queries", _u64), ("max_batch_bases", _u64), ("max_batch_keys", _u64),
                ("max_batch_ids", _u64), ("k", _u32), ("idle_wait_us", _u32)]


class ServerStats(C.Structure):
    _fields_ = [("queries", _u64), ("batches", _u64), ("inserts", _u64), ("keys", _u64), ("seconds", C.c_double),
                ("p50_ns", _u64), ("p99_ns", _u64), ("max_ns", _u64), ("admit_ns", _u64), ("finish_ns", _u64),
                ("insert_ns", _u64), ("idle_ns", _u64), ("deferred", _u64)]


class QueryConfig(C.Structure):
    _fields_ = [("lanes_per_key", _u32), ("words_per_lane", _u32), ("warps_per_block", _u32),
                ("blocks_per_sm", _u32), ("set_stage", _u32), ("visit_order", _u32), ("l2_fetch_bytes", _u32),
                ("cluster", _u32), ("row_load", _u32), ("warps_per_query", _u32), ("host_chunks", _u32),
                ("answer_staging", _u32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


# every symbol the header declares, with (restype, argtypes)
SIGNATURES = {
    "rambo_create": (_i32, [_u64, _u32, _u32, _u64, _u32, _u64, C.POINTER(_p)]),
    "rambo_destroy": (None, [_p]),
    "rambo_create_stacked": (_i32, [_u64, _u32, _u32, _u32, _u64, _u32, _u64, _u64, C.POINTER(_p)]),
    "rambo_node_of": (_u32, [_p, _u64]),
    "rambo_merge": (_i32, [_p, _p, _p]),
    "rambo_get_info": (_i32, [_p, C.POINTER(RamboInfo)]),
    "rambo_insert_batch": (_i32, [_p, _p, _p, _p, _u64, _i32, _p]),
    "rambo_insert": (_i32, [_p, _u64, _p, _u64, _i32, _p]),
    "rambo_suggest_params": (_i32, [_u64, C.c_double, C.c_double, C.c_double, C.c_double, C.POINTER(_u32),
                                    C.POINTER(_u32), C.POINTER(_u64), C.POINTER(_u32)]),
    "rambo_suggest_params_from_sample": (_i32, [_u64, _i32, _p, _p, _u64, _u32, C.c_double, C.c_double, C.c_double,
                                                C.POINTER(_u32), C.POINTER(_u32), C.POINTER(_u64), C.POINTER(_u32),
                                                C.POINTER(C.c_double)]),
    "rambo_insert_seq_batch": (_i32, [_p, _p, _p, _p, _u64, _u32, _i32, _p]),
    "rambo_query_batch": (_i32, [_p, _p, _p, _u64, _i32, C.POINTER(_p), C.POINTER(_p), _p]),
    "rambo_query_seq_batch": (_i32, [_p, _p, _p, _u64, _u32, _i32, C.POINTER(_p), C.POINTER(_p), _p]),
    "rambo_query_batch_into": (_i32, [_p, _p, _p, _u64, _i32, _p, _u64, _p, C.POINTER(_u64), _p]),
    "rambo_query_seq_batch_into": (_i32, [_p, _p, _p, _u64, _u32, _i32, _p, _u64, _p, C.POINTER(_u64), _p]),
    "rambo_query_seq_batch_noalloc": (_i32, [_p, _p, _p, _u64, _u32, _p, _u64, _p, C.POINTER(_u64), _p]),
    "rambo_export_index": (_i32, [_p, _p, _u64]),
    "rambo_export_registered": (_i32, [_p, _p, _u64]),
    "rambo_export_partition": (_i32, [_p, _p, _u64]),
    "rambo_cell_popcount": (_i32, [_p, _p, _p]),
    "rambo_fold": (_i32, [_p, _p]),
    "rambo_last_query_stats": (_i32, [_p, C.POINTER(QueryStats)]),
    "rambo_get_query_config": (_i32, [_p, C.POINTER(QueryConfig)]),
    "rambo_set_query_config": (_i32, [_p, C.POINTER(QueryConfig)]),
    "rambo_list_query_configs": (_i32, [_p, _p, _i32]),
    "rambo_set_build_tiling": (_i32, [_p, _u64, _i32]),
    "rambo_query_one_per_launch": (_i32, [_p, _i32, _p, _p, _u64, _u32, _p, _p, _p]),
    "rambo_plan_create": (_i32, [_p, _i32, _u64, _u64, _u64, _u32, C.POINTER(_p)]),
    "rambo_plan_destroy": (None, [_p]),
    "rambo_plan_buffers": (_i32, [_p, C.POINTER(_p), C.POINTER(_p), C.POINTER(_p), C.POINTER(_p)]),
    "rambo_plan_launch": (_i32, [_p, _u64, _u64, _i32, _p]),
    "rambo_plan_poll": (_i32, [_p]),
    "rambo_plan_wait": (_i32, [_p, _i32, C.POINTER(_p), C.POINTER(_p), C.POINTER(_u64), _p]),
    "rambo_plan_launches_per_replay": (_i32, [_p]),
    "rambo_plan_last_stats": (_i32, [_p, C.POINTER(QueryStats)]),
    "rambo_plan_set_timing": (_i32, [_p, _i32]),
    "rambo_server_create": (_i32, [_p, C.POINTER(ServerConfig), C.POINTER(_p)]),
    "rambo_server_submit": (_i32, [_p, _i32, _p, _u64, C.POINTER(_u64)]),
    "rambo_server_submit_insert": (_i32, [_p, _i32, _p, _p, _p, _u64, C.POINTER(_u64)]),
    "rambo_server_result": (_i32, [_p, _u64, _i32, _p, _u64, C.POINTER(_u64), C.POINTER(_u64)]),
    "rambo_server_drain": (_i32, [_p]),
    "rambo_server_stats": (_i32, [_p, C.POINTER(ServerStats)]),
    "rambo_server_reset_stats": (_i32, [_p]),
    "rambo_server_replay": (_i32, [_p, _p, _p, _p, _p, _u64, _p]),
    "rambo_server_inject_alloc_failures": (_i32, [_p, _u32]),
    "rambo_server_destroy": (None, [_p]),
    "rambo_autotune": (_i32, [_p, _i32, _p, _p, _u64, _u32, _i32, _i32, C.POINTER(QueryConfig), _p]),
    "rambo_save": (_i32, [_p, C.c_char_p]),
    "rambo_load": (_i32, [C.c_char_p, C.POINTER(_p)]),
    "rambo_random_row_probe": (_i32, [_p, _u64, _u32, _u64, _u32, _u32, _u64, _u32, C.POINTER(C.c_float), _p]),
    "rambo_l2_fetch_granularity": (_i32, [_u32, C.POINTER(_u32)]),
    "rambo_last_error_item": (_u64, [_p]),
    "rambo_strerror": (C.c_char_p, [_i32]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Loads librambo.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"librambo.so is not built ({_build.LIB}); run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RamboError(RuntimeError):
    def __init__(self, code: int, where: str = "", item: int | None = None):
        msg = load_library().rambo_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})" + (f" at item {item}" if item is not None else ""))
        self.code = code
        self.item = item


def _torch():
    import torch

    return torch


def _is_cuda_tensor(x) -> bool:
    try:
        torch = _torch()
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            torch = _torch()
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _CudaArray:
    """Exposes a device pointer through __cuda_array_interface__ so torch can
    copy it into a tensor it owns."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


def _device_copy(ptr: int, n: int, dtype: str, copy: bool = True):
    """A torch CUDA tensor over n elements at ptr: a copy, or (copy=False) a
    view that is valid while the memory is (the handle's result arena: until
    the next query call)."""
    torch = _torch()
    tdt = {"<u4": torch.int32, "<u8": torch.int64}[dtype]
    if n == 0:
        return torch.zeros(0, dtype=tdt, device="cuda")
    t = torch.as_tensor(_CudaArray(ptr, n, "<i4" if dtype == "<u4" else "<i8"), device="cuda")
    return t.clone() if copy else t


def _host_arr(x, dtype) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=dtype)


def _check_csr(data: np.ndarray, off: np.ndarray, what: str) -> None:
    """The C ABI reads data[offsets[0] .. offsets[n]); refuse host arrays that
    are shorter than that before handing pointers over."""
    if off.size < 1:
        raise ValueError(f"{what}: offsets must have n+1 >= 1 entries")
    if off.size > 1 and int(off[-1]) > data.size and int(off[-1]) >= int(off[0]):
        raise ValueError(f"{what}: offsets[-1]={int(off[-1])} exceeds the data length {data.size}")


class Rambo:
    """A RAMBO index resident in GPU memory (Secs. 2-3 of arXiv 1910.02611)."""

    def __init__(self, K: int, B: int, R: int, m: int, eta: int, seed: int = 42, *, _handle=None):
        L = load_library()
        if _handle is None:
            h = _p()
            rc = L.rambo_create(K, B, R, m, eta, seed, C.byref(h))
            if rc:
                raise RamboError(rc, "rambo_create")
            self._h = h
        else:
            self._h = _handle
        # plans and servers created over this index, closed before it is
        # (their captured graphs and worker threads use its memory)
        self._dependents = weakref.WeakSet()
        info = self.info()
        self.K, self.B, self.R, self.m, self.eta, self.seed = info.K, info.B, info.R, info.m, info.eta, info.seed
        self.row_stride = info.row_stride
        self.row_words = info.row_words

    @classmethod
    def stacked(cls, K: int, cells_per_node: int, nodes: int, R: int, m: int, eta: int, seed: int = 42,
                tau_seed: int = 0) -> "Rambo":
        """Two-level hash (Sec. 5.2): nodes x cells_per_node cells, set i in node tau(i)."""
        h = _p()
        rc = load_library().rambo_create_stacked(K, cells_per_node, nodes, R, m, eta, seed, tau_seed, C.byref(h))
        if rc:
            raise RamboError(rc, "rambo_create_stacked")
        return cls(0, 0, 0, 0, 0, _handle=h)

    def node_of(self, set_id: int) -> int:
        return int(load_library().rambo_node_of(self._h, set_id))

    def merge(self, other: "Rambo", stream=None) -> None:
        """ORs another index with identical parameters into this one."""
        self._check(load_library().rambo_merge(self._h, other._h, _stream_handle(stream)), "merge")

    @classmethod
    def load(cls, path: str) -> "Rambo":
        h = _p()
        rc = load_library().rambo_load(path.encode(), C.byref(h))
        if rc:
            raise RamboError(rc, "rambo_load")
        return cls(0, 0, 0, 0, 0, _handle=h)

    def close(self) -> None:
        for d in list(getattr(self, "_dependents", ())):
            d.close()
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load_library().rambo_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, where: str):
        if rc:
            item = None
            if rc in (EINVAL, ERANGE, EBADSEQ):
                item = int(load_library().rambo_last_error_item(self._h))
            raise RamboError(rc, where, item)

    # -- info ---------------------------------------------------------------
    def info(self) -> RamboInfo:
        out = RamboInfo()
        rc = load_library().rambo_get_info(self._h, C.byref(out))
        if rc:
            raise RamboError(rc, "rambo_get_info")
        return out

    # -- Algorithm 1 --------------------------------------------------------------
    def insert(self, set_ids, data, offsets, kind: str = "keys", k: int = 31, stream=None) -> None:
        """Inserts sets (keys, or DNA whose k-mers are the keys) given in CSR form."""
        L = load_library()
        dev = _is_cuda_tensor(data)
        if dev:
            ids_p, data_p, off_p = set_ids.data_ptr(), data.data_ptr(), offsets.data_ptr()
            n = offsets.numel() - 1
            keep = None
        else:
            ids = _host_arr(set_ids, np.uint64)
            d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
            off = _host_arr(offsets, np.uint64)
            _check_csr(d, off, "insert")
            if ids.size != off.size - 1:
                raise ValueError("insert: need one set ID per CSR item")
            keep = (ids, d, off)
            ids_p, data_p, off_p = ids.ctypes.data, d.ctypes.data, off.ctypes.data
            n = off.size - 1
        s = _stream_handle(stream)
        if kind == "keys":
            rc = L.rambo_insert_batch(self._h, ids_p, data_p, off_p, n, int(dev), s)
        else:
            rc = L.rambo_insert_seq_batch(self._h, ids_p, data_p, off_p, n, k, int(dev), s)
        del keep
        self._check(rc, "insert")

    def insert_set(self, set_id: int, keys, stream=None) -> None:
        """Algorithm 1 for one set of keys (rambo_insert)."""
        dev = _is_cuda_tensor(keys)
        if dev:
            rc = load_library().rambo_insert(self._h, set_id, keys.data_ptr(), keys.numel(), 1, _stream_handle(stream))
        else:
            k = _host_arr(keys, np.uint64)
            rc = load_library().rambo_insert(self._h, set_id, k.ctypes.data, k.size, 0, _stream_handle(stream))
        self._check(rc, "insert_set")

    # -- Algorithm 2 ----------------------------------------------------------------
    def query(self, data, offsets, kind: str = "keys", k: int = 31, stream=None, copy: bool = True):
        """Returns (ids, id_offsets): numpy arrays for host inputs, torch CUDA
        tensors for device inputs.  Query q's answer is ids[id_offsets[q]:id_offsets[q+1]].
        With copy=False the arrays are views of the handle's result arena
        (pinned host or device memory), valid until the next query call."""
        L = load_library()
        dev = _is_cuda_tensor(data)
        if dev:
            data_p, off_p, n = data.data_ptr(), offsets.data_ptr(), offsets.numel() - 1
            keep = None
        else:
            d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
            off = _host_arr(offsets, np.uint64)
            _check_csr(d, off, "query")
            keep = (d, off)
            data_p, off_p, n = d.ctypes.data, off.ctypes.data, off.size - 1
        ids_p, offo_p = _p(), _p()
        s = _stream_handle(stream)
        if kind == "keys":
            rc = L.rambo_query_batch(self._h, data_p, off_p, n, int(dev), C.byref(ids_p), C.byref(offo_p), s)
        else:
            rc = L.rambo_query_seq_batch(self._h, data_p, off_p, n, k, int(dev), C.byref(ids_p), C.byref(offo_p), s)
        del keep
        self._check(rc, "query")
        if dev:
            off_t = _device_copy(offo_p.value, n + 1, "<u8", copy)
            total = int(off_t[-1].item())
            return _device_copy(ids_p.value or 0, total, "<u4", copy), off_t
        offs = np.ctypeslib.as_array(C.cast(offo_p, C.POINTER(_u64)), shape=(n + 1,))
        offs = offs.copy() if copy else offs
        total = int(offs[-1])
        if total == 0:
            return np.zeros(0, np.uint32), offs
        ids = np.ctypeslib.as_array(C.cast(ids_p, C.POINTER(_u32)), shape=(total,))
        return (ids.copy() if copy else ids), offs

    def query_into(self, data, offsets, ids_out, id_offsets_out, kind: str = "keys", k: int = 31, stream=None) -> int:
        """Writes results into caller buffers (numpy or CUDA tensors).  Returns
        the number of IDs; raises RamboError(ENOSPC) if ids_out is too small."""
        L = load_library()
        dev = _is_cuda_tensor(data)
        needed = _u64(0)
        s = _stream_handle(stream)
        if dev:
            args = (data.data_ptr(), offsets.data_ptr(), offsets.numel() - 1)
            ids_p, cap, oo = ids_out.data_ptr(), ids_out.numel(), id_offsets_out.data_ptr()
        else:
            d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
            off = _host_arr(offsets, np.uint64)
            _check_csr(d, off, "query_into")
            args = (d.ctypes.data, off.ctypes.data, off.size - 1)
            assert ids_out.dtype == np.uint32 and id_offsets_out.dtype == np.uint64
            ids_p, cap, oo = ids_out.ctypes.data, ids_out.size, id_offsets_out.ctypes.data
        if kind == "keys":
            rc = L.rambo_query_batch_into(self._h, *args, int(dev), ids_p, cap, oo, C.byref(needed), s)
        else:
            rc = L.rambo_query_seq_batch_into(self._h, *args, k, int(dev), ids_p, cap, oo, C.byref(needed), s)
        if rc == ENOSPC:
            raise RamboError(rc, "query_into (item = IDs needed)", int(needed.value))
        self._check(rc, "query_into")
        return int(needed.value)

    def query_seq_noalloc(self, bases, offsets, ids_out, id_offsets_out, k: int = 31, stream=None) -> int:
        """Sequence query through the entry point that allocates nothing (all
        arguments CUDA tensors owned by the caller; the library's fixed device
        array holds the working memory).  Returns the number of IDs written."""
        needed = _u64(0)
        rc = load_library().rambo_query_seq_batch_noalloc(
            self._h, bases.data_ptr(), offsets.data_ptr(), offsets.numel() - 1, k, ids_out.data_ptr(),
            ids_out.numel(), id_offsets_out.data_ptr(), C.byref(needed), _stream_handle(stream))
        self._check(rc, "query_seq_noalloc")
        return int(needed.value)

    def query_one_per_launch(self, data, host_offsets, kind: str = "seq", k: int = 31, stream=None):
        """The plain one-query-per-launch baseline (one thread block launched per
        query).  data: CUDA tensor; host_offsets: numpy.  Returns (ids, offsets)
        as numpy arrays in the same CSR form as query()."""
        torch = _torch()
        off = _host_arr(host_offsets, np.uint64)
        n = off.size - 1
        ids = torch.empty(max(n, 1) * self.K, dtype=torch.int32, device=data.device)
        cnt = torch.empty(max(n, 1), dtype=torch.int32, device=data.device)
        rc = load_library().rambo_query_one_per_launch(self._h, 0 if kind == "keys" else 1, data.data_ptr(),
                                                       off.ctypes.data, n, k, ids.data_ptr(), cnt.data_ptr(),
                                                       _stream_handle(stream))
        self._check(rc, "query_one_per_launch")
        counts = cnt[:n].cpu().numpy().astype(np.uint64)
        out_off = np.zeros(n + 1, np.uint64)
        np.cumsum(counts, out=out_off[1:])
        per = ids[: n * self.K].view(n, self.K).cpu().numpy().view(np.uint32) if n else np.zeros((0, self.K), np.uint32)
        flat = np.concatenate([per[q, : int(counts[q])] for q in range(n)]) if n else np.zeros(0, np.uint32)
        return flat.astype(np.uint32), out_off

    def autotune(self, data, offsets, kind: str = "seq", k: int = 31, reps: int = 3, stream=None) -> dict:
        """Times every kernel configuration on a sample batch, keeps the fastest."""
        dev = _is_cuda_tensor(data)
        if dev:
            dp, op, n = data.data_ptr(), offsets.data_ptr(), offsets.numel() - 1
            keep = None
        else:
            d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
            off = _host_arr(offsets, np.uint64)
            _check_csr(d, off, "autotune")
            keep = (d, off)
            dp, op, n = d.ctypes.data, off.ctypes.data, off.size - 1
        best = QueryConfig()
        rc = load_library().rambo_autotune(self._h, 0 if kind == "keys" else 1, dp, op, n, k, int(dev), reps,
                                           C.byref(best), _stream_handle(stream))
        del keep
        self._check(rc, "autotune")
        return best.as_dict()

    def last_query_stats(self) -> dict:
        st = QueryStats()
        self._check(load_library().rambo_last_query_stats(self._h, C.byref(st)), "last_query_stats")
        out = {}
        for f, _ in st._fields_:
            v = getattr(st, f)
            out[f] = float(v) if f.endswith("_ms") else (list(v) if f == "stage_queries" else int(v))
        return out

    # -- configuration ------------------------------------------------------------
    def get_config(self) -> dict:
        c = QueryConfig()
        load_library().rambo_get_query_config(self._h, C.byref(c))
        return c.as_dict()

    def set_config(self, **kw) -> None:
        cur = self.get_config()
        cur.update(kw)
        c = QueryConfig(**cur)
        self._check(load_library().rambo_set_query_config(self._h, C.byref(c)), "set_config")

    def set_build_tiling(self, tile_bytes: int = 0, mode: int = 0) -> None:
        """mode 0 auto, 1 always window by window (L2-resident slices of
        tile_bytes), 2 single pass, 3 keys hashed once per input chunk with
        their updates filed and applied by window."""
        self._check(load_library().rambo_set_build_tiling(self._h, tile_bytes, mode), "set_build_tiling")

    def list_configs(self) -> list[dict]:
        L = load_library()
        n = L.rambo_list_query_configs(self._h, None, 0)
        arr = (QueryConfig * max(n, 1))()
        L.rambo_list_query_configs(self._h, C.cast(arr, _p), n)
        return [arr[i].as_dict() for i in range(n)]

    # -- inspection -----------------------------------------------------------------
    def export_index(self) -> np.ndarray:
        """Rows as uint32 [R, m, row_stride] (bit b of row (r,p) = bit p of cell b's filter)."""
        n = self.R * self.m * self.row_stride
        out = np.empty(n, np.uint32)
        self._check(load_library().rambo_export_index(self._h, out.ctypes.data, n), "export_index")
        return out.reshape(self.R, self.m, self.row_stride)

    def export_registered(self) -> np.ndarray:
        n = (self.K + 31) // 32
        out = np.empty(n, np.uint32)
        self._check(load_library().rambo_export_registered(self._h, out.ctypes.data, n), "export_registered")
        return np.unpackbits(out.view(np.uint8), bitorder="little")[: self.K].astype(bool)

    def export_partition(self) -> np.ndarray:
        n = self.K * self.R
        out = np.empty(n, np.uint16)
        self._check(load_library().rambo_export_partition(self._h, out.ctypes.data, n), "export_partition")
        return out.reshape(self.K, self.R)

    def cell_popcount(self, stream=None) -> np.ndarray:
        out = np.zeros(self.R * self.B, np.uint64)
        self._check(load_library().rambo_cell_popcount(self._h, out.ctypes.data, _stream_handle(stream)),
                    "cell_popcount")
        return out.reshape(self.R, self.B)

    def fold(self, stream=None) -> None:
        """Folding over: B -> B/2 by OR-ing cell b + B/2 onto cell b."""
        self._check(load_library().rambo_fold(self._h, _stream_handle(stream)), "fold")
        info = self.info()
        self.B, self.row_stride, self.row_words = info.B, info.row_stride, info.row_words

    def save(self, path: str) -> None:
        self._check(load_library().rambo_save(self._h, path.encode()), "save")


class Plan:
    """A graph-captured query plan (see rambo_plan_create): fixed buffers and a
    CUDA graph replayed for every batch up to the plan's capacity."""

    def __init__(self, index: "Rambo", kind: str, max_queries: int, max_items: int, max_ids: int, k: int = 31):
        L = load_library()
        self._index = index  # keeps the index alive while the plan exists
        self.kind = kind
        self.max_queries, self.max_items, self.max_ids = max_queries, max_items, max_ids
        h = _p()
        rc = L.rambo_plan_create(index._h, 0 if kind == "keys" else 1, max_queries, max_items, max_ids, k, C.byref(h))
        if rc:
            raise RamboError(rc, "rambo_plan_create")
        self._p = h
        index._dependents.add(self)
        hd, ho, dd, do = _p(), _p(), _p(), _p()
        L.rambo_plan_buffers(h, C.byref(hd), C.byref(ho), C.byref(dd), C.byref(do))
        self._elem = 8 if kind == "keys" else 1
        dt = np.uint64 if kind == "keys" else np.uint8
        self.host_data = np.ctypeslib.as_array(C.cast(hd, C.POINTER(C.c_uint64 if kind == "keys" else C.c_uint8)),
                                               shape=(max_items,)).view(dt)
        self.host_offsets = np.ctypeslib.as_array(C.cast(ho, C.POINTER(_u64)), shape=(max_queries + 1,))
        self.dev_data_ptr, self.dev_offsets_ptr = dd.value, do.value
        self.launches_per_replay = int(L.rambo_plan_launches_per_replay(h))
        self._n = 0

    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            load_library().rambo_plan_destroy(self._p)
        self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_host(self, data, offsets, stream=None) -> None:
        """Copies a batch into the plan's pinned buffers and launches it (async)."""
        d = _host_arr(data, np.uint64 if self.kind == "keys" else np.uint8)
        off = _host_arr(offsets, np.uint64)
        n = off.size - 1
        base = int(off[0])
        items = int(off[-1]) - base
        if n > self.max_queries or items > self.max_items:
            # the library rejects a batch beyond capacity before touching any buffer
            rc = load_library().rambo_plan_launch(self._p, n, items, 1, _stream_handle(stream))
            raise RamboError(rc if rc else EINVAL, "rambo_plan_launch")
        self.host_data[:items] = d[base: base + items]
        self.host_offsets[: n + 1] = off - np.uint64(base)
        self._n = n
        rc = load_library().rambo_plan_launch(self._p, n, items, 1, _stream_handle(stream))
        if rc:
            raise RamboError(rc, "rambo_plan_launch")

    def launch_device(self, n_queries: int, n_items: int, stream=None) -> None:
        """Launches a batch already written to the plan's device buffers."""
        self._n = n_queries
        rc = load_library().rambo_plan_launch(self._p, n_queries, n_items, 0, _stream_handle(stream))
        if rc:
            raise RamboError(rc, "rambo_plan_launch")

    def poll(self) -> bool:
        rc = load_library().rambo_plan_poll(self._p)
        if rc < 0:
            raise RamboError(rc, "rambo_plan_poll")
        return rc == 0

    def wait(self, to_host: bool = True, stream=None, copy: bool = True):
        """Results of the launched batch.  copy=False with to_host=False returns
        (ids device pointer, offsets device pointer, number of IDs) only."""
        ids_p, off_p, n_ids = _p(), _p(), _u64(0)
        rc = load_library().rambo_plan_wait(self._p, int(to_host), C.byref(ids_p), C.byref(off_p), C.byref(n_ids),
                                            _stream_handle(stream))
        if rc:
            raise RamboError(rc, "rambo_plan_wait", int(n_ids.value) if rc == ENOSPC else None)
        n = self._n
        total = int(n_ids.value)
        if not copy and not to_host:
            return ids_p.value, off_p.value, total
        if to_host:
            offs = np.ctypeslib.as_array(C.cast(off_p, C.POINTER(_u64)), shape=(n + 1,)).copy()
            ids = (np.ctypeslib.as_array(C.cast(ids_p, C.POINTER(_u32)), shape=(total,)).copy() if total
                   else np.zeros(0, np.uint32))
            return ids, offs
        return _device_copy(ids_p.value or 0, total, "<u4"), _device_copy(off_p.value, n + 1, "<u8")

    def set_timing(self, on: bool) -> None:
        """Replay the graph with (True, default) or without (False) its timing
        nodes (rambo_plan_set_timing)."""
        rc = load_library().rambo_plan_set_timing(self._p, int(on))
        if rc:
            raise RamboError(rc, "rambo_plan_set_timing")

    def last_stats(self) -> dict:
        """Counters and CUDA-event times of the last waited batch (rambo_plan_last_stats)."""
        st = QueryStats()
        rc = load_library().rambo_plan_last_stats(self._p, C.byref(st))
        if rc:
            raise RamboError(rc, "rambo_plan_last_stats")
        out = {}
        for f, _ in st._fields_:
            v = getattr(st, f)
            out[f] = float(v) if f.endswith("_ms") else (list(v) if f == "stage_queries" else int(v))
        return out


class Server:
    """Continuous-batching query server over an index (rambo_server_*)."""

    def __init__(self, index: "Rambo", slots: int = 3, max_batch_queries: int = 4096, max_batch_bases: int = 1 << 22,
                 max_batch_keys: int = 1 << 16, max_batch_ids: int = 1 << 22, k: int = 31, idle_wait_us: int = 20):
        cfg = ServerConfig(slots, max_batch_queries, max_batch_bases, max_batch_keys, max_batch_ids, k, idle_wait_us)
        h = _p()
        rc = load_library().rambo_server_create(index._h, C.byref(cfg), C.byref(h))
        if rc:
            raise RamboError(rc, "rambo_server_create")
        self._s = h
        self._index = index
        index._dependents.add(self)
        self.max_batch_ids = max_batch_ids

    def submit(self, data, kind: str = "seq") -> int:
        d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
        t = _u64(0)
        rc = load_library().rambo_server_submit(self._s, 0 if kind == "keys" else 1, d.ctypes.data, d.size, C.byref(t))
        if rc:
            raise RamboError(rc, "rambo_server_submit")
        return int(t.value)

    def submit_insert(self, set_ids, data, offsets, kind: str = "keys") -> int:
        ids = _host_arr(set_ids, np.uint64)
        d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
        off = _host_arr(offsets, np.uint64)
        _check_csr(d, off, "submit_insert")
        t = _u64(0)
        rc = load_library().rambo_server_submit_insert(self._s, 0 if kind == "keys" else 1, ids.ctypes.data,
                                                       d.ctypes.data, off.ctypes.data, ids.size, C.byref(t))
        if rc:
            raise RamboError(rc, "rambo_server_submit_insert")
        return int(t.value)

    def result(self, ticket: int, wait: bool = True):
        """(ids, latency_ns) once done; None if pending and wait is False."""
        L = load_library()
        cap = 1 << 16
        while True:
            buf = np.empty(cap, np.uint32)
            n, lat = _u64(0), _u64(0)
            rc = L.rambo_server_result(self._s, ticket, int(wait), buf.ctypes.data, cap, C.byref(n), C.byref(lat))
            if rc == 1:
                return None
            if rc == ENOSPC and int(n.value) > cap:
                cap = int(n.value)
                continue
            if rc:
                raise RamboError(rc, "rambo_server_result")
            return buf[: n.value], int(lat.value)

    def drain(self) -> None:
        load_library().rambo_server_drain(self._s)

    def stats(self) -> dict:
        st = ServerStats()
        load_library().rambo_server_stats(self._s, C.byref(st))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def reset_stats(self) -> None:
        load_library().rambo_server_reset_stats(self._s)

    def replay(self, kinds: np.ndarray, payload: np.ndarray, byte_offsets: np.ndarray, arrival_ns: np.ndarray):
        """Submits requests at the given arrival times (native load generator);
        returns their tickets."""
        k = _host_arr(kinds, np.uint8)
        b = _host_arr(payload, np.uint8)
        o = _host_arr(byte_offsets, np.uint64)
        a = _host_arr(arrival_ns, np.uint64)
        t = np.zeros(k.size, np.uint64)
        rc = load_library().rambo_server_replay(self._s, k.ctypes.data, b.ctypes.data, o.ctypes.data, a.ctypes.data,
                                                k.size, t.ctypes.data)
        if rc:
            raise RamboError(rc, "rambo_server_replay")
        return t

    def inject_alloc_failures(self, n: int) -> None:
        """Refuse the next n pinned allocations for answers (testing the deferral path)."""
        rc = load_library().rambo_server_inject_alloc_failures(self._s, n)
        if rc:
            raise RamboError(rc, "rambo_server_inject_alloc_failures")

    def close(self) -> None:
        if getattr(self, "_s", None) is not None and self._s.value:
            load_library().rambo_server_destroy(self._s)
        self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def suggest_params(K: int, n_mean: float, V: float = 1.0, p: float = 0.01, delta: float = 0.01) -> dict:
    """Parameter chooser (Lemma 4.4 for B, Lemma 4.2 for R, Bloom-filter sizing
    for m and eta); host-only.  Raises RamboError(ERANGE) if R <= RAMBO_MAX_R
    cannot reach delta (the dict is still attached as .params)."""
    B, R, m, eta = _u32(), _u32(), _u64(), _u32()
    rc = load_library().rambo_suggest_params(K, n_mean, V, p, delta, C.byref(B), C.byref(R), C.byref(m), C.byref(eta))
    out = dict(B=B.value, R=R.value, m=m.value, eta=eta.value)
    if rc:
        err = RamboError(rc, "suggest_params")
        err.params = out
        raise err
    return out


def suggest_params_from_sample(K: int, data, offsets, kind: str = "keys", k: int = 31, V: float = 1.0,
                               p: float = 0.01, delta: float = 0.01) -> dict:
    """Parameter chooser sized from a sampled prefix (Sec. 5.1): the mean
    distinct-key count of the sample's sets (CSR, host arrays) is the n_mean
    of suggest_params.  Returns the parameters and the measured n_mean."""
    d = _host_arr(data, np.uint64 if kind == "keys" else np.uint8)
    off = _host_arr(offsets, np.uint64)
    _check_csr(d, off, "suggest_params_from_sample")
    B, R, m, eta, nm = _u32(), _u32(), _u64(), _u32(), C.c_double(0.0)
    rc = load_library().rambo_suggest_params_from_sample(K, 0 if kind == "keys" else 1, d.ctypes.data,
                                                         off.ctypes.data, off.size - 1, k, V, p, delta, C.byref(B),
                                                         C.byref(R), C.byref(m), C.byref(eta), C.byref(nm))
    out = dict(B=B.value, R=R.value, m=m.value, eta=eta.value, n_mean=nm.value)
    if rc:
        err = RamboError(rc, "suggest_params_from_sample")
        err.params = out
        raise err
    return out


def l2_fetch_granularity(bytes_: int = 0) -> int:
    """Reads (and, if bytes_ > 0, sets) the CUDA context's L2 fetch
    granularity hint; returns the value before the call."""
    prev = _u32(0)
    rc = load_library().rambo_l2_fetch_granularity(bytes_, C.byref(prev))
    if rc:
        raise RamboError(rc, "l2_fetch_granularity")
    return int(prev.value)


def random_row_probe(buf, n_rows: int, row_words: int, reads_per_thread: int, blocks: int, threads: int = 256,
                     seed: int = 1, row_load: int = 0, stream=None) -> float:
    """Times the random-row read microbenchmark over a CUDA tensor; returns ms."""
    ms = C.c_float(0)
    rc = load_library().rambo_random_row_probe(buf.data_ptr(), n_rows, row_words, reads_per_thread, blocks, threads,
                                               seed, row_load, C.byref(ms), _stream_handle(stream))
    if rc:
        raise RamboError(rc, "random_row_probe")
    return float(ms.value)
