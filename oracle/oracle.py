"""ctypes wrapper of the plain CPU RAMBO in ``rambo_oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The GPU library never imports this.

The C file implements Algorithm 1 (insertion, Sec. 3.1) and Algorithm 2
(query, Sec. 3.2, with the sequence rule of Sec. 3.2.1) on B*R separate Bloom
filters (Sec. 2); see its header for the hash specification.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rambo_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OK, EINVAL, ERANGE, EBADSEQ, ENOMEM = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C + OpenMP); returns the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        u64, u32, i64, p = C.c_uint64, C.c_uint32, C.c_int64, C.c_void_p
        L.orc_create.restype = p
        L.orc_create.argtypes = [u64, u32, u32, u64, u32, u64]
        L.orc_destroy.argtypes = [p]
        L.orc_mix64.restype = u64
        L.orc_mix64.argtypes = [u64]
        L.orc_splitmix64_next.restype = u64
        L.orc_splitmix64_next.argtypes = [C.POINTER(u64)]
        L.orc_phi.restype = u32
        L.orc_phi.argtypes = [p, u32, u64]
        L.orc_pos.restype = u64
        L.orc_pos.argtypes = [p, u32, u32, u64]
        for name in ("orc_param_a", "orc_param_c"):
            getattr(L, name).restype = u64
            getattr(L, name).argtypes = [p, u32]
        L.orc_param_s.restype = u64
        L.orc_param_s.argtypes = [p, u32, u32]
        L.orc_base_code.restype = C.c_int
        L.orc_base_code.argtypes = [C.c_uint8]
        L.orc_kmers.restype = i64
        L.orc_kmers.argtypes = [p, u64, u32, p]
        L.orc_insert_keys.restype = C.c_int
        L.orc_insert_keys.argtypes = [p, u64, p, u64]
        L.orc_insert_seq.restype = C.c_int
        L.orc_insert_seq.argtypes = [p, u64, p, u64, u32]
        L.orc_insert_seq_batch.restype = C.c_int
        L.orc_insert_seq_batch.argtypes = [p, p, p, p, u64, u32, C.c_int]
        L.orc_insert_keys_batch.restype = C.c_int
        L.orc_insert_keys_batch.argtypes = [p, p, p, p, u64, C.c_int]
        L.orc_query_keys.restype = i64
        L.orc_query_keys.argtypes = [p, p, u64, p, u64]
        L.orc_query_seq.restype = i64
        L.orc_query_seq.argtypes = [p, p, u64, u32, p, u64]
        L.orc_query_batch.restype = C.c_int
        L.orc_query_batch.argtypes = [p, C.c_int, p, p, u64, u32, C.c_int, p, p, u64, p, p]
        L.orc_bf_contains.restype = C.c_int
        L.orc_bf_contains.argtypes = [p, u32, u32, u64]
        L.orc_is_registered.restype = C.c_int
        L.orc_is_registered.argtypes = [p, u64]
        L.orc_export_bf.argtypes = [p, u32, u32, p]
        L.orc_get_row.argtypes = [p, u32, u64, p]
        L.orc_cell_popcount.argtypes = [p, p]
        L.orc_export_reg.argtypes = [p, p]
        L.orc_create_stacked.restype = p
        L.orc_create_stacked.argtypes = [u64, u32, u32, u32, u64, u32, u64, u64]
        L.orc_node.restype = u32
        L.orc_node.argtypes = [p, u64]
        L.orc_fold.restype = C.c_int
        L.orc_fold.argtypes = [p]
        L.orc_merge.restype = C.c_int
        L.orc_merge.argtypes = [p, p]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z))


def splitmix64_stream(seed: int, n: int) -> list[int]:
    st = C.c_uint64(seed)
    return [int(lib().orc_splitmix64_next(C.byref(st))) for _ in range(n)]


def base_code(ch: int) -> int:
    return int(lib().orc_base_code(ch))


def kmers(seq: bytes | np.ndarray, k: int) -> np.ndarray:
    """The k-mer keys of one sequence (Sec. 3.2.1 sliding window)."""
    s = np.frombuffer(bytes(seq), dtype=np.uint8) if not isinstance(seq, np.ndarray) else np.ascontiguousarray(seq, np.uint8)
    n = lib().orc_kmers(_ptr(s), s.size, k, None)
    if n < 0:
        raise ValueError(f"orc_kmers error {n}")
    out = np.zeros(max(n, 1), np.uint64)
    lib().orc_kmers(_ptr(s), s.size, k, _ptr(out))
    return out[:n]


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"oracle error {code} {what}")
        self.code = code


class Oracle:
    """A plain RAMBO: B*R separate m-bit Bloom filters (Secs. 2-3)."""

    def __init__(self, K: int, B: int, R: int, m: int, eta: int, seed: int, *, nodes: int = 1, tau_seed: int = 0):
        """nodes > 1: the two-level hash of Sec. 5.2 with B cells per node
        (B * nodes cells in the stacked structure)."""
        self.K, self.R, self.m, self.eta, self.seed = K, R, m, eta, seed
        self.B = B * nodes
        if nodes > 1:
            h = lib().orc_create_stacked(K, B, nodes, R, m, eta, seed, tau_seed)
        else:
            h = lib().orc_create(K, B, R, m, eta, seed)
        if not h:
            raise OracleError(EINVAL, "orc_create rejected parameters")
        self._h = C.c_void_p(h)

    def node(self, set_id: int) -> int:
        return int(lib().orc_node(self._h, set_id))

    def fold(self) -> None:
        rc = lib().orc_fold(self._h)
        if rc:
            raise OracleError(rc, "fold")
        self.B //= 2

    def merge(self, other: "Oracle") -> None:
        rc = lib().orc_merge(self._h, other._h)
        if rc:
            raise OracleError(rc, "merge")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_destroy(h)
            self._h = None

    # -- hashes --------------------------------------------------------------
    def phi(self, r: int, set_id: int) -> int:
        return int(lib().orc_phi(self._h, r, set_id))

    def pos(self, r: int, j: int, key: int) -> int:
        return int(lib().orc_pos(self._h, r, j, key))

    def params(self):
        L = lib()
        a = [int(L.orc_param_a(self._h, r)) for r in range(self.R)]
        c = [int(L.orc_param_c(self._h, r)) for r in range(self.R)]
        s = [[int(L.orc_param_s(self._h, r, j)) for j in range(self.eta)] for r in range(self.R)]
        return a, c, s

    def phi_table(self) -> np.ndarray:
        return np.array([[self.phi(r, i) for r in range(self.R)] for i in range(self.K)], np.int64)

    @staticmethod
    def kmers_count(seq, k: int = 31) -> int:
        """Number of terms (windows) of a sequence, or a negative error code."""
        s = np.frombuffer(bytes(seq), np.uint8) if not isinstance(seq, np.ndarray) else np.ascontiguousarray(seq, np.uint8)
        return int(lib().orc_kmers(_ptr(s), s.size, k, None))

    # -- Algorithm 1 -----------------------------------------------------------
    def insert_keys(self, set_id: int, keys) -> None:
        k = np.ascontiguousarray(keys, dtype=np.uint64)
        rc = lib().orc_insert_keys(self._h, set_id, _ptr(k), k.size)
        if rc:
            raise OracleError(rc, "insert_keys")

    def insert_seq(self, set_id: int, seq, k: int = 31) -> None:
        s = np.frombuffer(bytes(seq), np.uint8) if not isinstance(seq, np.ndarray) else np.ascontiguousarray(seq, np.uint8)
        rc = lib().orc_insert_seq(self._h, set_id, _ptr(s), s.size, k)
        if rc:
            raise OracleError(rc, "insert_seq")

    def insert_seq_batch(self, set_ids, bases, offsets, k: int = 31, nthreads: int = 1) -> None:
        ids = np.ascontiguousarray(set_ids, np.uint64)
        b = np.ascontiguousarray(bases, np.uint8)
        off = np.ascontiguousarray(offsets, np.uint64)
        rc = lib().orc_insert_seq_batch(self._h, _ptr(ids), _ptr(b), _ptr(off), ids.size, k, nthreads)
        if rc:
            raise OracleError(rc, "insert_seq_batch")

    def insert_keys_batch(self, set_ids, keys, offsets, nthreads: int = 1) -> None:
        ids = np.ascontiguousarray(set_ids, np.uint64)
        kk = np.ascontiguousarray(keys, np.uint64)
        off = np.ascontiguousarray(offsets, np.uint64)
        rc = lib().orc_insert_keys_batch(self._h, _ptr(ids), _ptr(kk), _ptr(off), ids.size, nthreads)
        if rc:
            raise OracleError(rc, "insert_keys_batch")

    # -- Algorithm 2 -----------------------------------------------------------
    def query_keys(self, keys) -> np.ndarray:
        k = np.ascontiguousarray(keys, np.uint64)
        out = np.zeros(self.K, np.uint32)
        n = lib().orc_query_keys(self._h, _ptr(k), k.size, _ptr(out), self.K)
        if n < 0:
            raise OracleError(n, "query_keys")
        return out[:n].copy()

    def query_seq(self, seq, k: int = 31) -> np.ndarray:
        s = np.frombuffer(bytes(seq), np.uint8) if not isinstance(seq, np.ndarray) else np.ascontiguousarray(seq, np.uint8)
        out = np.zeros(self.K, np.uint32)
        n = lib().orc_query_seq(self._h, _ptr(s), s.size, k, _ptr(out), self.K)
        if n < 0:
            raise OracleError(n, "query_seq")
        return out[:n].copy()

    def query_batch(self, kind: str, data, offsets, k: int = 31, nthreads: int = 1):
        """kind 'keys' (uint64 terms) or 'seq' (ASCII bases).  Returns
        (ids uint32, offsets uint64[n+1]) in CSR form, ascending per query."""
        kd = 0 if kind == "keys" else 1
        d = np.ascontiguousarray(data, np.uint64 if kd == 0 else np.uint8)
        off = np.ascontiguousarray(offsets, np.uint64)
        nq = off.size - 1
        counts = np.zeros(max(nq, 1), np.uint64)
        total = C.c_uint64(0)
        bad = C.c_uint64(0)
        L = lib()
        # first pass sizes the output; the oracle recomputes on the second (it is plain, not fast)
        rc = L.orc_query_batch(self._h, kd, _ptr(d), _ptr(off), nq, k, nthreads, _ptr(counts), None, 0,
                               C.byref(total), C.byref(bad))
        if rc:
            raise OracleError(rc, f"query_batch (query {bad.value})")
        ids = np.zeros(max(total.value, 1), np.uint32)
        rc = L.orc_query_batch(self._h, kd, _ptr(d), _ptr(off), nq, k, nthreads, _ptr(counts), _ptr(ids),
                               ids.size, C.byref(total), C.byref(bad))
        if rc:
            raise OracleError(rc, "query_batch")
        out_off = np.zeros(nq + 1, np.uint64)
        np.cumsum(counts[:nq], out=out_off[1:])
        return ids[: total.value].copy(), out_off

    def query_batch_counts(self, kind: str, data, offsets, k: int = 31, nthreads: int = 1):
        """One pass that returns only the per-query result sizes (for timing)."""
        kd = 0 if kind == "keys" else 1
        d = np.ascontiguousarray(data, np.uint64 if kd == 0 else np.uint8)
        off = np.ascontiguousarray(offsets, np.uint64)
        nq = off.size - 1
        counts = np.zeros(max(nq, 1), np.uint64)
        total = C.c_uint64(0)
        bad = C.c_uint64(0)
        rc = lib().orc_query_batch(self._h, kd, _ptr(d), _ptr(off), nq, k, nthreads, _ptr(counts), None, 0,
                                   C.byref(total), C.byref(bad))
        if rc:
            raise OracleError(rc, f"query_batch (query {bad.value})")
        return counts[:nq].copy()

    # -- inspection ------------------------------------------------------------
    def bf_contains(self, r: int, b: int, key: int) -> bool:
        return bool(lib().orc_bf_contains(self._h, r, b, key))

    def is_registered(self, i: int) -> bool:
        return bool(lib().orc_is_registered(self._h, i))

    def export_bf(self, r: int, b: int) -> np.ndarray:
        out = np.zeros((self.m + 63) // 64, np.uint64)
        lib().orc_export_bf(self._h, r, b, _ptr(out))
        return out

    def bf_bits(self, r: int, b: int) -> np.ndarray:
        """The BF of (table r, cell b) as a 0/1 uint8 array of length m."""
        w = self.export_bf(r, b)
        return np.unpackbits(w.view(np.uint8), bitorder="little")[: self.m]

    def get_row(self, r: int, pos: int) -> np.ndarray:
        out = np.zeros((self.B + 63) // 64, np.uint64)
        lib().orc_get_row(self._h, r, pos, _ptr(out))
        return out

    def cell_popcount(self) -> np.ndarray:
        out = np.zeros(self.R * self.B, np.uint64)
        lib().orc_cell_popcount(self._h, _ptr(out))
        return out.reshape(self.R, self.B)

    def registered(self) -> np.ndarray:
        out = np.zeros((self.K + 63) // 64, np.uint64)
        lib().orc_export_reg(self._h, _ptr(out))
        return np.unpackbits(out.view(np.uint8), bitorder="little")[: self.K].astype(bool)
