"""Shared helpers of the GPU parity tests: build the same workload in the GPU
library (through the C ABI) and in the CPU oracle, and compare bit for bit.

Expected values come only from the oracle; the comparison code converts the
oracle's per-cell Bloom filters and the GPU's bit-sliced rows into each other
with plain numpy bit operations."""
from __future__ import annotations

import os

import numpy as np

NTHREADS = max(1, min(16, os.cpu_count() or 1))


def build_pair(w, gpu_cls, oracle_cls, nthreads: int = NTHREADS, insert_chunks: int = 1):
    g = gpu_cls(w.K, w.B, w.R, w.m, w.eta, w.seed)
    o = oracle_cls(w.K, w.B, w.R, w.m, w.eta, w.seed)
    n = len(w.sets)
    bounds = np.linspace(0, n, insert_chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        part = w.sets.subset(np.arange(a, b))
        g.insert(part.ids, part.data, part.offsets, kind=w.sets.kind, k=w.k)
    if w.sets.kind == "keys":
        o.insert_keys_batch(w.sets.ids, w.sets.data, w.sets.offsets, nthreads=nthreads)
    else:
        o.insert_seq_batch(w.sets.ids, w.sets.data, w.sets.offsets, w.k, nthreads=nthreads)
    return g, o


def assert_index_equal(g, o):
    rows = g.export_index()  # [R, m, S]
    R, m, S = rows.shape
    assert (R, m) == (o.R, o.m)
    W = (o.B + 31) // 32
    assert np.all(rows[:, :, W:] == 0), "padding words must stay zero"
    for r in range(R):
        for b in range(o.B):
            plane = ((rows[r, :, b >> 5] >> np.uint32(b & 31)) & 1).astype(np.uint8)
            ref = o.bf_bits(r, b)
            if not np.array_equal(plane, ref):
                bad = np.nonzero(plane != ref)[0]
                raise AssertionError(f"table {r} cell {b}: {bad.size} bits differ, first at {bad[:5]}")
        # unused high bits of the last word are zero
        if o.B % 32:
            assert np.all(rows[r, :, W - 1] >> np.uint32(o.B % 32) == 0)
    assert np.array_equal(g.export_registered(), o.registered())


def assert_partition_equal(g, o):
    assert np.array_equal(g.export_partition().astype(np.int64), o.phi_table())


def assert_query_equal(g, o, queries, k: int = 31, nthreads: int = NTHREADS, **gpu_kw):
    ids, off = g.query(queries.data, queries.offsets, kind=queries.kind, k=k, **gpu_kw)
    rids, roff = o.query_batch(queries.kind, queries.data, queries.offsets, k=k, nthreads=nthreads)
    ids = np.asarray(ids.cpu() if hasattr(ids, "cpu") else ids).astype(np.uint32)
    off = np.asarray(off.cpu() if hasattr(off, "cpu") else off).astype(np.uint64)
    assert off.shape == roff.shape
    if not np.array_equal(off, roff):
        q = int(np.nonzero(off != roff)[0][0]) - 1
        raise AssertionError(f"result sizes differ first at query {q}: gpu {off[q+1]-off[q]} oracle {roff[q+1]-roff[q]}")
    assert np.array_equal(ids, rids)
    return ids, off


def assert_index_equal_by_rows(g, o):
    """Index bits through the oracle's row view (bit p of every cell of a
    table): cheaper than per-cell filters when B is large."""
    rows = g.export_index()  # [R, m, S]
    R, m, S = rows.shape
    assert (R, m) == (o.R, o.m)
    W = (o.B + 31) // 32
    assert np.all(rows[:, :, W:] == 0), "padding words must stay zero"
    for r in range(R):
        ref = np.stack([o.get_row(r, p) for p in range(m)]).view(np.uint32)[:, :W]  # [m, W]
        if not np.array_equal(rows[r, :, :W], ref):
            bad = np.argwhere(rows[r, :, :W] != ref)
            raise AssertionError(f"table {r}: {len(bad)} words differ, first (pos, word) {bad[:3].tolist()}")
    assert np.array_equal(g.export_registered(), o.registered())
