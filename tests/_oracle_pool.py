"""Whole motion fields from the CPU oracle, fanned out over the host cores.

Test infrastructure: each oracle call stays the plain single-threaded search
(one frame pair per call); only independent pairs run side by side, one
process per core.  Processes are spawned, never forked, because a child
forked after CUDA was initialised in the parent can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _search(task):
    import oracle
    cur, ref, B, R, algo = task
    if algo == "fs":
        return oracle.fs(cur, ref, B, R)
    return oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))


class OraclePool:
    """with OraclePool() as p: fields = p.fields(pairs, B, algo), pairs = [(cur, ref, R), ...]."""

    def __init__(self, procs: int | None = None):
        self.procs = procs or os.cpu_count() or 1
        self.pool = None

    def __enter__(self):
        self.pool = mp.get_context("spawn").Pool(self.procs)
        return self

    def __exit__(self, *exc):
        self.pool.close()
        self.pool.join()
        return False

    def fields(self, pairs, B, algo):
        tasks = [(np.ascontiguousarray(c), np.ascontiguousarray(r), B, R, algo) for c, r, R in pairs]
        return self.pool.map(_search, tasks, chunksize=1)


def first_difference(got, want):
    """None if the (mv, sad, nsp) fields are equal, else a short description."""
    for name, g, w in zip(("mv", "sad", "nsp"), got, want):
        g = np.asarray(g)
        w = np.asarray(w)
        if g.shape != w.shape:
            return f"{name}: shape {g.shape} != {w.shape}"
        if not np.array_equal(g, w):
            bad = np.argwhere(g.reshape(len(g), -1) != w.reshape(len(w), -1))[:3, 0]
            return f"{name} differs at blocks {bad.tolist()}: gpu {g[bad].tolist()} oracle {w[bad].tolist()}"
    return None
