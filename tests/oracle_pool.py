"""Runs independent 1D oracle problems in parallel worker processes (test infrastructure).

The pool uses the spawn start method, so it is safe to create after the test process has
initialised CUDA (a forked child of a CUDA process can hang).
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os


def _run(args):
    slab, series = args
    import oracle

    st, ser = oracle.run1d(slab, series=series)
    return st, ser


def run_many(slabs, series=False, workers=None):
    """oracle.run1d for every slab (serial build, one slab per task); results in order."""
    workers = workers or max(1, min(len(slabs), os.cpu_count() or 1))
    import oracle

    oracle.build()  # once in the parent, so the workers only load it
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run, [(s, series) for s in slabs]))
