"""Oracle sampling over many processes -- TEST INFRASTRUCTURE ONLY.

Sample(G, count) of the oracle is keyed by sample id (every random draw of
sample s depends only on the seed and s), so the sets of ids [first,
first + count) are the concatenation of the sets of any split of that range.
This module splits the range over `spawn`-started worker processes, each
running the single-threaded oracle (oracle.c) on its share, and stitches the
pieces together.  It adds no arithmetic of its own; the split is pinned by
tests/test_oracle_sampling.py::test_ic_set_ids_continue_across_calls and by
test_parallel_split_equals_one_call below it.

Workers are started with the `spawn` method, so a process that has already
initialised CUDA can use it safely.  A `Sampler` keeps its workers (and the
graph they loaded once) for many calls; `sample()` makes one for a single call.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile
from types import SimpleNamespace

import numpy as np

from . import oracle as _O

_G = None   # the graph, in each worker process


def _init(path):
    global _G
    z = np.load(path)
    _G = SimpleNamespace(n=int(z["n"]), in_off=z["in_off"], in_src=z["in_src"], w=z["w"])


def _work(args):
    model, seed, first, count = args
    p = _O.sample(model, _G, seed, first, count)
    return p.set_off, p.members, p.examined


class Sampler:
    """`workers` oracle processes holding graph g; sample() splits an id range
    over them.  Use as a context manager (or call close())."""

    def __init__(self, g, workers: int | None = None):
        if workers is None:
            workers = max(1, min(32, os.cpu_count() or 1))
        self.workers = workers
        _O.build()
        self.pool = None
        self.tmp = tempfile.mkdtemp()
        try:
            path = os.path.join(self.tmp, "graph.npz")
            np.savez(path, n=np.int64(g.n), in_off=g.in_off, in_src=g.in_src, w=g.w)
            self.pool = mp.get_context("spawn").Pool(workers, initializer=_init,
                                                     initargs=(path,))
        except BaseException:
            shutil.rmtree(self.tmp, ignore_errors=True)   # no graph file left behind
            raise

    def sample(self, model: int, seed: int, first: int, count: int,
               chunk: int | None = None) -> _O.Pool:
        if chunk is None:
            chunk = max(1, -(-count // self.workers))
        jobs = [(model, seed, first + s, min(chunk, count - s)) for s in range(0, count, chunk)]
        parts = self.pool.map(_work, jobs)
        sizes = np.concatenate([np.diff(so) for so, _, _ in parts]) if parts \
            else np.zeros(0, np.int64)
        set_off = np.zeros(count + 1, np.int64)
        np.cumsum(sizes, out=set_off[1:])
        members = np.concatenate([m for _, m, _ in parts]) if parts else np.zeros(0, np.int32)
        return _O.Pool(set_off, members, sum(int(e) for _, _, e in parts))

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        shutil.rmtree(self.tmp, ignore_errors=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sample(model: int, g, seed: int, first: int, count: int, workers: int | None = None,
           chunk: int = 1 << 16) -> _O.Pool:
    """The oracle pool of ids [first, first + count), computed in parallel."""
    if workers is None:
        workers = max(1, min(32, os.cpu_count() or 1))
    if workers == 1 or count <= chunk:
        return _O.sample(model, g, seed, first, count)
    with Sampler(g, workers) as sm:
        return sm.sample(model, seed, first, count, chunk)
