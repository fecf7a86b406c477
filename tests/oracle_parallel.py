"""The oracle's Algorithm 1 with its M(z) evaluations spread over host processes (test infrastructure).

oracle.rk4_path asks for M at each node and step midpoint in order; here those positions are evaluated
ahead, a block at a time, by oracle.coupling_M in a pool of single-threaded worker processes, and handed
to oracle.rk4_path unchanged.  The arithmetic is the oracle's own; only the order in which independent
positions are computed differs.  The pool uses the 'spawn' start method, so it is safe to create after
CUDA has been initialised in the parent process.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_BASIS = None


def _init(basis):
    global _BASIS
    _BASIS = basis


def _coupling(args):
    from oracle import wpccc_oracle as O
    b, v, z = args
    return O.coupling_M(_BASIS, b, v, z)


def _call_order(zgrid: np.ndarray) -> list:
    """The positions oracle.rk4_path evaluates, in its order: the first node, then per step the
    midpoint and the next node."""
    zs = [zgrid[0]]
    for i in range(zgrid.size - 1):
        zs.append((zgrid[i] + zgrid[i + 1]) / 2.0)
        zs.append(zgrid[i + 1])
    return zs


def propagate(basis, b: float, v: float, zgrid: np.ndarray, workers: int | None = None, block: int = 96):
    """Amplitudes at the end of one path, as oracle.propagate, with M(z) evaluated in parallel."""
    from oracle import wpccc_oracle as O
    workers = workers or max(1, min(32, os.cpu_count() or 1))
    order = _call_order(np.asarray(zgrid, dtype=np.float64))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"       # one BLAS thread per worker (inherited by the spawned processes)
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_init, initargs=(basis,)) as pool:
            cache = {}
            nxt = 0

            def Mfun(z):
                nonlocal nxt
                while z not in cache:
                    blk = order[nxt:nxt + block]
                    res = pool.map(_coupling, [(b, v, zz) for zz in blk], chunksize=1)
                    cache.clear()
                    cache.update(zip(blk, res))
                    nxt += len(blk)
                return cache[z]

            return O.rk4_path(Mfun, np.asarray(zgrid, dtype=np.float64), O.initial_state(basis))
    finally:
        for k, val in saved.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val
