"""Oracle reference solves for the full-size parity tests, run side by side.

A converged oracle solve of a full-size column takes from tens of seconds to
a couple of minutes of single-threaded numpy. The full-size GPU tests submit
all of theirs to one process pool at the start of the module, so that the
solves run on the host cores while the GPU tests work through their own
columns; each test then waits for its reference.

The pool is started with ``spawn`` (never ``fork``: a process forked after
the CUDA context exists can hang), each worker limited to one BLAS thread.
Nothing here computes any part of the method: it only calls ``oracle``.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

_POOL = None
_JOBS = {}


def _solve(atom, col, n_mu, method, kw):
    """One converged oracle solve of (atom, column): Algorithm 2 from LTE, or
    the hybrid start (RH92 iterations, then Algorithm 2)."""
    from oracle import model as OM
    from oracle.hybrid import hybrid
    from oracle.jfnk import jfnk
    m = OM.build_model(atom, col, n_mu)
    r = hybrid(m, m.nstar, **kw) if method == "hybrid" else jfnk(m, m.nstar, **kw)
    return dict(n=r.n, J=r.J, converged=bool(r.converged), F_norm=float(r.F_norm),
                F_norm0=float(r.F_norm0), F_calls=int(r.F_calls), newton_iters=int(r.newton_iters),
                rh92_iters=int(getattr(r, "rh92_iters", 0)))


def pool():
    global _POOL
    if _POOL is None:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(v, "1")
        workers = max(1, min(16, (os.cpu_count() or 2) - 1))
        _POOL = ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    return _POOL


def submit(key, atom, col, n_mu, method, **kw):
    """Starts (once per key) the oracle solve of one column."""
    if key not in _JOBS:
        _JOBS[key] = pool().submit(_solve, atom, col, n_mu, method, kw)
    return _JOBS[key]


def result(key, timeout=1800):
    return _JOBS[key].result(timeout=timeout)


def shutdown():
    global _POOL
    if _POOL is not None:
        _POOL.shutdown(wait=False, cancel_futures=True)
        _POOL = None
    _JOBS.clear()
