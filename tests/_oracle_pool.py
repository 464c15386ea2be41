"""The float64 oracle over every order of a large field, on all host cores.

Test infrastructure: orders are dealt round-robin to single-threaded worker
processes started with the 'spawn' method (safe in a process that already
uses a GPU; a worker that dies fails the call instead of hanging it), and the rows of each worker's orders are put back together.
"""

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def _work(args):
    import oracle
    from paper_0910_5435_gb300 import inputs

    l, beta_seed, G_seed, r, n = args
    ms = list(range(r, 2 * l, n))
    beta = inputs.random_beta(l, seed=beta_seed, decay=True)
    Gin = inputs.random_G(l, seed=G_seed)
    off = oracle.triangle_offsets(l)
    Go = oracle.legendre_synthesis(beta, l, orders=ms)[ms]
    bo = oracle.legendre_analysis(Gin, l, orders=ms)
    ba = oracle.legendre_adjoint(Gin, l, orders=ms)
    sel = np.concatenate([np.arange(off[m], off[m + 1]) for m in ms])
    return ms, Go, sel, bo[sel], ba[sel]


def all_orders(l, beta_seed, G_seed, nproc=None):
    """(G, beta_analysis, beta_adjoint): the oracle's synthesis of
    random_beta(l, beta_seed, decay=True) and its analysis and adjoint of
    random_G(l, G_seed), every order m = 0..2l-1."""
    import oracle

    nproc = nproc or max(1, os.cpu_count() or 1)
    off = oracle.triangle_offsets(l)
    G = np.zeros((2 * l, 2 * l), np.complex128)
    bo = np.zeros(off[-1], np.complex128)
    ba = np.zeros(off[-1], np.complex128)
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        # a worker that dies raises BrokenProcessPool here instead of hanging
        with ProcessPoolExecutor(nproc, mp_context=mp.get_context("spawn")) as pool:
            for ms, Go, sel, b1, b2 in pool.map(_work, [(l, beta_seed, G_seed, r, nproc) for r in range(nproc)]):
                G[ms] = Go
                bo[sel] = b1
                ba[sel] = b2
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return G, bo, ba
