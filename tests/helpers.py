"""Test helpers: oracle evaluation of workload items and error metrics."""
import os

import numpy as np


def rel_fro(a, b):
    """||a - b||_F / ||b||_F over the trailing two axes."""
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b, axis=(-2, -1)) / np.linalg.norm(b, axis=(-2, -1))


def oracle_tinv_sites(orc, w, liz, spin, E):
    return orc.site_tinv(w.lmax, E, w.site_depths(liz, spin), w.r_mt)


def oracle_tau(orc, w, liz_index=0, items=None, nthreads=0):
    """Oracle tau_00 for (spin, energy) items of one LIZ of workload w.

    items: list of (spin, e_index) (collinear) or e_index (canted); default all.
    Returns array [len(items)][kap][kap] (row, col) and the oracle's own
    refinement estimate per item."""
    liz = w.lizs[liz_index]
    nE = len(w.energies)
    if w.canted:
        items = list(range(nE)) if items is None else list(items)
        E = np.array([w.energies[e] for e in items])
        tu = np.array([oracle_tinv_sites(orc, w, liz, 0, w.energies[e]) for e in items])
        td = np.array([oracle_tinv_sites(orc, w, liz, 1, w.energies[e]) for e in items])
        tau, err, _ = orc.tau00_batch(liz.pos, w.lmax, E, tu, td, liz.dirs, nthreads=nthreads)
        return tau, err
    if items is None:
        items = [(s, e) for s in range(w.nspin) for e in range(nE)]
    E = np.array([w.energies[e] for _, e in items])
    ti = np.array([oracle_tinv_sites(orc, w, liz, s, w.energies[e]) for s, e in items])
    tau, err, _ = orc.tau00_batch(liz.pos, w.lmax, E, ti, nthreads=nthreads)
    return tau, err


def ncpu():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1
