"""Write oracle tau_00 values of the large workloads to tests/golden/.

The oracle needs minutes to tens of minutes per item at these orders
(complex LU of order 4320 to 12450 on one core), too long to recompute in a
GPU test, so the values are computed once by this script and stored.  It
calls only the CPU oracle (``oracle/``) and the seeded input generator
(``paper_2308_16317_gb300.workload``, which holds none of the method's
arithmetic); no value here comes from the CUDA library.

Cases (each item is one (spin, energy) block, or one energy when canted):
  canted135              spin-canted 135-site lmax-3 LIZ, order 4320, unclamped
                         contour: both end points (Im E = 0.00215) and mid-contour
  niau249                NiAu-shaped 249-site lmax-4 LIZ, rank 6225 (Sec. 4.1):
                         lowest-Im energy, both spins
  cocrfemnni135_canted   CoCrFeMnNi-shaped canted rank 6750 (Sec. 4.1): lowest-Im energy
  niau249_canted         NiAu-shaped canted rank 12450 (Sec. 4.1): lowest-Im energy

Usage: python tests/golden/make_golden.py [case ...]   (default: all cases)
Each case is written to tests/golden/tau00_<case>.npz with the inputs that
identify it (energies, species, directions) so a test can check that the
generator still produces the same workload.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from helpers import oracle_tau  # noqa: E402
from paper_2308_16317_gb300 import workload as wl  # noqa: E402

# case -> (workload factory, n_e, items)
CASES = {
    "canted135": (wl.canted135, 32, [0, 15, 31]),
    "niau249": (wl.niau249, 8, [(0, 0), (1, 0)]),
    "cocrfemnni135_canted": (wl.cocrfemnni135_canted, 8, [0]),
    "niau249_canted": (wl.niau249_canted, 8, [0]),
}


def path_of(case: str) -> str:
    return os.path.join(HERE, "tau00_%s.npz" % case)


def make(case: str) -> None:
    factory, n_e, items = CASES[case]
    w = factory(n_e=n_e)
    liz = w.lizs[0]
    t0 = time.time()
    tau, err = oracle_tau(oracle, w, items=items, nthreads=len(items))
    dt = time.time() - t0
    items_arr = np.array(items, dtype=np.int64).reshape(len(items), -1)
    np.savez_compressed(
        path_of(case), tau=tau, oracle_err=err, items=items_arr, n_e=n_e, factory=factory.__name__,
        energies=np.asarray(w.energies), species=liz.species,
        dirs=liz.dirs if liz.dirs is not None else np.zeros((0, 3)), order=w.n_of(liz), kappa=w.kappa())
    print("%s: order %d, %d items, %.0f s, oracle refinement estimate max %.2e"
          % (case, w.n_of(liz), len(items), dt, float(np.max(err))), flush=True)


if __name__ == "__main__":
    oracle.build()
    for c in (sys.argv[1:] or list(CASES)):
        make(c)
