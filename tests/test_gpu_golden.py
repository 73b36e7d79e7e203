"""The large workloads against stored oracle tau_00 (tests/golden/tau00_*.npz,
written by tests/golden/make_golden.py, which calls only the CPU oracle).

Orders 4320 (spin-canted 135-site LIZ, Im E down to 0.00215), 6225 (NiAu-
shaped, Sec. 4.1), 6750 and 12450 (CoCrFeMnNi- and NiAu-shaped canted,
Sec. 4.1): the plain FP64 path and the mixed path (BF16x3 factors) with the
split-integer and with the tensor-core residual (the benchmark's
configuration) against the oracle,
per item, by relative Frobenius error: <= 1e-11 (FP64), <= 1e-9 (mixed).
The CPU test checks that the generator still produces the stored inputs.
"""
import os

import numpy as np
import pytest

from helpers import rel_fro
from paper_2308_16317_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = ["canted135", "niau249", "cocrfemnni135_canted", "niau249_canted"]
TOL64, TOLMIX = 1e-11, 1e-9


def _load(case):
    path = os.path.join(GOLDEN, "tau00_%s.npz" % case)
    if not os.path.exists(path):
        pytest.fail("missing golden file %s (run tests/golden/make_golden.py %s)" % (path, case))
    return dict(np.load(path))


def _workload(g):
    """The stored case's workload, restricted to the energies of its items."""
    w = getattr(wl, str(g["factory"]))(n_e=int(g["n_e"]))
    items = g["items"]
    e_idx = sorted(set(int(i[-1]) for i in items))
    sub = wl.Workload(w.name, w.lmax, w.lizs, np.asarray(w.energies)[e_idx].copy(), w.v_species, w.r_mt, w.canted)
    return w, sub, e_idx


@pytest.mark.parametrize("case", CASES)
def test_golden_inputs_reproduce(case):
    g = _load(case)
    w, _, _ = _workload(g)
    liz = w.lizs[0]
    # the contour nodes and moment directions come out of numpy's floating
    # point, which may differ in the last bit between host architectures
    assert np.allclose(np.asarray(w.energies), g["energies"], rtol=1e-14, atol=0.0)
    assert np.array_equal(liz.species, g["species"])
    if w.canted:
        assert np.allclose(liz.dirs, g["dirs"], rtol=0.0, atol=1e-15)
    assert w.n_of(liz) == int(g["order"]) and w.kappa() == int(g["kappa"])
    assert g["tau"].shape == (len(g["items"]), w.kappa(), w.kappa())
    assert np.isfinite(g["tau"]).all() and (g["oracle_err"] < 1e-13).all()


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("path", ["fp64", "mixed_int", "mixed_tc"])
def test_large_orders_vs_oracle_golden(B, case, path):
    import torch
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    g = _load(case)
    w, sub, e_idx = _workload(g)
    opts = {"fp64": B.must_default_opts(0), "mixed_int": B.must_default_opts(1, residual=2),
            "mixed_tc": B.must_default_opts(1, residual=3)}[path]
    s = Session(sub)
    tau, st = s.solve(opts)
    torch.cuda.synchronize()
    tau = blocks_to_numpy(tau)            # [n_out][len(e_idx)][kap][kap] (row, col)
    st = st.cpu().numpy()
    del s
    torch.cuda.empty_cache()
    pos = {e: q for q, e in enumerate(e_idx)}
    got = []
    for it in g["items"]:
        if w.canted:
            got.append(tau[0, pos[int(it[0])]])
            assert st[0, pos[int(it[0])]] == 0
        else:
            got.append(tau[int(it[0]), pos[int(it[1])]])
            assert st[int(it[0]), pos[int(it[1])]] == 0
    err = rel_fro(np.array(got), g["tau"])
    print(case, path, "order", int(g["order"]), "per-item rel err vs oracle:",
          ["%s Im E=%.5f: %.2e" % (tuple(int(v) for v in it), float(np.asarray(w.energies)[int(it[-1])].imag), e)
           for it, e in zip(g["items"], err)])
    assert err.max() <= (TOL64 if path == "fp64" else TOLMIX), err
