"""GPU parity of the mixed-precision path (FP32 factors with tensor-core
trailing updates, FP64 residual refinement) against the CPU oracle: relative
Frobenius error per (energy, spin) <= 1e-9, including the points closest to
the real axis; and the status reporting of the refinement loop."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau, rel_fro
from paper_2308_16317_gb300 import workload as wl

pytestmark = pytest.mark.gpu
TOLMIX = 1e-9
PRECISIONS = [1, 2]   # MUST_MIXED_BF16X3, MUST_MIXED_TF32X3


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _gpu_tau(B, w, precision, **kw):
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    s = Session(w)
    opts = B.must_default_opts(precision, **kw)
    tau, st = s.solve(opts)
    return blocks_to_numpy(tau), st.cpu().numpy()


@pytest.mark.parametrize("residual", [0, 1])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mixed_first_shell(B, orc, precision, residual):
    w = wl.first_shell_small()
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w)
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, 9, 9), ref).max() <= TOLMIX


@pytest.mark.parametrize("residual", [0, 1])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shells,lmax,seed", [(2, 3, 1), (3, 2, 2), (3, 3, 5)])
def test_mixed_ragged_sizes(B, orc, precision, shells, lmax, seed, residual):
    """n = 304, 387, 688: several 128-row tensor-core tiles plus ragged tails."""
    rng = np.random.default_rng(seed)
    pos, _ = wl.fcc_cluster(shells)
    liz = wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))
    w = wl.Workload("ragged", lmax, [liz], wl.semicircle_contour(6), wl.spin_depths(2), wl.R_MT)
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, w.kappa(), w.kappa()), ref).max() <= TOLMIX


@pytest.mark.parametrize("residual", [0, 1])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mixed_canted_small(B, orc, precision, residual):
    rng = np.random.default_rng(9)
    pos, _ = wl.fcc_cluster(2)
    liz = wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32), wl.random_unit_vectors(rng, pos.shape[0]))
    w = wl.Workload("canted19", 2, [liz], wl.semicircle_contour(6), wl.spin_depths(2), wl.R_MT, canted=True)
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, 18, 18), ref).max() <= TOLMIX


def test_mixed_iteration_cap_zero_reports_noconv(B):
    w = wl.first_shell_small()
    _, st = _gpu_tau(B, w, 1, max_iter=0)
    assert (st == 5).all()


@pytest.mark.parametrize("residual", [0, 1])
def test_mixed_full_size_sampled(B, orc, residual):
    """n = 2160, all 64 solves in the benchmark's launch configuration;
    per-energy error against the oracle at the lowest Im E (both spins),
    mid-contour and the Fermi end."""
    w = wl.liz135()
    tau, st = _gpu_tau(B, w, 1, residual=residual)
    assert (st == 0).all() and np.isfinite(tau).all()
    items = [(0, 0), (1, 0), (0, 16), (1, 31)]
    ref, _ = oracle_tau(orc, w, items=items, nthreads=min(len(items), ncpu()))
    got = np.array([tau[s, e] for s, e in items])
    err = rel_fro(got, ref)
    print("per-energy rel err (bf16x3, residual %d):" % residual, dict(zip(map(str, items), err)))
    assert err.max() <= TOLMIX, err
