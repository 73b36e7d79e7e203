"""The paper's own matrix shapes (Sec. 4.1): lmax = 4, kappa = 25 per spin.
Small lmax = 4 LIZs against the oracle; the full NiAu-shaped rank 6225 and
CoCrFeMnNi-shaped canted rank 6750 on the mixed path against the plain FP64
path (itself checked against the oracle at every smaller size), since the
oracle needs minutes per item at these ranks."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau, rel_fro
from paper_2308_16317_gb300 import workload as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _tau(B, w, precision, **kw):
    import torch
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    s = Session(w)
    tau, st = s.solve(B.must_default_opts(precision, **kw))
    torch.cuda.synchronize()
    return blocks_to_numpy(tau), st.cpu().numpy()


@pytest.mark.parametrize("canted", [False, True])
def test_lmax4_small_vs_oracle(B, orc, canted):
    rng = np.random.default_rng(44)
    pos, _ = wl.fcc_cluster(1)
    species = rng.integers(0, 2, pos.shape[0]).astype(np.int32)
    dirs = wl.random_unit_vectors(rng, pos.shape[0]) if canted else None
    w = wl.Workload("lmax4_13", 4, [wl.Liz(pos, species, dirs)], wl.semicircle_contour(3), wl.spin_depths(2),
                    wl.R_MT, canted=canted)
    k = w.kappa()
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    # FP64, and the mixed path with the double-float and the split-integer
    # residual (kap = 50 canted: the widest residual CTA)
    for precision, tol, residual in ((0, 1e-11, 1), (1, 1e-9, 1), (1, 1e-9, 2), (1, 1e-9, 3)):
        tau, st = _tau(B, w, precision, residual=residual)
        assert (st == 0).all()
        err = rel_fro(tau.reshape(-1, k, k), ref)
        assert err.max() <= tol, (precision, residual, err)


@pytest.mark.parametrize("shape", ["niau249", "cocrfemnni135_canted"])
def test_paper_rank_mixed_vs_fp64(B, shape):
    w = getattr(wl, shape)(n_e=8)
    E = np.asarray(w.energies)
    pick = [0, 4]                       # the contour end closest to the real axis, and mid-contour
    w = wl.Workload(w.name, w.lmax, w.lizs, E[pick].copy(), w.v_species, w.r_mt, w.canted)
    n = w.lizs[0].pos.shape[0] * w.kappa()
    assert n in (6225, 6750)
    t64, s64 = _tau(B, w, 0)
    tmx, smx = _tau(B, w, 1, residual=1)
    assert (s64 == 0).all() and (smx == 0).all()
    k = w.kappa()
    err = rel_fro(tmx.reshape(-1, k, k), t64.reshape(-1, k, k))
    print(shape, "rank", n, "mixed vs FP64 per item:", err)
    assert err.max() <= 1e-9
