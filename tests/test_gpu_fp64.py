"""GPU parity of the plain FP64 path against the CPU oracle (relative
Frobenius error per (energy, spin) <= 1e-11), through the C ABI."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau, rel_fro
from paper_2308_16317_gb300 import workload as wl

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _session(w, **kw):
    from paper_2308_16317_gb300.runner import Session
    return Session(w, **kw)


def _gpu_tau(w, opts=None, **kw):
    from paper_2308_16317_gb300.runner import blocks_to_numpy
    s = _session(w)
    tau, st = s.solve(opts, **kw)
    return blocks_to_numpy(tau), st.cpu().numpy(), s


def test_tinv_matches_oracle(B, orc):
    import torch
    for w in (wl.first_shell_small(), wl.liz135(), wl.canted135()):
        s = _session(w)
        got = s.tinv.cpu().numpy().reshape(w.nspin, 2, len(w.energies), w.lmax + 1)
        for sp in range(w.nspin):
            for k in range(2):
                for e, E in enumerate(w.energies):
                    _, ref = orc.square_well(w.lmax, E, w.v_species[sp][k], w.r_mt)
                    assert (np.abs(got[sp, k, e] - ref) <= 1e-13 * np.abs(ref)).all(), (sp, k, e)


def test_fp64_first_shell_all_energies(B, orc):
    w = wl.first_shell_small()
    tau, st, _ = _gpu_tau(w)
    ref, _ = oracle_tau(orc, w)
    assert (st == 0).all()
    err = rel_fro(tau.reshape(-1, 9, 9), ref)
    assert err.max() <= TOL64, err


@pytest.mark.parametrize("shells,lmax,seed", [(2, 3, 1), (3, 2, 2), (4, 1, 3), (2, 4, 4)])
def test_fp64_ragged_sizes(B, orc, shells, lmax, seed):
    """n = 19*16 = 304, 43*9 = 387, 55*4 = 220, 19*25 = 475: several 64-wide
    tiles plus ragged tails, panels that straddle the Schur boundary."""
    rng = np.random.default_rng(seed)
    pos, _ = wl.fcc_cluster(shells)
    liz = wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))
    w = wl.Workload("ragged", lmax, [liz], wl.semicircle_contour(5), wl.spin_depths(2), wl.R_MT)
    tau, st, _ = _gpu_tau(w)
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    assert (st == 0).all()
    err = rel_fro(tau.reshape(-1, w.kappa(), w.kappa()), ref)
    assert err.max() <= TOL64, err


def test_fp64_single_and_two_sites(B, orc):
    for N in (1, 2):
        pos = wl.fcc_cluster(1)[0][:N]
        w = wl.Workload("tiny", 3, [wl.Liz(pos, np.array([1, 0][:N], np.int32))], wl.semicircle_contour(4),
                        wl.spin_depths(2), wl.R_MT)
        tau, st, _ = _gpu_tau(w)
        ref, _ = oracle_tau(orc, w)
        assert (st == 0).all()
        assert rel_fro(tau.reshape(-1, 16, 16), ref).max() <= TOL64
        if N == 1:   # tau_00 = t exactly
            for s in range(2):
                for e, E in enumerate(w.energies):
                    t, _ = orc.square_well(3, E, w.v_species[s][1], wl.R_MT)
                    d = np.diag(tau[s, e])
                    assert np.abs(d - t[orc.l_of_L(3)]).max() <= 1e-13 * np.abs(t).max()


def test_fp64_canted_small(B, orc):
    rng = np.random.default_rng(9)
    pos, _ = wl.fcc_cluster(1)
    liz = wl.Liz(pos, rng.integers(0, 2, 13).astype(np.int32), wl.random_unit_vectors(rng, 13))
    w = wl.Workload("canted13", 2, [liz], wl.semicircle_contour(6), wl.spin_depths(2), wl.R_MT, canted=True)
    tau, st, _ = _gpu_tau(w)
    ref, _ = oracle_tau(orc, w)
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, 18, 18), ref).max() <= TOL64


def test_fp64_host_pointers_and_chunking_match(B):
    """Host buffers (staged through the workspace) and a workspace that only
    fits one energy at a time give bit-identical results."""
    import torch
    from paper_2308_16317_gb300.runner import blocks_to_numpy
    w = wl.first_shell_small()
    s = _session(w)
    tau_d, st_d = s.solve()
    ref = tau_d.cpu().numpy()
    E_h = np.ascontiguousarray(w.energies)
    tinv_h = s.tinv.cpu().numpy()
    tau_h = np.zeros((1, 8, 9, 9), np.complex128)
    st_h = np.zeros((1, 8), np.int32)
    nb = B.must_workspace_bytes(s.lizs[0], 8)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.must_tau00_solve(s.lizs[0], E_h, tinv_h, 2, 1, None, ws, nb, tau_h, st_h)
    assert np.array_equal(tau_h, ref) and (st_h == 0).all()
    one = B.must_workspace_bytes(s.lizs[0], 1)
    tau_c, st_c = s.solve(ws_bytes=one)
    torch.cuda.synchronize()
    assert np.array_equal(tau_c.cpu().numpy(), ref)


def test_fp64_singular_and_nonfinite_status(B):
    """An isolated site with t^{-1} = 0 is exactly singular; NaN in t^{-1}
    gives a non-finite result.  Both are reported per solve, not raised."""
    import torch
    liz = B.must_liz_build(np.zeros((1, 3)), np.zeros(1, np.int32), 2)
    E = torch.tensor([0.3 + 0.1j, 0.2 + 0.2j], dtype=torch.complex128, device="cuda")
    tinv = torch.zeros((1, 1, 2, 3), dtype=torch.complex128, device="cuda")
    tinv[0, 0, 1] = 1.0
    tinv[0, 0, 1, 2] = float("nan")
    tau = torch.empty((1, 2, 9, 9), dtype=torch.complex128, device="cuda")
    st = torch.full((1, 2), -1, dtype=torch.int32, device="cuda")
    nb = B.must_workspace_bytes(liz, 2)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.must_tau00_solve(liz, E, tinv, 1, 1, None, ws, nb, tau, st)
    assert st.cpu().numpy().tolist() == [[4, 6]]


def test_fp64_argument_errors(B):
    import torch
    liz = B.must_liz_build(np.zeros((1, 3)), np.zeros(1, np.int32), 2)
    E = torch.zeros(2, dtype=torch.complex128, device="cuda")
    tinv = torch.ones((1, 1, 2, 3), dtype=torch.complex128, device="cuda")
    tau = torch.empty((1, 2, 9, 9), dtype=torch.complex128, device="cuda")
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.MustError) as ei:   # workspace too small
        B.must_tau00_solve(liz, E, tinv, 1, 1, None, ws, 1024, tau)
    assert ei.value.code == 2
    with pytest.raises(B.MustError) as ei:   # species index 0 needs n_species >= 1, nspin 3 invalid
        B.must_tau00_solve(liz, E, tinv, 1, 3, None, ws, 1024, tau)
    assert ei.value.code == 1
    with pytest.raises(B.MustError):
        B.must_liz_build(np.zeros((2, 3)), np.zeros(2, np.int32), 2)   # coincident sites


def test_fp64_full_size_sampled(B, orc):
    """n = 2160 (135-site LIZ, lmax 3), all 64 (energy, spin) solves in the
    launch configuration the benchmark times; the oracle checks the solves at
    the lowest Im E, mid-contour and the Fermi end for both spins, and every
    solve is checked for tau_00 = tau_00^T and finiteness."""
    w = wl.liz135()
    tau, st, _ = _gpu_tau(w)
    assert (st == 0).all()
    assert np.isfinite(tau).all()
    sym = np.abs(tau - tau.swapaxes(-1, -2)).max(axis=(-2, -1)) / np.abs(tau).max(axis=(-2, -1))
    assert sym.max() < 1e-10
    items = [(0, 0), (1, 0), (0, 15), (1, 16), (0, 31), (1, 31)]
    ref, _ = oracle_tau(orc, w, items=items, nthreads=min(len(items), ncpu()))
    got = np.array([tau[s, e] for s, e in items])
    err = rel_fro(got, ref)
    assert err.max() <= TOL64, err
