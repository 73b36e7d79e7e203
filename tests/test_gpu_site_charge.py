"""Site charge inside the sphere (the energy-contour integral of Eq. 2 over the
site Green's function of Eq. 3), computed on the device from tau_00, against
the oracle's restatement (oracle/site_charge.py)."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau
from oracle import site_charge as sc
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


def _device_charge(B, w, tau, E, wt):
    """tau: torch [n_out][nE][kap][kap] complex128 on the device."""
    import torch
    dev = tau.device
    V = torch.tensor([w.site_depths(w.lizs[0], s)[0] for s in range(tau.shape[0])], dtype=torch.float64, device=dev)
    Ed = torch.tensor(E, dtype=torch.complex128, device=dev)
    wd = torch.tensor(wt, dtype=torch.complex128, device=dev)
    nE = torch.zeros(tau.shape[:2], dtype=torch.float64, device=dev)
    N = torch.zeros(tau.shape[0], dtype=torch.float64, device=dev)
    B.must_site_charge(w.lmax, Ed, wd, V, w.r_mt, tau, nE, N)
    torch.cuda.synchronize()
    return nE.cpu().numpy(), N.cpu().numpy()


def test_contour_weights_match_the_oracle(B):
    for n in (1, 8, 32):
        E, wt = B.must_contour_weights(n)
        E2, w2 = sc.contour_weights(n)
        assert np.abs(E - E2).max() <= 1e-15 and np.abs(wt - w2).max() <= 1e-15


@pytest.mark.parametrize("case", ["lone_site", "first_shell", "fcc135"])
def test_site_charge_matches_oracle(B, orc, case):
    import torch
    from paper_2308_16317_gb300.runner import Session
    if case == "lone_site":
        w = wl.Workload("one", 3, [wl.Liz(np.zeros((1, 3)), np.array([1], np.int32))], wl.semicircle_contour(16),
                        wl.spin_depths(2), wl.R_MT)
    elif case == "first_shell":
        w = wl.first_shell_small()
    else:
        w = wl.liz135(n_e=32, im_min=None)       # unclamped nodes: exactly the semicircle
    nE = len(w.energies)
    E, wt = B.must_contour_weights(nE)
    assert np.abs(E - np.asarray(w.energies)).max() <= 1e-14
    s = Session(w)
    tau, st = s.solve(B.must_default_opts(0))     # FP64 path
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    n_dev, N_dev = _device_charge(B, w, tau, E, wt)
    taus = tau.cpu().numpy().swapaxes(-1, -2)     # (row, col)
    for spin in range(tau.shape[0]):
        V = w.site_depths(w.lizs[0], spin)[0]
        n_ref, N_ref = sc.site_charge(w.lmax, E, wt, V, w.r_mt, taus[spin])
        assert np.abs(n_dev[spin] - n_ref).max() <= 1e-10 * np.abs(n_ref).max(), case
        assert abs(N_dev[spin] - N_ref) <= 1e-10 * abs(N_ref), (case, N_dev[spin], N_ref)
    if case != "fcc135":
        # the whole chain against the oracle's own tau_00
        ref, _ = oracle_tau(orc, w, nthreads=ncpu())
        k = w.kappa()
        ref = ref.reshape(w.nspin, nE, k, k)
        for spin in range(w.nspin):
            V = w.site_depths(w.lizs[0], spin)[0]
            _, N_ref = sc.site_charge(w.lmax, E, wt, V, w.r_mt, ref[spin])
            assert abs(N_dev[spin] - N_ref) <= 1e-9 * abs(N_ref)
    if case == "lone_site":
        # tau = t: the charge is that of an isolated well
        assert abs(N_dev[0] - N_dev[1]) > 0     # the two spin depths differ


@pytest.mark.parametrize("case", ["lone_site", "fcc135"])
def test_site_density_matches_oracle(B, case):
    """The radial density inside the sphere on the device against the oracle's
    restatement at the same tau_00; its radial quadrature against the device's
    own site charge; radii outside (0, r_mt] come back as NaN."""
    import torch
    from paper_2308_16317_gb300.runner import Session
    if case == "lone_site":
        w = wl.Workload("one", 3, [wl.Liz(np.zeros((1, 3)), np.array([1], np.int32))], wl.semicircle_contour(16),
                        wl.spin_depths(2), wl.R_MT)
    else:
        w = wl.liz135(n_e=32, im_min=None)
    nE = len(w.energies)
    E, wt = B.must_contour_weights(nE)
    s = Session(w)
    tau, st = s.solve(B.must_default_opts(0))
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    dev = tau.device
    V = torch.tensor([w.site_depths(w.lizs[0], sp)[0] for sp in range(tau.shape[0])], dtype=torch.float64,
                     device=dev)
    Ed = torch.tensor(E, dtype=torch.complex128, device=dev)
    wd = torch.tensor(wt, dtype=torch.complex128, device=dev)
    x, W = np.polynomial.legendre.leggauss(48)
    r = 0.5 * w.r_mt * (x + 1.0)
    radii = np.concatenate([r, [0.0, -1.0, 1.01 * w.r_mt]])
    rd = torch.tensor(radii, dtype=torch.float64, device=dev)
    out = torch.zeros((tau.shape[0], radii.size), dtype=torch.float64, device=dev)
    B.must_site_density(w.lmax, Ed, wd, V, w.r_mt, tau, rd, out)
    torch.cuda.synchronize()
    n_dev = out.cpu().numpy()
    _, N_dev = _device_charge(B, w, tau, E, wt)
    taus = tau.cpu().numpy().swapaxes(-1, -2)
    for spin in range(tau.shape[0]):
        Vs = w.site_depths(w.lizs[0], spin)[0]
        n_ref = sc.radial_density(w.lmax, E, wt, Vs, w.r_mt, taus[spin], r)
        assert np.abs(n_dev[spin, :r.size] - n_ref).max() <= 1e-10 * np.abs(n_ref).max(), case
        quad_N = 4.0 * np.pi * np.sum(0.5 * w.r_mt * W * r * r * n_dev[spin, :r.size])
        assert abs(quad_N - N_dev[spin]) <= 1e-9 * abs(N_dev[spin]), (case, quad_N, N_dev[spin])
        assert np.isnan(n_dev[spin, r.size:]).all()
