"""Pins of the oracle's full-KKR restatement (periodic crystal, Sec. 5 of the
paper) against things other than itself:

- the Ewald lattice sums equal the plain Bloch sums of the (already pinned)
  real-space Hankel functions and structure-constant blocks where those
  converge (large Im E);
- the Ewald splitting parameter eta drops out, down to Im E = 0.005;
- the LSMS tau_00 of a growing LIZ converges to the crystal's tau (the LIZ
  is the crystal truncated, Sec. 2.2);
- the 4-site cubic cell of a pure fcc element gives the primitive cell's tau
  on every site;
- tau = tau^T (reciprocity) and the cubic pattern of a pure fcc element
  (diagonal for l <= 2, equal p entries, e_g and t_2g pairs).
"""
import numpy as np
import pytest

from paper_2308_16317_gb300 import workload as wl

A = wl.A_LAT
PRIM = wl.FCC_PRIMITIVE
CUBIC = A * np.eye(3)
BASIS4 = wl.FCC_CUBIC_BASIS


def _lattice_points(lat, rmax):
    n = int(rmax / np.min(np.linalg.norm(lat, axis=1))) + 3
    g = np.arange(-n, n + 1)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    v = m @ lat
    r = np.linalg.norm(v, axis=1)
    return v[r <= rmax]


def test_ewald_lattice_sum_equals_direct_bloch_sum(orc):
    """D_L(k) = sum_{R != 0} e^{ik.R} h_l(kappa|R|) Y_L(-R^) for l <= 6, where
    the plain sum converges (Im kappa ~ 0.75: terms below 1e-14 beyond 45 bohr)."""
    E = -0.1 + 1.0j
    kap = np.sqrt(E)
    k = np.array([0.13, 0.07, 0.21])
    D = orc.kkr_lattice_sum(6, E, PRIM, [0, 0, 0], k, eta=0.6)
    pts = _lattice_points(PRIM, 45.0)
    ref = np.zeros(49, complex)
    for v in pts:
        r = np.linalg.norm(v)
        if r == 0.0:
            continue
        _, _, h = orc.sph_jyh(6, kap * r)
        Y = orc.real_ylm(6, -v)
        ph = np.exp(1j * (k @ v))
        for l in range(7):
            ref[l * l:(l + 1) ** 2] += ph * h[l] * Y[l * l:(l + 1) ** 2]
    assert np.abs(D - ref).max() <= 1e-12 * np.abs(ref).max()


def test_kkr_structure_constants_equal_bloch_sum_of_blocks(orc):
    """G^{st}(k) of two sites of the cubic cell (a displaced pair included)
    equals sum_R e^{ik.R} G(b_s - b_t - R) built from the pinned real-space
    blocks; Im kappa ~ 1.0, so 38 bohr reaches 1e-14."""
    E = -0.1 + 2.0j
    k = np.array([0.13, 0.07, 0.21])
    basis = BASIS4[:2]
    G = orc.kkr_struct_const(2, E, CUBIC, basis, k, eta=0.25)
    ref = np.zeros((2, 2, 9, 9), complex)
    for v in _lattice_points(CUBIC, 40.0):
        for s in range(2):
            for t in range(2):
                rho = basis[s] - basis[t] - v
                r = np.linalg.norm(rho)
                if r < 1e-9 or r > 38.0:
                    continue
                ref[s, t] += np.exp(1j * (k @ v)) * orc.struct_const(2, E, rho)
    ref = ref.transpose(0, 2, 1, 3).reshape(18, 18)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("E", [0.6 + 0.005j, -0.3 + 0.005j, 0.2 + 0.5j])
def test_ewald_independent_of_eta(orc, E):
    k = np.array([0.13, 0.07, 0.21])
    for x in (np.zeros(3), BASIS4[1] - BASIS4[2]):
        D1 = orc.kkr_lattice_sum(6, E, CUBIC, x, k, eta=0.15)
        D2 = orc.kkr_lattice_sum(6, E, CUBIC, x, k, eta=0.6)
        assert np.abs(D1 - D2).max() <= 1e-13 * np.abs(D1).max()


def test_lsms_tau_converges_to_crystal_tau(orc):
    """tau_00 of the LIZ through S shells approaches the crystal's tau as S
    grows (Im kappa ~ 0.75, lmax = 1)."""
    lmax, E = 1, -0.1 + 1.0j
    _, ti = orc.square_well(lmax, E, -1.0, wl.R_MT)
    tk, _ = orc.kkr_tau(lmax, PRIM, [[0.0, 0.0, 0.0]], [E], ti[None, None, :], nk=10, eta=0.6)
    tk = tk[0, 0]
    errs = []
    for S in (1, 3, 5, 7):
        pos, _ = wl.fcc_cluster(S)
        tl, _, _ = orc.tau00_batch(pos, lmax, [E], np.tile(ti, (len(pos), 1))[None])
        errs.append(np.linalg.norm(tl[0] - tk) / np.linalg.norm(tk))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs


def test_cubic_cell_equals_primitive_cell(orc):
    lmax, E = 2, -0.1 + 1.5j
    _, ti = orc.square_well(lmax, E, -1.0, wl.R_MT)
    tp, _ = orc.kkr_tau(lmax, PRIM, [[0.0, 0.0, 0.0]], [E], ti[None, None, :], nk=8, eta=0.6)
    tc, _ = orc.kkr_tau(lmax, CUBIC, BASIS4, [E], np.tile(ti, (1, 4, 1)), nk=5, eta=0.25)
    for s in range(4):
        assert np.linalg.norm(tc[0, s] - tp[0, 0]) <= 1e-9 * np.linalg.norm(tp[0, 0]), s


@pytest.mark.parametrize("E", [0.5 + 0.01j, -0.2 + 0.3j])
def test_crystal_tau_symmetry_and_cubic_pattern(orc, E):
    lmax = 2
    _, ti = orc.square_well(lmax, E, -1.4, wl.R_MT)
    tau, _ = orc.kkr_tau(lmax, PRIM, [[0.0, 0.0, 0.0]], [E], ti[None, None, :], nk=6, eta=0.6)
    T = tau[0, 0]
    scale = np.abs(T).max()
    assert np.abs(T - T.T).max() <= 1e-13 * scale
    off = T - np.diag(np.diag(T))
    assert np.abs(off).max() <= 1e-12 * scale
    d = np.diag(T)
    assert np.abs(d[1:4] - d[1]).max() <= 1e-12 * scale          # p
    assert np.abs(d[[4, 5, 7]] - d[4]).max() <= 1e-12 * scale     # t2g: xy, yz, xz
    assert abs(d[6] - d[8]) <= 1e-12 * scale                      # eg: z^2, x^2 - y^2
    assert abs(d[4] - d[6]) > 1e-6 * scale                        # the cubic field splits them


def test_crystal_generators():
    c = wl.fcc_crystal()
    assert c.n_basis == 1 and c.lmax == 3 and len(c.energies) == 32 and c.nspin == 2
    vol = abs(np.linalg.det(c.lattice))
    assert abs(vol - A ** 3 / 4) < 1e-9
    c4 = wl.l12_crystal()
    assert c4.n_basis == 4 and list(c4.species) == [1, 0, 0, 0]
    assert abs(abs(np.linalg.det(c4.lattice)) - A ** 3) < 1e-9
    # nearest-neighbour distance a / sqrt(2) between basis sites
    d = np.linalg.norm(c4.basis[1] - c4.basis[2])
    assert abs(d - A / np.sqrt(2)) < 1e-12
