"""Pins for the CPU oracle: closed forms, special cases, library cross-checks,
invariants and brute force -- chosen so that a dropped term, a wrong sign,
index or phase convention, or a transposed operand fails at least one test.

Paper: arXiv 2308.16317, Eq. 4 (tau = [t^{-1} - g0]^{-1}, g0 between
different sites), Sec. 2.1 (rank N(lmax+1)^2, 2N(lmax+1)^2 when canted),
Sec. 2.2 (LSMS: LIZ matrix, only the first block of M^{-1} is needed).
"""
import numpy as np
import pytest
import scipy.special as sp

from paper_2308_16317_gb300 import workload as wl

ZS = [0.3 + 0.01j, 1.3 + 0.2j, 3.14159 + 0.001j, 5.0 - 0.02j, 8.0 + 0.5j, 11.5 + 0.05j, 0.002 + 0.001j]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def l_of_L(lmax):
    return np.array([l for l in range(lmax + 1) for _ in range(2 * l + 1)])


# ---------------------------------------------------------------- Bessel ----

@pytest.mark.parametrize("z", ZS)
def test_bessel_matches_scipy(orc, z):
    """j_l, y_l against scipy's independent implementation (complex argument)."""
    j, y = orc.sph_jy(8, z)
    for l in range(9):
        # relative, with an absolute floor near zeros of j_l (cancellation in sin z)
        assert abs(j[l] - sp.spherical_jn(l, z)) <= 1e-13 * abs(j[l]) + 1e-15 * np.abs(j).max()
        assert abs(y[l] - sp.spherical_yn(l, z)) <= 1e-13 * abs(y[l])


@pytest.mark.parametrize("z", ZS[:-1])
def test_bessel_wronskian_and_hankel0(orc, z):
    """j_l y_l' - j_l' y_l = 1/z^2 (A&S 10.1.6) and h_0 = -i e^{iz}/z."""
    j, y = orc.sph_jy(9, z)
    for l in range(1, 8):
        dj = j[l - 1] - (l + 1) / z * j[l]
        dy = y[l - 1] - (l + 1) / z * y[l]
        w = j[l] * dy - dj * y[l]
        assert abs(w * z * z - 1.0) < 1e-11
    h0 = j[0] + 1j * y[0]
    assert abs(h0 - (-1j * np.exp(1j * z) / z)) < 1e-14 * abs(h0)


@pytest.mark.parametrize("z", [0.06 + 7.26j, 0.004 + 2.74j, 1.3 + 0.2j, 9.5 + 0.3j, 0.02 + 13.0j, 0.4 + 0.05j])
def test_hankel_closed_form_against_mpmath(orc, z):
    """h_l = j_l + i y_l against 40-digit mpmath, including arguments with a
    large imaginary part (kappa |R| near the bottom of the contour), where
    forming j_l + i y_l in double precision cancels catastrophically."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    zz = mp.mpc(z.real, z.imag)
    _, _, h = orc.sph_jyh(8, z)
    for l in range(9):
        f = mp.sqrt(mp.pi / (2 * zz))
        ref = complex(f * (mp.besselj(l + 0.5, zz) + 1j * mp.bessely(l + 0.5, zz)))
        assert abs(h[l] - ref) <= 1e-14 * abs(ref), (l, h[l], ref)


# ---------------------------------------------------- real harmonics -------

def test_real_ylm_closed_forms(orc):
    """Cartesian closed forms for l <= 2 (no Condon-Shortley phase):
    Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x, Y_2,-2 ~ xy, Y_2,-1 ~ yz, Y_2,0 ~ 3z^2-r^2,
    Y_2,1 ~ xz, Y_2,2 ~ x^2-y^2."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        v = rng.standard_normal(3)
        x, y, z = v / np.linalg.norm(v)
        c1 = np.sqrt(3 / (4 * np.pi))
        c2 = np.sqrt(15 / (4 * np.pi))
        ref = [1 / np.sqrt(4 * np.pi), c1 * y, c1 * z, c1 * x,
               c2 * x * y, c2 * y * z, np.sqrt(5 / (16 * np.pi)) * (3 * z * z - 1), c2 * x * z,
               np.sqrt(15 / (16 * np.pi)) * (x * x - y * y)]
        got = orc.real_ylm(2, v * 3.7)
        assert np.allclose(got, ref, atol=1e-15, rtol=1e-14)


def _scipy_real_ylm(lmax, v):
    """Real harmonics from scipy's complex (Condon-Shortley) ones:
    Y_l,m>0 = sqrt2 (-1)^m Re Y_lm, Y_l,m<0 = sqrt2 (-1)^m Im Y_l|m|."""
    r = np.linalg.norm(v)
    th, ph = np.arccos(v[2] / r), np.arctan2(v[1], v[0])
    out = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            Y = sp.sph_harm_y(l, abs(m), th, ph)
            if m > 0:
                out.append(np.sqrt(2) * (-1) ** m * Y.real)
            elif m < 0:
                out.append(np.sqrt(2) * (-1) ** m * Y.imag)
            else:
                out.append(Y.real)
    return np.array(out)


def test_real_ylm_matches_scipy_and_orthonormal(orc):
    rng = np.random.default_rng(2)
    for _ in range(5):
        v = rng.standard_normal(3)
        assert np.allclose(orc.real_ylm(7, v), _scipy_real_ylm(7, v), atol=1e-13)
    # orthonormality by numpy's Gauss-Legendre x uniform phi (exact for degree 14)
    xg, wg = np.polynomial.legendre.leggauss(12)
    nph = 20
    gram = np.zeros((49, 49))
    for x, w in zip(xg, wg):
        s = np.sqrt(1 - x * x)
        for k in range(nph):
            ph = 2 * np.pi * k / nph
            Y = orc.real_ylm(6, [s * np.cos(ph), s * np.sin(ph), x])
            gram += w * (2 * np.pi / nph) * np.outer(Y, Y)
    assert np.abs(gram - np.eye(49)).max() < 1e-13


# ------------------------------------------------------------- Gaunt -------

def test_gaunt_special_values_and_selection(orc):
    C = orc.gaunt(3, 3, 6)
    # C(L, L', 00) = delta_LL' / sqrt(4 pi)
    assert np.allclose(C[:, :, 0], np.eye(16) / np.sqrt(4 * np.pi), atol=1e-15)
    l1, l3 = l_of_L(3), l_of_L(6)
    for a in range(16):
        for b in range(16):
            for c in range(49):
                if (l1[a] + l1[b] + l3[c]) % 2 or l3[c] > l1[a] + l1[b] or l3[c] < abs(l1[a] - l1[b]):
                    assert C[a, b, c] == 0.0
    assert np.count_nonzero(C) == 708          # real-Gaunt nonzeros for l, l' <= 3
    assert np.allclose(C, C.transpose(1, 0, 2))


def test_gaunt_matches_wigner3j(orc):
    """Real Gaunt coefficients from sympy's exact complex Gaunt integrals
    (Wigner 3j) and the complex->real transform verified above."""
    sym = pytest.importorskip("sympy.physics.wigner")
    lmax = 2
    C = orc.gaunt(lmax, lmax, 2 * lmax)

    def U(l):
        # real Y_lm = sum_mu U[m, mu] Y_l,mu (complex, CS phase); rows m = -l..l
        M = np.zeros((2 * l + 1, 2 * l + 1), complex)
        for m in range(-l, l + 1):
            if m > 0:    # sqrt2 (-1)^m Re Y_lm = (-1)^m/sqrt2 (Y_lm + (-1)^m Y_l,-m)
                M[m + l, m + l] += (-1) ** m / np.sqrt(2)
                M[m + l, -m + l] += 1 / np.sqrt(2)
            elif m < 0:  # sqrt2 (-1)^m Im Y_l|m| = (-1)^m/(sqrt2 i) (Y_l|m| - (-1)^m Y_l,-|m|)
                am = -m
                M[m + l, am + l] += (-1) ** am / (np.sqrt(2) * 1j)
                M[m + l, -am + l] += -1 / (np.sqrt(2) * 1j)
            else:
                M[l, l] = 1.0
        return M

    Ls = [(l, m) for l in range(2 * lmax + 1) for m in range(-l, l + 1)]
    for a, (la, ma) in enumerate(Ls[:9]):
        for b, (lb, mb) in enumerate(Ls[:9]):
            for c, (lc, mc) in enumerate(Ls):
                Ua, Ub, Uc = U(la)[ma + la], U(lb)[mb + lb], U(lc)[mc + lc]
                s = 0j
                for mua in range(-la, la + 1):
                    for mub in range(-lb, lb + 1):
                        muc = -(mua + mub)
                        if abs(muc) > lc:
                            continue
                        g = float(sym.gaunt(la, lb, lc, mua, mub, muc))
                        s += Ua[mua + la] * Ub[mub + lb] * Uc[muc + lc] * g
                assert abs(s.imag) < 1e-14
                assert abs(s.real - C[a, b, c]) < 1e-14


# --------------------------------------------- structure constants ---------

def _jY(orc, lmax, kap, v):
    r = np.linalg.norm(v)
    j, _ = orc.sph_jy(lmax, kap * r)
    return j[l_of_L(lmax)] * orc.real_ylm(lmax, v)


@pytest.mark.parametrize("E", [0.3 + 0.2j, -0.25 + 0.01j, 0.6 + 0.4j, -0.3 + 0.005j])
def test_two_centre_expansion_reproduces_free_green_function(orc, E):
    """g0(x, x') = -exp(i k |x-x'|) / (4 pi |x-x'|) must equal
    sum_LL' j_l(k r) Y_L(r^) G^{ij}_LL' j_l'(k r') Y_L'(r'^) for x = r + R_i,
    x' = r' + R_j; the truncation error falls rapidly with lmax."""
    kap = np.sqrt(E)
    Ri, Rj = np.array([0.0, 0.0, 0.0]), np.array([3.5, -2.0, 1.5])
    rv, rp = np.array([0.3, 0.2, -0.25]), np.array([-0.1, 0.35, 0.2])
    d = np.linalg.norm(rv + Ri - rp - Rj)
    exact = -np.exp(1j * kap * d) / (4 * np.pi * d)
    errs = []
    for lmax in (3, 6, 10):
        G = orc.struct_const(lmax, E, Ri - Rj)
        approx = _jY(orc, lmax, kap, rv) @ G @ _jY(orc, lmax, kap, rp)
        errs.append(abs(approx - exact) / abs(exact))
    assert errs[0] < 1e-3 and errs[1] < 1e-6 and errs[2] < 1e-9
    assert errs[2] < errs[1] < errs[0]


def test_structure_constant_identities(orc):
    """G^{ij}_{LL'} = G^{ji}_{L'L} (reciprocity of g0) and
    G^{ji}_{LL'} = (-1)^{l+l'} G^{ij}_{LL'} (parity).  The combined form
    G^{ij}_{LL'} = (-1)^{l+l'} G^{ji}_{L'L} does not hold in general."""
    R = np.array([2.1, -4.0, 3.3])
    E = 0.41 + 0.07j
    G = orc.struct_const(3, E, R)
    Gt = orc.struct_const(3, E, -R)
    l = l_of_L(3)
    P = (-1.0) ** np.add.outer(l, l)
    scale = np.abs(G).max()
    assert np.abs(G - Gt.T).max() < 1e-13 * scale
    assert np.abs(Gt - P * G).max() < 1e-13 * scale
    assert np.abs(G - P * Gt.T).max() > 1e-2 * scale


def test_structure_constant_axial_block_is_m_diagonal(orc):
    """For R along z only Y_l''0 survives, so G couples only equal m."""
    G = orc.struct_const(3, 0.3 + 0.1j, [0.0, 0.0, 5.0])
    m = np.array([mm for l in range(4) for mm in range(-l, l + 1)])
    off = m[:, None] != m[None, :]
    assert np.abs(G[off]).max() < 1e-14 * np.abs(G).max()


# ------------------------------------------------------- t-matrices -------

def test_t_zero_depth_vanishes(orc):
    t, _ = orc.square_well(3, 0.3 + 0.05j, 0.0, wl.R_MT)
    assert np.abs(t).max() < 1e-15


@pytest.mark.parametrize("E", [0.5 + 0.1j, -0.2 + 0.3j])
def test_t_born_limit(orc, E):
    """t_l / V -> int_0^a j_l(k r)^2 r^2 dr = (a^3/2)[j_l^2 - j_{l-1} j_{l+1}](k a)
    (Lommel integral; j_{-1}(z) = cos z / z)."""
    a = wl.R_MT
    kap = np.sqrt(E)
    # Richardson extrapolation of t/V over two small depths removes the O(V)
    # second Born term while keeping cancellation error (~eps/V) small.
    V1, V2 = -1e-4, -2e-4
    t1, _ = orc.square_well(3, E, V1, a)
    t2, _ = orc.square_well(3, E, V2, a)
    lim = 2 * t1 / V1 - t2 / V2
    z = kap * a
    j = sp.spherical_jn(np.arange(5), z)
    jm1 = np.cos(z) / z
    for l in range(4):
        prev = jm1 if l == 0 else j[l - 1]
        born = 0.5 * a ** 3 * (j[l] ** 2 - prev * j[l + 1])
        assert abs(lim[l] - born) < 1e-6 * abs(born)
        assert abs(t1[l] / V1 - born) > 1e-7 * abs(born)   # the limit is non-trivial


@pytest.mark.parametrize("E", [0.05, 0.35, 0.69])
def test_t_unitarity_and_s_wave_closed_form(orc, E):
    """Real E > 0, real V: Im t_l^{-1} = kappa; the s-wave phase shift is
    delta_0 = -k a + arctan(k tan(q a) / q) and t_0 = -(1/k) sin d e^{i d}."""
    a, V = wl.R_MT, -1.4
    k, q = np.sqrt(E), np.sqrt(E - V)
    t, ti = orc.square_well(3, E, V, a)
    assert np.allclose(ti.imag, k, rtol=1e-13, atol=0)
    d0 = -k * a + np.arctan(k * np.tan(q * a) / q)
    t0 = -np.sin(d0) * np.exp(1j * d0) / k
    assert abs(t[0] - t0) < 1e-13 * abs(t0)


def test_t_pole_at_s_bound_state(orc):
    """The isolated well's l=0 bound state (q cot(q a) = -sqrt(-E)) is a zero of
    t_0^{-1} at real E < 0."""
    from scipy.optimize import brentq
    a, V = wl.R_MT, -1.0
    f = lambda E: np.sqrt(E - V) / np.tan(np.sqrt(E - V) * a) + np.sqrt(-E)
    Eb = brentq(f, -0.9, -0.05, xtol=1e-15)
    assert -0.29 < Eb < -0.27
    _, ti_b = orc.square_well(0, Eb, V, a)
    _, ti_off = orc.square_well(0, Eb + 0.05, V, a)
    assert abs(ti_b[0]) < 1e-12 * abs(ti_off[0])


# ----------------------------------------------------- linear algebra ------

def test_lu_solve_matches_lapack(orc):
    rng = np.random.default_rng(3)
    for n in (1, 5, 37):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        B = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
        assert rel(orc.lu_solve(A, B), np.linalg.solve(A, B)) < 1e-12


def test_gauss_jordan_matches_lapack(orc):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((23, 23)) + 1j * rng.standard_normal((23, 23))
    assert rel(orc.inverse(A), np.linalg.inv(A)) < 1e-12


def test_first_block_refinement_is_exact_on_integer_inverse(orc):
    """M = L U with integer unit-triangular factors has an exact integer inverse;
    the refined first block must reproduce it to rounding."""
    rng = np.random.default_rng(7)
    n, kap = 40, 4
    L = np.tril(rng.integers(-1, 2, (n, n)), -1) + np.eye(n, dtype=int)
    U = np.triu(rng.integers(-1, 2, (n, n)), 1) + np.eye(n, dtype=int)
    Mi = (L @ U).astype(object)
    Linv = np.eye(n, dtype=object)
    for i in range(n):
        for k in range(i):
            Linv[i] -= L[i, k] * Linv[k]
    Uinv = np.eye(n, dtype=object)
    for i in reversed(range(n)):
        for k in range(i + 1, n):
            Uinv[i] -= U[i, k] * Uinv[k]
    exact = (Uinv @ Linv)[:kap, :kap].astype(np.float64)
    M = (Mi.astype(np.float64) * (1 + 0.5j))
    assert np.linalg.cond(M) > 1e9
    tau, err = orc.first_block(M, kap)
    assert rel(tau, exact / (1 + 0.5j)) < 1e-15
    assert err < 1e-15


def test_first_block_refinement_beats_plain_solve_on_ill_conditioned(orc):
    """Against a 50-digit mpmath inverse of an ill-conditioned complex matrix
    (cond ~1e11), the double-double refined block is accurate to ~1e-15 while
    an unrefined LAPACK inverse loses about cond * eps."""
    mp = pytest.importorskip("mpmath")
    rng = np.random.default_rng(11)
    n, kap = 24, 3
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    M = Q1 @ np.diag(np.logspace(0, -11, n)) @ Q2
    mp.mp.dps = 50
    Mm = mp.matrix([[mp.mpc(complex(M[i, j])) for j in range(n)] for i in range(n)])
    Mi = Mm ** -1
    ref = np.array([[complex(Mi[i, j]) for j in range(kap)] for i in range(kap)])
    tau, _ = orc.first_block(M, kap)
    assert rel(tau, ref) < 1e-14
    assert rel(np.linalg.inv(M)[:kap, :kap], ref) > 1e2 * rel(tau, ref)


# ------------------------------------------------- KKR matrix and tau ------

def _tinv_sites(orc, w, liz, spin, E):
    return orc.site_tinv(w.lmax, E, w.site_depths(liz, spin), w.r_mt)


def test_matrix_structure_and_symmetry(orc):
    w = wl.first_shell_small()
    liz = w.lizs[0]
    E = w.energies[3]
    ti = _tinv_sites(orc, w, liz, 0, E)
    M = orc.assemble(liz.pos, w.lmax, E, ti)
    nl = 9
    assert M.shape == (13 * nl, 13 * nl)
    l = l_of_L(2)
    for i in range(13):
        blk = M[i * nl:(i + 1) * nl, i * nl:(i + 1) * nl]
        assert np.allclose(blk, np.diag(ti[i][l]), atol=0)
    G01 = orc.struct_const(2, E, liz.pos[0] - liz.pos[1])
    assert np.allclose(M[:nl, nl:2 * nl], -G01, atol=0)
    assert np.abs(M - M.T).max() < 1e-13 * np.abs(M).max()


def test_tau_single_site_is_t(orc):
    """N_LIZ = 1: M = t^{-1}, so tau_00 = diag(t_l)."""
    E = 0.2 + 0.3j
    t, ti = orc.square_well(3, E, -1.4, wl.R_MT)
    M = orc.assemble(np.zeros((1, 3)), 3, E, ti[None, :])
    tau, _ = orc.first_block(M, 16)
    assert rel(tau, np.diag(t[l_of_L(3)])) < 1e-15


def test_tau_first_block_equals_brute_force_inverse(orc):
    w = wl.first_shell_small()
    liz = w.lizs[0]
    for E in w.energies[[0, 7]]:
        M = orc.assemble(liz.pos, w.lmax, E, _tinv_sites(orc, w, liz, 0, E))
        tau, _ = orc.first_block(M, 9)
        full = orc.inverse(M)
        assert rel(tau, full[:9, :9]) < 1e-13
        assert rel(tau, np.linalg.inv(M)[:9, :9]) < 1e-12
        assert np.abs(tau - tau.T).max() < 1e-12 * np.abs(tau).max()


def test_tau_weak_scattering_series(orc):
    """Zero-depth limit: for wells of depth V -> 0, tau_00 -> t_0 + t_0 sum_j
    G^{0j} t_j G^{j0} t_0 with a remainder of fourth order in t (and tau -> 0)."""
    liz = wl.fcc_cluster(1)[0]
    E, lmax = 0.3 + 0.2j, 2
    l = l_of_L(lmax)
    for V in (-1e-3, -1e-4):
        t, ti = orc.square_well(lmax, E, V, wl.R_MT)
        M = orc.assemble(liz, lmax, E, np.tile(ti, (13, 1)))
        tau, _ = orc.first_block(M, 9)
        T = np.diag(t[l])
        second = sum(orc.struct_const(lmax, E, liz[0] - liz[j]) @ T @ orc.struct_const(lmax, E, liz[j] - liz[0])
                     for j in range(1, 13))
        approx = T + T @ second @ T
        rem = np.linalg.norm(tau - approx)
        assert rem < 1e-2 * np.linalg.norm(T @ second @ T)
        assert np.linalg.norm(tau) < 1e3 * abs(V)


@pytest.mark.parametrize("shells", [1, 2])
def test_tau_cubic_symmetry_pure_element(orc, shells):
    """All sites one species on an O_h-symmetric cluster: tau_00 vanishes for
    l + l' odd, p is a multiple of 1_3, d splits into t2g (xy, yz, xz) and
    e_g (z^2, x^2-y^2) with no d-d off-diagonal coupling."""
    pos = wl.fcc_cluster(shells)[0]
    E = 0.1 + 0.15j
    _, ti = orc.square_well(2, E, -1.2, wl.R_MT)
    M = orc.assemble(pos, 2, E, np.tile(ti, (pos.shape[0], 1)))
    tau, _ = orc.first_block(M, 9)
    s = np.abs(tau).max()
    l = l_of_L(2)
    odd = (np.add.outer(l, l) % 2) == 1
    assert np.abs(tau[odd]).max() < 1e-12 * s
    p = tau[1:4, 1:4]
    assert np.abs(p - p[0, 0] * np.eye(3)).max() < 1e-12 * s
    d = tau[4:9, 4:9]
    assert np.abs(d - np.diag(np.diag(d))).max() < 1e-12 * s
    dd = np.diag(d)   # order m = -2 (xy), -1 (yz), 0 (z^2), 1 (xz), 2 (x^2-y^2)
    assert abs(dd[0] - dd[1]) < 1e-12 * s and abs(dd[0] - dd[3]) < 1e-12 * s
    assert abs(dd[2] - dd[4]) < 1e-12 * s
    assert abs(dd[0] - dd[2]) > 1e-6 * s


# ----------------------------------------------------------- canted -------

def _su2(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    sx = np.array([[0, 1], [1, 0]], complex)
    sy = np.array([[0, -1j], [1j, 0]], complex)
    sz = np.array([[1, 0], [0, -1]], complex)
    sn = axis[0] * sx + axis[1] * sy + axis[2] * sz
    return np.cos(angle / 2) * np.eye(2) - 1j * np.sin(angle / 2) * sn


def _rot(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def _canted_setup(orc, lmax=1, shells=1, seed=7):
    rng = np.random.default_rng(seed)
    pos = wl.fcc_cluster(shells)[0]
    N = pos.shape[0]
    E = 0.25 + 0.1j
    spc = rng.integers(0, 2, N)
    tu = np.array([orc.square_well(lmax, E, wl.V_SPECIES[s] - 0.05, wl.R_MT)[1] for s in spc])
    td = np.array([orc.square_well(lmax, E, wl.V_SPECIES[s] + 0.05, wl.R_MT)[1] for s in spc])
    return pos, E, tu, td, wl.random_unit_vectors(rng, N)


def test_canted_collinear_limit(orc):
    pos, E, tu, td, _ = _canted_setup(orc)
    N, nl = pos.shape[0], 4
    dirs = np.tile([0.0, 0.0, 1.0], (N, 1))
    M = orc.assemble(pos, 1, E, tu, td, dirs)
    assert M.shape == (2 * N * nl, 2 * N * nl)
    tau, _ = orc.first_block(M, 2 * nl)
    up, _ = orc.first_block(orc.assemble(pos, 1, E, tu), nl)
    dn, _ = orc.first_block(orc.assemble(pos, 1, E, td), nl)
    assert rel(tau[:nl, :nl], up) < 1e-13 and rel(tau[nl:, nl:], dn) < 1e-13
    assert np.abs(tau[:nl, nl:]).max() < 1e-14 * np.abs(tau).max()


def test_canted_global_rotation_covariance(orc):
    """Rotating every moment by R: tau_00 -> (U x 1) tau_00 (U x 1)^dagger, U in SU(2)."""
    pos, E, tu, td, dirs = _canted_setup(orc)
    axis, ang = [0.3, -0.5, 0.8], 0.9
    tau, _ = orc.first_block(orc.assemble(pos, 1, E, tu, td, dirs), 8)
    dirs2 = dirs @ _rot(axis, ang).T
    tau2, _ = orc.first_block(orc.assemble(pos, 1, E, tu, td, dirs2), 8)
    W = np.kron(_su2(axis, ang), np.eye(4))
    assert rel(tau2, W @ tau @ W.conj().T) < 1e-12


def test_canted_time_reversal(orc):
    """tau(e)^T = (sigma_y x 1) tau(-e) (sigma_y x 1)."""
    pos, E, tu, td, dirs = _canted_setup(orc)
    tau, _ = orc.first_block(orc.assemble(pos, 1, E, tu, td, dirs), 8)
    taum, _ = orc.first_block(orc.assemble(pos, 1, E, tu, td, -dirs), 8)
    Sy = np.kron(np.array([[0, -1j], [1j, 0]]), np.eye(4))
    assert rel(tau.T, Sy @ taum @ Sy) < 1e-12
