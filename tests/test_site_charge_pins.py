"""Pins of the oracle's site charge (oracle/site_charge.py): the radial
integrals against quadrature, the contour weights, path independence of the
contour integral, the free-electron limit, slope continuity of the regular
solution at the sphere, and the weight of the bound state inside the sphere
(from its wave function, with no Green's function involved)."""
import numpy as np
import pytest

import oracle
from oracle import site_charge as sc

A = 2.50545   # r_mt of the workloads (bohr)


def test_lommel_matches_quadrature():
    from scipy.integrate import quad
    from scipy.special import spherical_jn, spherical_yn
    for q in (0.7, 1.3):
        jq, yq = sc._jy_ext(4, q * A)
        for l in range(5):
            ljj = sc.lommel(l, q * A, jq, jq).real / q ** 3
            ljy = sc.lommel(l, q * A, jq, yq, lower=(2 * l + 1) / 4.0).real / q ** 3
            rjj = quad(lambda r: spherical_jn(l, q * r) ** 2 * r * r, 0, A)[0]
            rjy = quad(lambda r: spherical_jn(l, q * r) * spherical_yn(l, q * r) * r * r, 0, A, limit=200)[0]
            assert abs(ljj - rjj) <= 1e-13 * max(1.0, abs(rjj))
            assert abs(ljy - rjy) <= 1e-12 * max(1.0, abs(rjy))


def test_contour_weights_integrate_polynomials():
    E, w = sc.contour_weights(32)
    for m in range(4):
        exact = (0.7 ** (m + 1) - (-0.3) ** (m + 1)) / (m + 1)
        assert abs(np.sum(w * E ** m) - exact) <= 1e-13


def test_regular_solution_slope_is_continuous():
    """Z_l inside is fixed by its value at r = a; the slope must then match the
    outside form j_l/t_l - i kappa h_l by the t-matrix definition alone."""
    for E in (0.3 + 0.05j, -0.2 + 0.1j, 0.6 + 0.4j):
        for V in (-1.0, -1.4):
            kap, q = np.sqrt(E), np.sqrt(E - V)
            t, _ = oracle.square_well(3, E, V, A)
            jk, yk = sc._jy_ext(3, kap * A)
            jq, _ = sc._jy_ext(3, q * A)
            hk = jk + 1j * yk
            for l in range(4):
                k = l + 1
                dj = lambda f, z: f[k - 1] - (l + 1) / z * f[k]
                za = jk[k] / t[l] - 1j * kap * hk[k]
                c = za / jq[k]
                slope_in = c * q * dj(jq, q * A)
                slope_out = kap * dj(jk, kap * A) / t[l] - 1j * kap * kap * dj(hk, kap * A)
                assert abs(slope_in - slope_out) <= 1e-10 * abs(slope_out)


def test_contour_integral_is_path_independent():
    """tau = t (a lone site) is analytic in the upper half plane: the semicircle
    and a rectangle over the same end points give the same N."""
    lmax, V = 3, -1.0
    E1, w1 = sc.contour_weights(48)
    taus1 = [np.diag(oracle.square_well(lmax, e, V, A)[0][oracle.l_of_L(lmax)]) for e in E1]
    _, N1 = sc.site_charge(lmax, E1, w1, V, A, taus1)
    # rectangle -0.3 -> -0.3+0.6i -> 0.7+0.6i -> 0.7, Gauss-Legendre per leg
    x, W = np.polynomial.legendre.leggauss(160)
    legs = [(-0.3 + 0j, -0.3 + 0.6j), (-0.3 + 0.6j, 0.7 + 0.6j), (0.7 + 0.6j, 0.7 + 0j)]
    E2, w2 = [], []
    for a, b in legs:
        E2 += list(0.5 * (a + b) + 0.5 * (b - a) * x)
        w2 += list(0.5 * (b - a) * W)
    taus2 = [np.diag(oracle.square_well(lmax, e, V, A)[0][oracle.l_of_L(lmax)]) for e in E2]
    _, N2 = sc.site_charge(lmax, np.array(E2), np.array(w2), V, A, taus2)
    assert abs(N1 - N2) <= 1e-7 * abs(N2)


def test_free_electron_limit():
    """V -> 0: n(E) -> (kappa / pi) sum_l (2l+1) int_0^a j_l^2 r^2 dr -> kappa a^3 / (3 pi)."""
    lmax = 12
    for E in (0.2, 0.5):
        V = -1e-7
        tau = np.diag(oracle.square_well(lmax, E, V, A)[0][oracle.l_of_L(lmax)])
        g = sc.site_integrand(lmax, E, V, A, tau)
        n = -g.imag / np.pi
        assert abs(n - np.sqrt(E) * A ** 3 / (3 * np.pi)) <= 1e-5 * n


def test_bound_state_weight_inside_the_sphere():
    """Moving the contour's lower end from below to above the l = 0 bound
    state of the V = -1.0 well changes N by that state's probability inside
    the sphere, computed from its wave function by quadrature."""
    from scipy.integrate import quad
    from scipy.optimize import brentq
    from scipy.special import spherical_jn
    lmax, V = 2, -1.0

    def N(e_bot, n=64):
        E, w = sc.contour_weights(n, e_bot=e_bot, e_f=0.7)
        taus = [np.diag(oracle.square_well(lmax, e, V, A)[0][oracle.l_of_L(lmax)]) for e in E]
        return sc.site_charge(lmax, E, w, V, A, taus)[1]

    dN = N(-0.3) - N(-0.25)
    # s-wave bound state: q cot(q a) = -gamma with q = sqrt(E - V), gamma = sqrt(-E)
    f = lambda E: np.sqrt(E - V) / np.tan(np.sqrt(E - V) * A) + np.sqrt(-E)
    Eb = brentq(f, -0.29, -0.26)
    q, g = np.sqrt(Eb - V), np.sqrt(-Eb)
    inside = quad(lambda r: spherical_jn(0, q * r) ** 2 * r * r, 0, A)[0]
    # outside u(r) = C e^{-g r} / r, continuous with j_0(q r) at r = a
    C = spherical_jn(0, q * A) * A * np.exp(g * A)
    outside = C * C * np.exp(-2 * g * A) / (2 * g)
    p_in = inside / (inside + outside)
    assert -0.3 < Eb < -0.25
    assert abs(dN - p_in) <= 1e-6


def test_radial_density_integrates_to_the_site_charge():
    """4 pi int_0^a n(r) r^2 dr (Gauss-Legendre in r) must equal the charge
    that the Lommel integrals give, for the lone-site tau = t and for a tau
    that is not t (each l channel scaled differently), both spins' depths."""
    lmax = 3
    E, w = sc.contour_weights(24)
    x, W = np.polynomial.legendre.leggauss(48)
    r, wr = 0.5 * A * (x + 1.0), 0.5 * A * W
    lL = oracle.l_of_L(lmax)
    for V in (-0.95, -1.45):
        for scale in ([1.0, 1.0, 1.0, 1.0], [1.2 + 0.1j, 0.8, 1.0 - 0.2j, 1.5]):
            taus = []
            for e in E:
                t, _ = oracle.square_well(lmax, e, V, A)
                taus.append(np.diag((t * np.asarray(scale))[lL]))
            _, N = sc.site_charge(lmax, E, w, V, A, taus)
            n = sc.radial_density(lmax, E, w, V, A, taus, r)
            assert np.isfinite(n).all()
            assert abs(4.0 * np.pi * np.sum(wr * r * r * n) - N) <= 1e-11 * abs(N)


def test_radial_density_of_a_lone_site_on_the_real_axis():
    """tau = t at one real energy above the well bottom (unit weight): the
    local density of states is kappa/(4 pi^2) sum_l (2l+1) R_l(r)^2 with the
    real regular solution R_l = cos(d_l) j_l(kappa r) - sin(d_l) y_l(kappa r)
    outside and its continuation d j_l(q r) inside, the phase shifts d_l from
    the textbook log-derivative matching (no t-matrix or Green's function)."""
    from scipy.special import spherical_jn, spherical_yn
    lmax, V = 3, -1.0
    for E in (0.15, 0.45):
        kap, q = np.sqrt(E), np.sqrt(E - V)
        t, _ = oracle.square_well(lmax, E + 0j, V, A)
        tau = np.diag(t[oracle.l_of_L(lmax)])
        r = np.linspace(0.1, 1.0, 10) * A
        n = sc.radial_density(lmax, [E + 0j], [1.0 + 0j], V, A, [tau], r)
        ref = np.zeros_like(r)
        for l in range(lmax + 1):
            jk, djk = spherical_jn(l, kap * A), spherical_jn(l, kap * A, derivative=True)
            yk, dyk = spherical_yn(l, kap * A), spherical_yn(l, kap * A, derivative=True)
            jq, djq = spherical_jn(l, q * A), spherical_jn(l, q * A, derivative=True)
            # tan d = (kap j' j_q - q j_q' j) / (kap y' j_q - q j_q' y)
            d = np.arctan2(kap * djk * jq - q * djq * jk, kap * dyk * jq - q * djq * yk)
            Ra = np.cos(d) * jk - np.sin(d) * yk
            R = Ra / jq * spherical_jn(l, q * r)
            ref += (2 * l + 1) * R * R
        ref *= kap / (4.0 * np.pi ** 2)
        assert np.abs(n - ref).max() <= 1e-12 * np.abs(ref).max(), (E, n, ref)
