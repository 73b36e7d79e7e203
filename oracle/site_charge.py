"""Site charge inside the muffin-tin sphere from tau_00 -- TEST INFRASTRUCTURE ONLY.

Plain numpy restatement, for the square-well single-site problem, of the
Green's function of one site (Eq. 3 of the paper),
    G(r, r; E) = sum_LL' Z_L(r) tau_LL'(E) Z_L'(r) - sum_L Z_L(r) J_L(r),
integrated over the sphere r < a, and of the charge integral (Eq. 2) taken
along the complex energy contour:
    n(E) = -(1/pi) Im int_sphere G(r, r; E) d^3r,
    N    = -(1/pi) Im sum_k w_k int_sphere G(r, r; E_k) d^3r.
Conventions (readings, stated where the paper is silent): the retarded G of
this project (g0 = -e^{i kappa |x - x'|} / (4 pi |x - x'|)), hence the minus
sign in front of (1/pi) Im; outside the sphere Z_l = j_l(kappa r)/t_l -
i kappa h_l(kappa r) and J_l = j_l(kappa r) (so that tau = t reproduces the
single-site G = -i kappa sum_L R_L(r<) H_L(r>)); inside, Z_l and J_l are the
regular and irregular well solutions continued with matching value and
slope at r = a.  Real harmonics are orthonormal, so the angular integral
leaves the diagonal tau_LL.  Radial integrals by the Lommel identity
    int_0^x u_l v_l s^2 ds = (s^3/2)[u_l v_l - (u_{l-1} v_{l+1} + u_{l+1} v_{l-1})/2] |_0^x
for any two spherical-Bessel-type solutions u, v of order l (lower limit
(2l+1)/4 when one of them is y_l and the other j_l, else 0).
The radial density inside the sphere is the spherical average of the same
G(r, r; E) (real harmonics are orthonormal, and sum_m Y_lm^2 = (2l+1)/(4 pi)):
    n(r) = -(1/pi) Im sum_k w_k (1/(4 pi)) [sum_L tau_LL Z_l(r)^2
                                            - sum_l (2l+1) Z_l(r) J_l(r)],
so that 4 pi int_0^a n(r) r^2 dr = N.
Pinned in tests/test_site_charge_pins.py (quadrature of the radial
integrals, contour weights, path independence, free-electron limit, the
radial quadrature of n(r) against N, and n(r) on the real axis).
"""
from __future__ import annotations

import numpy as np

import oracle


def _jy_ext(lmax: int, z: complex):
    """j_l, y_l for l = -1 .. lmax+1 (index l+1); j_{-1} = cos z / z, y_{-1} = sin z / z."""
    j, y, _ = oracle.sph_jyh(lmax + 1, z)
    jm = np.cos(z) / z
    ym = np.sin(z) / z
    return np.concatenate([[jm], j]), np.concatenate([[ym], y])


def lommel(l: int, x: complex, u, v, lower: float = 0.0) -> complex:
    """(x^3/2)[u_l v_l - (u_{l-1} v_{l+1} + u_{l+1} v_{l-1})/2] - lower, with u, v indexed l+1."""
    k = l + 1
    return x ** 3 / 2.0 * (u[k] * v[k] - 0.5 * (u[k - 1] * v[k + 1] + u[k + 1] * v[k - 1])) - lower


def inside_coefficients(lmax: int, E: complex, V: float, a: float):
    """Per l: c, alpha, beta of Z_l = c j_l(q r) and J_l = alpha j_l(q r) + beta y_l(q r)
    inside the well (value of Z and value and slope of J matched at r = a), and t_l."""
    kap = np.sqrt(complex(E))
    q = np.sqrt(complex(E) - V)
    t, _ = oracle.square_well(lmax, E, V, a)
    jk, yk = _jy_ext(lmax, kap * a)
    jq, yq = _jy_ext(lmax, q * a)
    _, _, hk = oracle.sph_jyh(lmax + 1, kap * a)
    c = np.zeros(lmax + 1, np.complex128)
    al = np.zeros(lmax + 1, np.complex128)
    be = np.zeros(lmax + 1, np.complex128)
    for l in range(lmax + 1):
        k = l + 1
        # derivatives d/dz f_l(z) = f_{l-1} - (l+1)/z f_l
        djk = jk[k - 1] - (l + 1) / (kap * a) * jk[k]
        djq = jq[k - 1] - (l + 1) / (q * a) * jq[k]
        dyq = yq[k - 1] - (l + 1) / (q * a) * yq[k]
        # regular: Z_l(a) = j_l(kap a)/t_l - i kap h_l(kap a), inside c j_l(q r)
        c[l] = (jk[k] / t[l] - 1j * kap * hk[l]) / jq[k]
        # irregular: alpha j_l(q r) + beta y_l(q r) with value j_l(kap a) and slope kap j_l'(kap a)
        A = np.array([[jq[k], yq[k]], [q * djq, q * dyq]])
        al[l], be[l] = np.linalg.solve(A, np.array([jk[k], kap * djk]))
    return c, al, be, t


def radial_integrals(lmax: int, E: complex, V: float, a: float):
    """F_l = int_0^a Z_l^2 r^2 dr and I_l = int_0^a Z_l J_l r^2 dr, l = 0..lmax, and t_l."""
    kap = np.sqrt(complex(E))
    q = np.sqrt(complex(E) - V)
    t, _ = oracle.square_well(lmax, E, V, a)
    jk, yk = _jy_ext(lmax, kap * a)
    jq, yq = _jy_ext(lmax, q * a)
    _, _, hk = oracle.sph_jyh(lmax + 1, kap * a)
    F = np.zeros(lmax + 1, np.complex128)
    I = np.zeros(lmax + 1, np.complex128)
    for l in range(lmax + 1):
        k = l + 1
        # derivatives d/dz f_l(z) = f_{l-1} - (l+1)/z f_l
        djk = jk[k - 1] - (l + 1) / (kap * a) * jk[k]
        djq = jq[k - 1] - (l + 1) / (q * a) * jq[k]
        dyq = yq[k - 1] - (l + 1) / (q * a) * yq[k]
        # regular: Z_l(a) = j_l(kap a)/t_l - i kap h_l(kap a), inside c j_l(q r)
        Za = jk[k] / t[l] - 1j * kap * hk[l]
        c = Za / jq[k]
        # irregular: alpha j_l(q r) + beta y_l(q r) with value j_l(kap a) and slope kap j_l'(kap a)
        A = np.array([[jq[k], yq[k]], [q * djq, q * dyq]])
        alpha, beta = np.linalg.solve(A, np.array([jk[k], kap * djk]))
        x = q * a
        Ljj = lommel(l, x, jq, jq) / q ** 3
        Ljy = lommel(l, x, jq, yq, lower=(2 * l + 1) / 4.0) / q ** 3
        F[l] = c * c * Ljj
        I[l] = c * (alpha * Ljj + beta * Ljy)
    return F, I, t


def contour_weights(n_e: int, e_bot: float = -0.3, e_f: float = 0.7):
    """Nodes and weights of int_{e_bot}^{e_f} f(E) dE along the upper semicircle:
    Gauss-Legendre in the angle theta (theta = pi/2 (1 - x), from pi to 0)."""
    x, W = np.polynomial.legendre.leggauss(n_e)
    theta = 0.5 * np.pi * (1.0 - x)
    c, r = 0.5 * (e_bot + e_f), 0.5 * (e_f - e_bot)
    E = c + r * np.exp(1j * theta)
    w = W * (-0.5 * np.pi) * (1j * r * np.exp(1j * theta))
    return E, w


def site_integrand(lmax: int, E: complex, V: float, a: float, tau: np.ndarray) -> complex:
    """int_sphere G(r, r; E) d^3r for the centre site with diagonal tau_LL."""
    F, I, _ = radial_integrals(lmax, E, V, a)
    lL = oracle.l_of_L(lmax)
    return complex(np.sum(np.diag(tau) * F[lL]) - np.sum((2 * np.arange(lmax + 1) + 1) * I))


def site_charge(lmax: int, E, w, V: float, a: float, taus):
    """n(E_k) per node and N = -(1/pi) Im sum_k w_k int_sphere G(E_k)."""
    g = np.array([site_integrand(lmax, e, V, a, t) for e, t in zip(E, taus)])
    return -np.imag(g) / np.pi, float(-np.imag(np.sum(np.asarray(w) * g)) / np.pi)


def radial_density(lmax: int, E, w, V: float, a: float, taus, r):
    """n(r) inside the sphere (0 < r <= a): -(1/pi) Im sum_k w_k (1/4pi) [sum_L tau_LL Z_l^2
    - sum_l (2l+1) Z_l J_l] at the radii r."""
    r = np.asarray(r, dtype=np.float64)
    lL = oracle.l_of_L(lmax)
    acc = np.zeros(r.shape, np.complex128)
    for e, wk, tau in zip(E, w, taus):
        q = np.sqrt(complex(e) - V)
        c, al, be, _ = inside_coefficients(lmax, e, V, a)
        d = np.array([np.sum(np.diag(tau)[lL == l]) for l in range(lmax + 1)])
        g = np.zeros(r.shape, np.complex128)
        for i, ri in enumerate(r.ravel()):
            jq, yq = _jy_ext(lmax, q * ri)
            Z = c * jq[1:lmax + 2]
            J = al * jq[1:lmax + 2] + be * yq[1:lmax + 2]
            g.ravel()[i] = np.sum(d * Z * Z) - np.sum((2 * np.arange(lmax + 1) + 1) * Z * J)
        acc += wk * g
    return -np.imag(acc) / (4.0 * np.pi * np.pi)
