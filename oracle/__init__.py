"""CPU oracle for the LSMS tau_00 hot path -- TEST INFRASTRUCTURE ONLY.

Plain complex128 implementation of what the library computes (arXiv
2308.16317, Eq. 4 and Secs. 2.1-2.2, 3.2): free-electron structure constants
from Gaunt coefficients, spherical Hankel functions and real Y_L; square-well
single-site t-matrices; the KKR matrix M = t^{-1} - g0 over a local
interaction zone; and tau_00 = [M^{-1}]_00 by LU with partial pivoting plus
iterative refinement on a double-double residual.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arm of ``bench.py`` may import this package.  It shares no code with the CUDA
library; the two meet only through the seeded input generator
(``paper_2308_16317_gb300.workload``), which holds none of the method's
arithmetic.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, special cases, library cross-checks and brute force).  The MLP
reference (``oracle.mlp``) is pinned by finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "must_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain -O2, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            c_int, c_dbl = ctypes.c_int, ctypes.c_double
            sig = {
                "orc_sph_jyh": (None, [c_int, c_dbl, c_dbl, D, D, D]),
                "orc_real_ylm": (None, [c_int, c_dbl, c_dbl, c_dbl, D]),
                "orc_gauss_legendre": (None, [c_int, D, D]),
                "orc_gaunt": (None, [c_int, c_int, c_int, D]),
                "orc_struct_const": (None, [c_int, c_dbl, c_dbl, D, D]),
                "orc_square_well": (None, [c_int, c_dbl, c_dbl, c_dbl, c_dbl, D, D]),
                "orc_assemble": (None, [c_int, D, c_int, c_dbl, c_dbl, D, D, D, D]),
                "orc_lu_solve": (c_int, [c_int, D, c_int, D]),
                "orc_first_block": (c_dbl, [c_int, D, c_int, D, I]),
                "orc_inverse": (c_int, [c_int, D, D]),
                "orc_tau00_batch": (c_int, [c_int, D, c_int, c_int, D, D, D, D, c_int, D, D, I]),
                "orc_kkr_lattice_sum": (None, [c_int, c_dbl, c_dbl, D, D, D, c_dbl, c_dbl, D]),
                "orc_kkr_struct_const": (None, [c_int, c_dbl, c_dbl, D, c_int, D, D, c_dbl, c_dbl, D]),
                "orc_kkr_tau": (c_int, [c_int, D, c_int, D, c_int, D, D, c_int, c_dbl, c_dbl, c_int, D]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def nL(lmax: int) -> int:
    return (lmax + 1) ** 2


def l_of_L(lmax: int) -> np.ndarray:
    """l for each L = l*l + l + m, m = -l..l."""
    return np.array([l for l in range(lmax + 1) for _ in range(2 * l + 1)])


# -- special functions ------------------------------------------------------

def sph_jy(lmax: int, z: complex):
    """Spherical Bessel j_l(z), y_l(z), l = 0..lmax (A&S 10.1)."""
    return sph_jyh(lmax, z)[:2]


def sph_jyh(lmax: int, z: complex):
    """j_l(z), y_l(z) and the outgoing Hankel h_l(z) (closed form), l = 0..lmax."""
    j = np.zeros(lmax + 1, np.complex128)
    y = np.zeros(lmax + 1, np.complex128)
    h = np.zeros(lmax + 1, np.complex128)
    _load().orc_sph_jyh(lmax, float(np.real(z)), float(np.imag(z)), _dp(j.view(np.float64)), _dp(y.view(np.float64)),
                        _dp(h.view(np.float64)))
    return j, y, h


def real_ylm(lmax: int, v) -> np.ndarray:
    """Real spherical harmonics Y_L(v^), L = l*l + l + m (no Condon-Shortley phase)."""
    out = np.zeros(nL(lmax))
    _load().orc_real_ylm(lmax, float(v[0]), float(v[1]), float(v[2]), _dp(out))
    return out


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().orc_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def gaunt(l1max: int, l2max: int, l3max: int) -> np.ndarray:
    """C[L1, L2, L3] = int Y_L1 Y_L2 Y_L3 dOmega (product quadrature)."""
    C = np.zeros((nL(l1max), nL(l2max), nL(l3max)))
    _load().orc_gaunt(l1max, l2max, l3max, _dp(C))
    return C


def struct_const(lmax: int, E: complex, R) -> np.ndarray:
    """Free-electron structure-constant block G_{LL'}(R), R = R_i - R_j (Eq. 4's g0)."""
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    G = np.zeros((nL(lmax), nL(lmax)), np.complex128)
    _load().orc_struct_const(lmax, float(np.real(E)), float(np.imag(E)), _dp(R), _dp(G.view(np.float64)))
    return G


def square_well(lmax: int, E: complex, V: float, a: float):
    """(t_l, t_l^{-1}) for a square well of depth V and radius a, l = 0..lmax."""
    t = np.zeros(lmax + 1, np.complex128)
    ti = np.zeros(lmax + 1, np.complex128)
    _load().orc_square_well(lmax, float(np.real(E)), float(np.imag(E)), float(V), float(a),
                            _dp(t.view(np.float64)), _dp(ti.view(np.float64)))
    return t, ti


def site_tinv(lmax: int, E: complex, V_sites, a: float) -> np.ndarray:
    """t^{-1}_l for every site, [N][lmax+1], from each site's well depth."""
    out = np.zeros((len(V_sites), lmax + 1), np.complex128)
    cache = {}
    for i, V in enumerate(V_sites):
        key = float(V)
        if key not in cache:
            cache[key] = square_well(lmax, E, key, a)[1]
        out[i] = cache[key]
    return out


# -- KKR matrix and tau_00 --------------------------------------------------

def assemble(pos, lmax: int, E: complex, tinv_a, tinv_b=None, dirs=None) -> np.ndarray:
    """KKR matrix M = t^{-1} - g0 (row-major, centre site first)."""
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    N = pos.shape[0]
    spins = 1 if dirs is None else 2
    n = spins * N * nL(lmax)
    M = np.zeros((n, n), np.complex128)
    ta = _c128(tinv_a)
    tb = _c128(tinv_b) if tinv_b is not None else None
    dd = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64)) if dirs is not None else None
    _load().orc_assemble(N, _dp(pos), lmax, float(np.real(E)), float(np.imag(E)), _dp(ta.view(np.float64)),
                         _dp(tb.view(np.float64)) if tb is not None else None,
                         _dp(dd) if dd is not None else None, _dp(M.view(np.float64)))
    return M


def lu_solve(A, B) -> np.ndarray:
    A = _c128(A)
    X = _c128(B).copy()
    if X.ndim == 1:
        X = X[:, None]
    _load().orc_lu_solve(A.shape[0], _dp(A.view(np.float64)), X.shape[1], _dp(X.view(np.float64)))
    return X


def first_block(M, kap: int):
    """(tau, rel_correction): first kap x kap block of M^{-1}, refined."""
    M = _c128(M)
    tau = np.zeros((kap, kap), np.complex128)
    st = np.zeros(1, np.int32)
    err = _load().orc_first_block(M.shape[0], _dp(M.view(np.float64)), kap, _dp(tau.view(np.float64)), _ip(st))
    return tau, err


def inverse(A) -> np.ndarray:
    """Full inverse by Gauss-Jordan (tiny matrices only)."""
    A = _c128(A)
    out = np.zeros_like(A)
    s = _load().orc_inverse(A.shape[0], _dp(A.view(np.float64)), _dp(out.view(np.float64)))
    if s:
        raise ZeroDivisionError("singular matrix")
    return out


def tau00_batch(pos, lmax: int, E, tinv_a, tinv_b=None, dirs=None, nthreads: int = 0):
    """tau_00 for many independent items over one LIZ geometry.

    E: [n_items] complex; tinv_a (and tinv_b for canted): [n_items][N][lmax+1].
    Returns (tau [n_items][kap][kap], rel_correction [n_items], threads_used).
    """
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    N = pos.shape[0]
    E = _c128(E).reshape(-1)
    n_items = E.shape[0]
    spins = 1 if dirs is None else 2
    kap = spins * nL(lmax)
    ta = _c128(tinv_a).reshape(n_items, N, lmax + 1)
    tb = _c128(tinv_b).reshape(n_items, N, lmax + 1) if tinv_b is not None else None
    dd = np.ascontiguousarray(np.asarray(dirs, dtype=np.float64)) if dirs is not None else None
    tau = np.zeros((n_items, kap, kap), np.complex128)
    err = np.zeros(n_items)
    st = np.zeros(n_items, np.int32)
    used = _load().orc_tau00_batch(N, _dp(pos), lmax, n_items, _dp(E.view(np.float64)), _dp(ta.view(np.float64)),
                                   _dp(tb.view(np.float64)) if tb is not None else None,
                                   _dp(dd) if dd is not None else None, int(nthreads),
                                   _dp(tau.view(np.float64)), _dp(err), _ip(st))
    if st.any():
        raise ZeroDivisionError("oracle met a zero pivot")
    return tau, err, used


# -- full KKR (periodic crystal; Sec. 5) -----------------------------------

def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def kkr_lattice_sum(l2max: int, E: complex, lattice, x, k, eta: float, cut: float = 50.0) -> np.ndarray:
    """Ewald lattice sum D_L(k) = sum_{R: x-R != 0} e^{ik.R} h_l(kappa|x-R|) Y_L((x-R)^), L < (l2max+1)^2.

    lattice: rows a1, a2, a3 (bohr); x = b_s - b_t; cut: truncation exponent of both sums.
    """
    D = np.zeros((l2max + 1) ** 2, np.complex128)
    lat, xx, kk = _f64(lattice, (3, 3)), _f64(x, (3,)), _f64(k, (3,))
    _load().orc_kkr_lattice_sum(l2max, float(np.real(E)), float(np.imag(E)), _dp(lat), _dp(xx), _dp(kk),
                                float(eta), float(cut), _dp(D.view(np.float64)))
    return D


def kkr_struct_const(lmax: int, E: complex, lattice, basis, k, eta: float, cut: float = 50.0) -> np.ndarray:
    """Bloch-summed structure constants G(k), n x n with n = N_b (lmax+1)^2, index (site, L)."""
    basis = _f64(basis).reshape(-1, 3)
    nb = basis.shape[0]
    n = nb * nL(lmax)
    G = np.zeros((n, n), np.complex128)
    lat, kk = _f64(lattice, (3, 3)), _f64(k, (3,))
    _load().orc_kkr_struct_const(lmax, float(np.real(E)), float(np.imag(E)), _dp(lat), nb, _dp(basis), _dp(kk),
                                 float(eta), float(cut), _dp(G.view(np.float64)))
    return G


def kkr_tau(lmax: int, lattice, basis, E, tinv, nk: int, eta: float, cut: float = 50.0, nthreads: int = 0):
    """Site-diagonal scattering-path blocks of the crystal, tau^{ss}(E) = <[t^{-1} - G(k)]^{-1}>_BZ.

    E: [n_items] complex; tinv: [n_items][N_b][lmax+1]; Gamma-centred uniform mesh of nk^3 points.
    Returns (tau [n_items][N_b][kap][kap], threads_used).
    """
    basis = _f64(basis).reshape(-1, 3)
    nb = basis.shape[0]
    E = _c128(E).reshape(-1)
    n_items = E.shape[0]
    ti = _c128(tinv).reshape(n_items, nb, lmax + 1)
    kap = nL(lmax)
    tau = np.zeros((n_items, nb, kap, kap), np.complex128)
    lat = _f64(lattice, (3, 3))
    used = _load().orc_kkr_tau(lmax, _dp(lat), nb, _dp(basis), n_items, _dp(E.view(np.float64)),
                               _dp(ti.view(np.float64)), int(nk), float(eta), float(cut), int(nthreads),
                               _dp(tau.view(np.float64)))
    if used < 0:
        raise ZeroDivisionError("oracle met a singular M(k)")
    return tau, used
