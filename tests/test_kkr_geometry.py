"""Host set-up of the full-KKR path (periodic crystal, Sec. 5), through
must_kkr_geometry and without a GPU: the point group the library finds, the
orbits of the k mesh it inverts, the site displacements and the real- and
reciprocal-space vector counts, each recounted here in numpy by brute force
(independent of the library's host code)."""
import itertools

import numpy as np
import pytest

from paper_2308_16317_gb300 import workload as wl

CUT, ECAP = 40.0, 1.5      # Gaussian cut e^{-40}; energies up to Re E = 1.5 Ry


@pytest.fixture(scope="module")
def B():
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _signed_perms():
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            g = np.zeros((3, 3))
            for r in range(3):
                g[r, perm[r]] = signs[r]
            yield g


def _is_lattice_vector(v, lattice):
    f = np.linalg.solve(np.asarray(lattice, float).T, v)
    return np.abs(f - np.round(f)).max() < 1e-8


def _point_group(lattice, basis, classes):
    """Signed axis permutations mapping the lattice onto itself and every site
    onto a site of its own class, modulo the lattice."""
    lat = np.asarray(lattice, float)
    ops = []
    for g in _signed_perms():
        if not all(_is_lattice_vector(g @ a, lat) for a in lat):
            continue
        ok = True
        for t, bt in enumerate(basis):
            hits = [u for u, bu in enumerate(basis) if _is_lattice_vector(g @ bt - bu, lat)]
            if len(hits) != 1 or classes[hits[0]] != classes[t]:
                ok = False
                break
        if ok:
            ops.append(g)
    return ops


def _mesh(lattice, n_k):
    """Gamma-centred mesh: integer coordinates m and Cartesian k (folded)."""
    Bv = 2 * np.pi * np.linalg.inv(np.asarray(lattice, float)).T     # rows: reciprocal vectors
    m = np.array(list(itertools.product(range(n_k), repeat=3)))
    f = np.where(2 * m > n_k, m - n_k, m)
    return m, (f / n_k) @ Bv, Bv


def _orbits(lattice, n_k, ops):
    """One representative mesh index per orbit of the group generated by ops
    and k -> -k (the sign flip of all axes)."""
    lat = np.asarray(lattice, float)
    m, k, _ = _mesh(lattice, n_k)
    index = {tuple(v): i for i, v in enumerate(m)}
    ops = list(ops) + [-np.eye(3)]
    seen, reps = np.zeros(len(m), bool), []
    for i in range(len(m)):
        if seen[i]:
            continue
        reps.append(i)
        stack = [i]
        seen[i] = True
        while stack:
            j = stack.pop()
            for g in ops:
                mm = tuple(int(round(x)) % n_k for x in lat @ (g @ k[j]) / (2 * np.pi) * n_k)
                jj = index[mm]
                if not seen[jj]:
                    seen[jj] = True
                    stack.append(jj)
    return reps, k


def _default_eta(lattice, n_basis):
    omega = abs(np.linalg.det(np.asarray(lattice, float)))
    return 4 * np.pi / omega ** (2 / 3) * (0.7 if n_basis == 1 else 1.0)


def _lattice_points(lat, center, rmax):
    lat = np.asarray(lat, float)
    n = int(rmax / np.min(np.linalg.norm(lat, axis=1)) * 2) + 3
    g = np.arange(-n, n + 1)
    v = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) @ lat
    return v[np.linalg.norm(v - center, axis=1) <= rmax]


def _recount(c, classes, n_k, flags=0):
    basis = np.asarray(c.basis, float)
    nb = len(basis)
    ops = [] if flags else _point_group(c.lattice, basis, classes)
    if len(ops) <= 1:
        ops = []
    reps, k = _orbits(c.lattice, n_k, ops)
    eta = _default_eta(c.lattice, nb)
    # reciprocal terms: |k + K| <= sqrt(eta cut + E_cap) for each inverted k
    qmax = np.sqrt(eta * CUT + ECAP)
    _, _, Bv = _mesh(c.lattice, n_k)
    Ks = _lattice_points(Bv, np.zeros(3), qmax + np.linalg.norm(k, axis=1).max())
    n_kK = sum(int((np.linalg.norm(k[i] + Ks, axis=1) <= qmax).sum()) for i in reps)
    # displacements b_s - b_t: 0 and the nonzero ones; a pair (x, -x) shares its points
    disp = {tuple(basis[s] - basis[t]) for s in range(nb) for t in range(nb)}
    nonzero = sorted(x for x in disp if any(x))
    groups = {min(x, tuple(-np.asarray(x) + 0.0)) for x in nonzero}
    rho_max = np.sqrt(4 * (CUT + ECAP / eta) / eta)
    R0 = _lattice_points(c.lattice, np.zeros(3), rho_max)
    n_pts0 = (len(R0) - 1) // 2                                        # one of each pair {R, -R}
    n_pts = n_pts0
    for x in groups:
        pts = _lattice_points(c.lattice, np.asarray(x), rho_max)
        n_pts += int((np.linalg.norm(np.asarray(x) - pts, axis=1) > 1e-10).sum())
    return dict(n=nb * (c.lmax + 1) ** 2, n_kpts=len(reps), n_disp=len(disp), n_pts=n_pts, n_kK=n_kK,
                n_mesh=n_k ** 3, n_pts0=n_pts0, n_ops=len(ops)), eta


CASES = [
    ("fcc primitive", wl.fcc_crystal(lmax=3), [0], 8, 0, 48),
    ("fcc primitive odd mesh", wl.fcc_crystal(lmax=2), [0], 5, 0, 48),
    ("L12 with classes", wl.l12_crystal(lmax=1), [1, 0, 0, 0], 6, 0, 48),
    ("L12 without classes", wl.l12_crystal(lmax=1), None, 6, 0, 8),
    ("L12 no symmetry", wl.l12_crystal(lmax=1), [1, 0, 0, 0], 4, 1, 0),
    ("fcc cubic cell, one class", wl.l12_crystal(lmax=1), [0, 0, 0, 0], 5, 0, 48),
]


@pytest.mark.parametrize("name,c,classes,n_k,flags,n_ops", CASES, ids=[x[0] for x in CASES])
def test_kkr_geometry_matches_a_brute_force_recount(B, name, c, classes, n_k, flags, n_ops):
    got = B.must_kkr_geometry(c.lattice, c.basis, c.lmax, n_k, flags=flags, site_class=classes)
    cls = list(range(c.n_basis)) if classes is None else classes
    want, eta = _recount(c, cls, n_k, flags)
    assert got["n_ops"] == n_ops
    assert abs(got["eta"] - eta) <= 1e-14 * eta
    for key, v in want.items():
        assert got[key] == v, (key, got[key], v)
    assert got["n_kg"] >= 1


def test_kkr_geometry_pair_count_without_symmetry(B):
    """k / -k pairing: (n^3 + self-paired points) / 2, the self-paired points
    being the 8 (n even) or 1 (n odd) with 2m = 0 mod n."""
    c = wl.fcc_crystal(lmax=1)
    for n_k in (4, 5, 6, 7):
        got = B.must_kkr_geometry(c.lattice, c.basis, c.lmax, n_k, flags=B.MUST_KKR_NO_SYMMETRY)
        self_paired = 8 if n_k % 2 == 0 else 1
        assert got["n_kpts"] == (n_k ** 3 + self_paired) // 2 and got["n_ops"] == 0


def test_kkr_geometry_explicit_eta_and_rejections(B):
    c = wl.l12_crystal(lmax=1)
    got = B.must_kkr_geometry(c.lattice, c.basis, c.lmax, 4, eta=0.3)
    assert got["eta"] == 0.3
    assert B.must_kkr_geometry(c.lattice, c.basis, 3, 4)["n"] == 64   # 4 sites x 16: the largest order
    with pytest.raises(B.MustError):
        B.must_kkr_geometry(c.lattice, c.basis, 4, 4)                     # 4 x 25 > 64
    with pytest.raises(B.MustError):
        B.must_kkr_geometry(c.lattice, np.vstack([c.basis, c.basis[:1] + c.lattice[1]]), 1, 4)
    # the table switch does not change the set-up; unknown flag bits are rejected
    assert B.must_kkr_geometry(c.lattice, c.basis, 1, 4, flags=B.MUST_KKR_NO_TABLE) == \
        B.must_kkr_geometry(c.lattice, c.basis, 1, 4)
    with pytest.raises(B.MustError):
        B.must_kkr_geometry(c.lattice, c.basis, 1, 4, flags=4)
