"""Checks on the seeded input generator against what the paper fixes (ranks,
LIZ sizes) and the stated workload recipe (contour, vacancies, species)."""
import os

import numpy as np

from paper_2308_16317_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_ranks.txt")


def test_paper_ranks_from_fcc_shells():
    """Sec. 2.1/2.2 rank rule with the paper's printed ranks (Sec. 3, 4.1)."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for label, lmax, nliz, canted, rank, shells, *_ in rows:
        lmax, nliz, canted, rank, shells = map(int, (lmax, nliz, canted, rank, shells))
        pos, _ = wl.fcc_cluster(shells)
        assert pos.shape[0] == nliz, label
        assert (2 if canted else 1) * nliz * (lmax + 1) ** 2 == rank, label


def test_fcc_shell_counts_and_order():
    off, shell, radii = wl.fcc_shell_table(12)
    counts = np.cumsum(np.bincount(shell))
    assert counts.tolist() == [1, 13, 19, 43, 55, 79, 87, 135, 141, 177, 201, 225, 249]
    assert np.all(off[0] == 0)
    assert np.all(np.diff(shell) >= 0)
    d = np.sqrt((off ** 2).sum(1)) * wl.A_LAT / 2
    assert abs(d[1] - wl.A_LAT / np.sqrt(2)) < 1e-12          # nearest neighbour a/sqrt2
    assert abs(d[134] - np.sqrt(14) * wl.A_LAT / 2) < 1e-12   # shell 7 radius


def test_contour_nodes():
    E = wl.semicircle_contour(32)
    assert abs(E.imag.min() - 0.00215) < 2e-5 and E.imag.max() < 0.5
    assert np.allclose(np.abs(E - 0.2), 0.5)
    assert E.real[0] < -0.29 and E.real[-1] > 0.69          # ordered E_bot -> E_F
    assert wl.semicircle_contour(32, im_min=0.005).imag.min() == 0.005
    assert wl.semicircle_contour(8).imag.min() > 0.03


def test_configs_shapes():
    w1 = wl.first_shell_small()
    assert w1.n_of(w1.lizs[0]) == 117 and w1.kappa() == 9 and len(w1.energies) == 8
    w2 = wl.liz135()
    assert w2.n_of(w2.lizs[0]) == 2160 and w2.nspin == 2 and len(w2.energies) == 32
    assert np.allclose(w2.v_species, [[-1.05, -1.45], [-0.95, -1.35]])
    w4 = wl.canted135()
    assert w4.n_of(w4.lizs[0]) == 4320 and w4.kappa() == 32
    assert np.allclose(np.linalg.norm(w4.lizs[0].dirs, axis=1), 1.0)


def test_supercell_vacancy_recipe():
    w = wl.batched_supercell()
    sizes = np.array([l.n_sites for l in w.lizs])
    assert len(w.lizs) == 256
    assert sizes.min() >= 43 and sizes.max() <= 135
    assert set(np.unique(sizes)) & {43, 55, 79, 87}          # full cut-offs without vacancies occur
    for l in w.lizs:
        assert np.all(l.pos[0] == 0)
    # exact 50/50 species over the supercell
    rng = np.random.default_rng(wl.SEED_BASE + 3)
    _, sp = wl.supercell_species(rng)
    assert sp.sum() == 128
    # deterministic from the seed
    w_again = wl.batched_supercell()
    assert all(np.array_equal(a.species, b.species) for a, b in zip(w.lizs, w_again.lizs))


def test_paper_shaped_workloads_have_the_paper_ranks():
    """Sec. 4.1: NiAu rank 6225 (249 sites, lmax 4), CoCrFeMnNi canted rank 6750."""
    w = wl.niau249()
    assert w.lizs[0].pos.shape[0] * w.kappa() == 6225 and not w.canted
    frac_ni = float((w.lizs[0].species == 0).mean())
    assert 0.2 < frac_ni < 0.4
    w = wl.cocrfemnni135_canted()
    assert w.lizs[0].pos.shape[0] * w.kappa() == 6750 and w.canted
    assert set(np.unique(w.lizs[0].species)) == set(range(5))
    assert np.allclose(np.linalg.norm(w.lizs[0].dirs, axis=1), 1.0)
