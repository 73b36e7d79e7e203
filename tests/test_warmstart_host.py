"""Host-side marshalling of the learned warm start (no GPU): the contour
schedule, the one-hot occupancy and the gathering of training samples from a
batch solution, checked on CPU tensors with values that identify their
(LIZ, spin, energy) origin."""
import numpy as np
import torch

from paper_2308_16317_gb300 import warmstart as ws


def test_schedule_predicts_the_odd_interior_points():
    # even points and the last one are solved; odd k in 1..nE-3 are predicted
    assert ws.predicted_points(32) == list(range(1, 30, 2))
    assert ws.predicted_points(8) == [1, 3, 5]
    assert ws.predicted_points(3) == []
    for nE in (5, 8, 32):
        for k in ws.predicted_points(nE):
            assert k % 2 == 1 and 0 <= k - 1 and k + 1 <= nE - 1


def test_input_width():
    # both neighbours as (half-difference, mean) in re/im: 4 kap^2, one-hot pairs, 8 scalars
    assert ws.n_inputs(16) == 4 * 256 + 270 + 8 == 1302


def test_occupancy_is_one_hot_per_site():
    w = ws.random_liz_workload(100000, 1, n_e=4, lmax=1)
    liz = w.lizs[0]
    occ = ws.occupancy(liz)
    assert occ.shape == (2 * ws.N_OCC_SITES,)
    pairs = occ.reshape(-1, 2)
    n = min(len(liz.species), ws.N_OCC_SITES)
    assert (pairs[:n].sum(axis=1) == 1).all() and (pairs[n:] == 0).all()
    assert (pairs[:n, 1] == np.asarray(liz.species[:n])).all()


def test_samples_gather_the_right_neighbours():
    nE, kap, n_liz, n_out = 8, 2, 2, 2
    w = ws.random_liz_workload(100000, n_liz, n_e=nE, lmax=0)
    # tau[l][s][k] filled with a value that encodes (l, s, k)
    code = (np.arange(n_liz)[:, None, None] * 100 + np.arange(n_out)[None, :, None] * 10
            + np.arange(nE)[None, None, :]).astype(np.float64)
    tau = torch.tensor(np.broadcast_to(code[..., None, None], (n_liz, n_out, nE, kap, kap)).copy()
                       ).to(torch.complex128)
    tprev, tnext, ttgt, E3, spin, occ = ws.samples_from_solution(tau, w)
    ks = ws.predicted_points(nE)
    assert tprev.shape[0] == n_liz * n_out * len(ks)
    i = 0
    for l in range(n_liz):
        for s in range(n_out):
            for k in ks:
                assert tprev[i, 0, 0].real == l * 100 + s * 10 + k - 1
                assert tnext[i, 0, 0].real == l * 100 + s * 10 + k + 1
                assert ttgt[i, 0, 0].real == l * 100 + s * 10 + k
                assert complex(E3[i, 1]) == complex(w.energies[k])
                assert complex(E3[i, 0]) == complex(w.energies[k - 1])
                assert complex(E3[i, 2]) == complex(w.energies[k + 1])
                assert float(spin[i]) == (1.0 if s == 0 else -1.0)
                assert np.array_equal(occ[i].numpy(), ws.occupancy(w.lizs[l]))
                i += 1
