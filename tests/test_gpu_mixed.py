"""GPU parity of the mixed-precision path (FP32 factors with tensor-core
trailing updates, FP64 residual refinement) against the CPU oracle: relative
Frobenius error per (energy, spin) <= 1e-9, including the points closest to
the real axis; and the status reporting of the refinement loop."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau, rel_fro
from paper_2308_16317_gb300 import workload as wl

pytestmark = pytest.mark.gpu
TOLMIX = 1e-9
PRECISIONS = [1, 2]   # MUST_MIXED_BF16X3, MUST_MIXED_TF32X3


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _gpu_tau(B, w, precision, **kw):
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    s = Session(w)
    opts = B.must_default_opts(precision, **kw)
    tau, st = s.solve(opts)
    return blocks_to_numpy(tau), st.cpu().numpy()


@pytest.mark.parametrize("residual", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mixed_first_shell(B, orc, precision, residual):
    w = wl.first_shell_small()
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w)
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, 9, 9), ref).max() <= TOLMIX


@pytest.mark.parametrize("residual", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("shells,lmax,seed", [(2, 3, 1), (3, 2, 2), (3, 3, 5)])
def test_mixed_ragged_sizes(B, orc, precision, shells, lmax, seed, residual):
    """n = 304, 387, 688: several 128-row tensor-core tiles plus ragged tails."""
    rng = np.random.default_rng(seed)
    pos, _ = wl.fcc_cluster(shells)
    liz = wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))
    w = wl.Workload("ragged", lmax, [liz], wl.semicircle_contour(6), wl.spin_depths(2), wl.R_MT)
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, w.kappa(), w.kappa()), ref).max() <= TOLMIX


@pytest.mark.parametrize("residual", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mixed_canted_small(B, orc, precision, residual):
    rng = np.random.default_rng(9)
    pos, _ = wl.fcc_cluster(2)
    liz = wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32), wl.random_unit_vectors(rng, pos.shape[0]))
    w = wl.Workload("canted19", 2, [liz], wl.semicircle_contour(6), wl.spin_depths(2), wl.R_MT, canted=True)
    tau, st = _gpu_tau(B, w, precision, residual=residual)
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    assert (st == 0).all()
    assert rel_fro(tau.reshape(-1, 18, 18), ref).max() <= TOLMIX


def test_mixed_iteration_cap_zero_reports_noconv(B):
    w = wl.first_shell_small()
    _, st = _gpu_tau(B, w, 1, max_iter=0)
    assert (st == 5).all()


@pytest.mark.parametrize("residual", [0, 1, 2, 3])
def test_mixed_full_size_sampled(B, orc, residual):
    """n = 2160, all 64 solves in the benchmark's launch configuration;
    per-energy error against the oracle at the lowest Im E (both spins),
    mid-contour and the Fermi end."""
    w = wl.liz135()
    tau, st = _gpu_tau(B, w, 1, residual=residual)
    assert (st == 0).all() and np.isfinite(tau).all()
    items = [(0, 0), (1, 0), (0, 16), (1, 31)]
    ref, _ = oracle_tau(orc, w, items=items, nthreads=min(len(items), ncpu()))
    got = np.array([tau[s, e] for s, e in items])
    err = rel_fro(got, ref)
    print("per-energy rel err (bf16x3, residual %d):" % residual, dict(zip(map(str, items), err)))
    assert err.max() <= TOLMIX, err


@pytest.mark.parametrize("residual", [1, 3])
def test_mixed_canted_full_size_sampled(B, orc, residual):
    """Spin-canted 135-site LIZ (order 4320, kap = 32), unclamped contour
    (Im E down to 0.00215): all 32 energies on the mixed path; the two
    end-point energies, closest to the real axis, checked against the oracle
    (the golden-file tests cover them again with stored oracle values)."""
    w = wl.canted135()
    tau, st = _gpu_tau(B, w, 1, residual=residual)
    assert (st == 0).all() and np.isfinite(tau).all()
    items = [0, 31]
    ref, _ = oracle_tau(orc, w, items=items, nthreads=min(len(items), ncpu()))
    got = np.array([tau[0, e] for e in items])
    err = rel_fro(got, ref)
    print("canted per-energy rel err:", dict(zip(items, err)))
    assert err.max() <= TOLMIX, err


@pytest.mark.parametrize("case", ["odd_base", "fcc135"])
def test_streamed_update_matches_per_tile_kernel(B, orc, case):
    """The streamed trailing-update kernels (C through shared memory, or
    through registers with either A-ring depth) issue the same MMAs for every
    run length and subtract the accumulator from C the same way, so tau_00
    must agree bit for bit across all of them; against the one-CTA-per-tile
    kernel (which sums the three split products in another order) it agrees
    to the refinement tolerance.  The 42-site l_max = 2 LIZ has r = n - kap =
    369, so the last panel step starts its trailing block at an odd row (tiles
    then start one row above it)."""
    if case == "odd_base":
        pos, _ = wl.fcc_cluster(3)
        pos = pos[:42]
        rng = np.random.default_rng(11)
        w = wl.Workload("odd_base", 2, [wl.Liz(pos, rng.integers(0, 2, 42).astype(np.int32))],
                        wl.semicircle_contour(4), wl.spin_depths(2), wl.R_MT)
    else:
        w = wl.liz135(n_e=4)
    old = (B.must_tune_get(2), B.must_tune_get(3), B.must_tune_get(11))
    taus = []
    try:
        B.must_tune_set(11, 0)   # one panel step per pass: paired steps use the TMA-C kernel only
        for streamed, run in ((1, 8), (1, 1), (1, 64), (1, 3), (0, 8), (2, 8), (2, 1), (2, 64), (3, 3)):
            B.must_tune_set(2, streamed)
            B.must_tune_set(3, run)
            tau, st = _gpu_tau(B, w, 1, residual=1)
            assert (st == 0).all()
            taus.append(tau)
    finally:
        B.must_tune_set(2, old[0])
        B.must_tune_set(3, old[1])
        B.must_tune_set(11, old[2])
    for t in taus[1:4] + taus[5:9]:
        assert np.array_equal(t, taus[0])
    k = w.kappa()
    assert rel_fro(taus[4].reshape(-1, k, k), taus[0].reshape(-1, k, k)).max() <= TOLMIX
    if case == "odd_base":
        ref, _ = oracle_tau(orc, w, nthreads=ncpu())
        for t in (taus[0], taus[4]):
            assert rel_fro(t.reshape(-1, k, k), ref).max() <= TOLMIX


@pytest.mark.parametrize("case", ["fcc13", "ragged387", "canted19", "lmax4_13"])
def test_cluster_correction_matches_one_cta_correction(B, orc, case):
    """The correction on thread-block clusters of 2, 4 or 8 CTAs (knob 6 = 1,
    the default, and knob 7) and on one CTA per item (knob 6 = 0) apply the same substitutions in another
    summation order: both reach the oracle within the mixed tolerance, and
    they agree with each other to the refinement tolerance.  The cases cover
    eliminated widths r = n - kap that are not multiples of the 32-row blocks
    (117 - 9, 387 - 9, 342 - 18, 325 - 25) and several right-hand-side groups."""
    rng = np.random.default_rng(3)
    if case == "fcc13":
        w = wl.first_shell_small()
    elif case == "ragged387":
        pos, _ = wl.fcc_cluster(3)
        w = wl.Workload(case, 2, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))],
                        wl.semicircle_contour(4), wl.spin_depths(2), wl.R_MT)
    elif case == "canted19":
        pos, _ = wl.fcc_cluster(2)
        w = wl.Workload(case, 2, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32),
                                         wl.random_unit_vectors(rng, pos.shape[0]))],
                        wl.semicircle_contour(4), wl.spin_depths(2), wl.R_MT, canted=True)
    else:
        pos, _ = wl.fcc_cluster(1)
        w = wl.Workload(case, 4, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))],
                        wl.semicircle_contour(3), wl.spin_depths(2), wl.R_MT)
    k = w.kappa()
    old = (B.must_tune_get(6), B.must_tune_get(7))
    try:
        taus = []
        for kern, ctas in ((0, 4), (1, 2), (1, 4), (1, 8)):
            B.must_tune_set(6, kern)
            B.must_tune_set(7, ctas)
            tau, st = _gpu_tau(B, w, 1, residual=3)
            assert (st == 0).all()
            taus.append(tau.reshape(-1, k, k))
    finally:
        B.must_tune_set(6, old[0])
        B.must_tune_set(7, old[1])
    ref, _ = oracle_tau(orc, w, nthreads=ncpu())
    for t in taus:
        assert rel_fro(t, ref).max() <= TOLMIX
    for t in taus[1:]:
        assert rel_fro(t, taus[0]).max() <= TOLMIX


def test_persistent_u12_solve_matches_per_tile_kernel(B):
    """The persistent U12 solve (knob 9 = 1, the default) runs the same
    products in the same order as the one-CTA-per-tile kernel (knob 9 = 0):
    tau_00 is identical bit for bit, on a ragged order (n = 387) and on the
    135-site LIZ (several items per run and runs crossing items)."""
    rng = np.random.default_rng(12)
    pos, _ = wl.fcc_cluster(3)
    ws = [wl.Workload("ragged387", 2, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))],
                      wl.semicircle_contour(5), wl.spin_depths(2), wl.R_MT), wl.liz135(n_e=4)]
    old = B.must_tune_get(9)
    try:
        for w in ws:
            taus = []
            for v in (1, 0):
                B.must_tune_set(9, v)
                tau, st = _gpu_tau(B, w, 1, residual=3)
                assert (st == 0).all()
                taus.append(tau)
            assert np.array_equal(taus[0], taus[1])
    finally:
        B.must_tune_set(9, old)


def test_a_pack_placements_match(B):
    """Where the A operand (L21 as BF16 pairs) of each panel step is packed
    (knob 10: 0 a kernel on the main stream, 1 a kernel on the side stream
    into the pack's second buffer, 2 the panel kernel itself) changes where
    and when the same values are written, not the values: tau_00 is
    identical bit for bit across the three, with and without look-ahead
    (knob 4), on a ragged order (n = 387, an odd number of panel steps and a
    last panel narrower than 64) and on the 135-site LIZ (34 panel steps)."""
    rng = np.random.default_rng(13)
    pos, _ = wl.fcc_cluster(3)
    ws = [wl.Workload("ragged387", 2, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))],
                      wl.semicircle_contour(5), wl.spin_depths(2), wl.R_MT), wl.liz135(n_e=4)]
    old = (B.must_tune_get(4), B.must_tune_get(10), B.must_tune_get(11))
    try:
        B.must_tune_set(11, 0)   # paired steps keep the pack on the main stream
        for w in ws:
            taus = []
            for la, where in ((1, 0), (1, 1), (1, 2), (0, 2), (0, 1)):
                B.must_tune_set(4, la)
                B.must_tune_set(10, where)
                tau, st = _gpu_tau(B, w, 1, residual=3)
                assert (st == 0).all()
                taus.append(tau)
            for t in taus[1:]:
                assert np.array_equal(taus[0], t)
    finally:
        B.must_tune_set(4, old[0])
        B.must_tune_set(10, old[1])
        B.must_tune_set(11, old[2])


def test_concurrent_solves_on_two_streams_are_bit_identical(B):
    """Two solves running at the same time on two CUDA streams (separate
    workspaces, the same inputs) give tau_00 identical bit for bit to a solve
    running alone: no kernel may depend on what else runs on the GPU.  (The
    trailing update that takes C tiles by TMA once returned stale tiles under
    such concurrency, which the refinement mostly hid and occasionally could
    not; each of the three update kernels is checked.)"""
    import torch
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    w = wl.liz135(n_e=16)
    opts = B.must_default_opts(1, residual=3)
    old = B.must_tune_get(2)
    try:
        for kern in (3, 2, 1):
            B.must_tune_set(2, kern)
            ref, st = _gpu_tau(B, w, 1, residual=3)
            assert (st == 0).all()
            for _ in range(3):
                sa, sb = Session(w), Session(w)
                oa, ob = sa.alloc_out(1), sb.alloc_out(1)
                a, b = torch.cuda.Stream(), torch.cuda.Stream()
                torch.cuda.synchronize()
                sa.solve(opts, out=oa, stream=a)
                sb.solve(opts, out=ob, stream=b)
                torch.cuda.synchronize()
                for o in (oa, ob):
                    assert (o[1].cpu().numpy() == 0).all()
                    assert np.array_equal(blocks_to_numpy(o[0][0]), ref), kern
    finally:
        B.must_tune_set(2, old)


@pytest.mark.parametrize("pair_rows", [1, 200])
def test_paired_steps_match_oracle_and_single_steps(B, orc, pair_rows):
    """Paired panel steps (knob 11): two steps' trailing updates in one K = 128
    pass, with the second panel's interchanges applied to the first step's
    packed A operand and the first step's update of the second panel's rows
    done separately.  The result follows the oracle within the mixed
    tolerance and the single-step schedule within it too, on a ragged order
    (n = 387: pairs, then single steps where no full pair is left, and with
    pair_rows = 200 a switch from pairs to single steps) and on the 135-site
    LIZ (with and without look-ahead)."""
    rng = np.random.default_rng(14)
    pos, _ = wl.fcc_cluster(3)
    w = wl.Workload("ragged387", 2, [wl.Liz(pos, rng.integers(0, 2, pos.shape[0]).astype(np.int32))],
                    wl.semicircle_contour(5), wl.spin_depths(2), wl.R_MT)
    big = wl.liz135(n_e=4)
    old = (B.must_tune_get(11), B.must_tune_get(4))
    try:
        B.must_tune_set(11, 0)
        single, st = _gpu_tau(B, w, 1, residual=3)
        single_big, _ = _gpu_tau(B, big, 1, residual=3)
        B.must_tune_set(11, pair_rows)
        paired, st = _gpu_tau(B, w, 1, residual=3)
        assert (st == 0).all()
        k = w.kappa()
        ref, _ = oracle_tau(orc, w, nthreads=ncpu())
        assert rel_fro(paired.reshape(-1, k, k), ref).max() <= TOLMIX
        assert rel_fro(paired.reshape(-1, k, k), single.reshape(-1, k, k)).max() <= TOLMIX
        kb = big.kappa()
        for la in (1, 0):
            B.must_tune_set(4, la)
            pb, stb = _gpu_tau(B, big, 1, residual=3)
            assert (stb == 0).all()
            assert rel_fro(pb.reshape(-1, kb, kb), single_big.reshape(-1, kb, kb)).max() <= TOLMIX
    finally:
        B.must_tune_set(11, old[0])
        B.must_tune_set(4, old[1])


@pytest.mark.parametrize("late", [404, 808, 204])
def test_late_correction_shape(B, orc, late):
    """From the third correction on, few items are still iterating; knob 12
    gives those launches another cluster shape (more, smaller CTAs per item).
    The substitutions are the same in another summation order: the result
    follows the oracle and the default shape within the mixed tolerance, and
    the same items converge."""
    w = wl.first_shell_small()
    old = B.must_tune_get(12)
    try:
        B.must_tune_set(12, 0)
        ref_dev, st0 = _gpu_tau(B, w, 1, residual=3)
        B.must_tune_set(12, late)
        tau, st = _gpu_tau(B, w, 1, residual=3)
    finally:
        B.must_tune_set(12, old)
    assert (st == 0).all() and (st0 == 0).all()
    ref, _ = oracle_tau(orc, w)
    assert rel_fro(tau.reshape(-1, 9, 9), ref).max() <= TOLMIX
    assert rel_fro(tau.reshape(-1, 9, 9), ref_dev.reshape(-1, 9, 9)).max() <= TOLMIX


def test_paired_pass_kernels_identical(B):
    """The paired (K = 128) pass on the TMA-C kernel (knob 13 = 3) and on the
    register-C kernel with the deeper A ring (13 = 2) issue the same MMAs and
    subtract the same way: tau_00 is identical bit for bit (135-site LIZ,
    every possible step paired)."""
    w = wl.liz135(n_e=4)
    old = (B.must_tune_get(11), B.must_tune_get(13))
    try:
        B.must_tune_set(11, 1)
        taus = []
        for kern in (3, 2):
            B.must_tune_set(13, kern)
            tau, st = _gpu_tau(B, w, 1, residual=3)
            assert (st == 0).all()
            taus.append(tau)
        assert np.array_equal(taus[0], taus[1])
    finally:
        B.must_tune_set(11, old[0])
        B.must_tune_set(13, old[1])
