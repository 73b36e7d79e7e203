"""must_tau00_batch: LIZs of uneven size in shared launches (each LIZ padded
with decoupled identity sites to a common order), checked against
must_tau00_solve on each LIZ alone and against the CPU oracle."""
import numpy as np
import pytest

from helpers import ncpu, oracle_tau, rel_fro
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


def _uneven_workload(lmax=2, n_e=4, seed=3):
    """LIZs with 12..19 sites (first two fcc shells with vacancies)."""
    rng = np.random.default_rng(seed)
    pos2, shell2 = wl.fcc_cluster(2)
    lizs = []
    for keep in (19, 17, 13, 12, 19, 15):
        sel = [0] + sorted(rng.choice(np.arange(1, 19), size=keep - 1, replace=False).tolist())
        lizs.append(wl.Liz(pos2[sel], rng.integers(0, 2, keep).astype(np.int32)))
    return wl.Workload("uneven", lmax, lizs, wl.semicircle_contour(n_e), wl.spin_depths(2), wl.R_MT)


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-9)])
def test_batch_matches_single_solves_and_oracle(B, orc, precision, tol):
    import torch
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    w = _uneven_workload()
    s = Session(w)
    opts = B.must_default_opts(precision, residual=1 if precision else 0)
    tau_b, st_b = s.solve_batch(opts)
    torch.cuda.synchronize()
    assert (st_b.cpu().numpy() == 0).all()
    tb = blocks_to_numpy(tau_b)
    for j in range(len(w.lizs)):
        t1, st1 = s.solve(opts, liz_index=j)
        torch.cuda.synchronize()
        assert (st1.cpu().numpy() == 0).all()
        one = blocks_to_numpy(t1)
        assert rel_fro(tb[j], one).max() <= tol
        ref, _ = oracle_tau(orc, w, liz_index=j)
        assert rel_fro(tb[j].reshape(-1, 9, 9), ref).max() <= tol


def test_batch_small_workspace_chunks_per_liz(B):
    """A workspace that fits one energy of one LIZ still gives the same result."""
    import torch
    from paper_2308_16317_gb300.runner import Session
    w = _uneven_workload()
    s = Session(w)
    ref, _ = s.solve_batch(None)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    small = B.must_workspace_bytes(s.lizs[0], 2) * 2 + (1 << 20)
    tau, st = s.solve_batch(None, ws_bytes=small)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    assert np.abs(tau.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_batched_supercell_sample(B, orc):
    """Per-site LIZs of the 256-site supercell with vacancies (n 688..2160,
    lmax 3): 8 LIZs x 4 energies x 2 spins in one mixed-precision batch call;
    the smallest and largest LIZ are checked against the oracle."""
    import torch
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    full = wl.batched_supercell(n_sites=8)
    w = wl.Workload(full.name, full.lmax, full.lizs, wl.semicircle_contour(4, im_min=0.005), full.v_species,
                    full.r_mt)
    s = Session(w)
    tau, st = s.solve_batch(B.must_default_opts(1, residual=1))
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    tb = blocks_to_numpy(tau)
    sizes = [l.n_sites for l in w.lizs]
    for j in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        items = [(0, 0), (1, 3)]
        ref, _ = oracle_tau(orc, w, liz_index=j, items=items, nthreads=min(2, ncpu()))
        got = np.array([tb[j, s_, e] for s_, e in items])
        assert rel_fro(got, ref).max() <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_plan_replay_matches_batch_call(B, precision):
    """A captured plan, replayed twice (with new t^{-1} contents in the same
    buffer in between), matches must_tau00_batch on the same inputs."""
    import torch
    from paper_2308_16317_gb300.runner import Session
    w = _uneven_workload()
    s = Session(w)
    opts = B.must_default_opts(precision, residual=1 if precision else 0)
    ref, _ = s.solve_batch(opts)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    items = len(w.energies) * s.nspin
    nb = B.must_batch_workspace_bytes(s.lizs, items, opts)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    tau, st = s.alloc_out(len(s.lizs))
    plan = B.must_plan_batch(s.lizs, s.E, s.tinv, s.n_species, s.nspin, opts, ws, nb, tau, st)
    l0 = B.must_launch_count()
    B.must_plan_launch(plan)
    torch.cuda.synchronize()
    assert B.must_launch_count() > l0
    assert (st.cpu().numpy() == 0).all()
    assert np.abs(tau.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    # new t^{-1} (deeper wells) in the same buffer: the replay follows it
    saved = s.tinv.clone()
    V = torch.tensor((np.asarray(w.v_species) - 0.1).reshape(-1), device="cuda")
    B.must_tinv_square_well(s.E, V, w.r_mt, w.lmax, s.tinv)
    ref2, _ = s.solve_batch(opts)
    B.must_plan_launch(plan)
    torch.cuda.synchronize()
    assert np.abs(tau.cpu().numpy() - ref2.cpu().numpy()).max() <= 1e-12 * np.abs(ref2.cpu().numpy()).max()
    assert np.abs(ref2.cpu().numpy() - ref).max() > 1e-3 * np.abs(ref).max()
    s.tinv.copy_(saved)


def test_tuning_knobs_change_nothing_numerically(B):
    import torch
    from paper_2308_16317_gb300.runner import Session
    w = _uneven_workload()
    s = Session(w)
    opts = B.must_default_opts(1, residual=1)
    ref, _ = s.solve_batch(opts)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    old = (B.must_tune_get(0), B.must_tune_get(1))
    try:
        for bucket, tile in ((1, 256), (8, 128)):
            B.must_tune_set(0, bucket)
            B.must_tune_set(1, tile)
            tau, st = s.solve_batch(opts)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all()
            assert rel_fro(tau.cpu().numpy(), ref).max() <= 1e-9
        with pytest.raises(B.MustError):
            B.must_tune_set(1, 96)
    finally:
        B.must_tune_set(0, old[0])
        B.must_tune_set(1, old[1])


def test_autotuner_on_uneven_batch(B, tmp_path):
    """The tuner measures every knob combination on the device, caches the
    fastest, and the tuned setting still solves correctly."""
    import os
    import torch
    from paper_2308_16317_gb300 import autotune
    from paper_2308_16317_gb300.runner import Session
    w = _uneven_workload()
    s = Session(w)
    opts = B.must_default_opts(1, residual=1)
    ref, _ = s.solve_batch(opts)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    knobs = (0, 1, 3, 7)
    old = {k: B.must_tune_get(k) for k in knobs}
    try:
        path = os.path.join(tmp_path, "tune.json")
        best, results = autotune.tune_session(s, opts, cache_path=path, reps=1)
        assert len(results) == 4 * 2 * 3 * 2 and all(ms > 0 for _, ms in results)
        for name, k in autotune.KNOBS.items():
            assert B.must_tune_get(k) == best[name]
        again, none = autotune.tune_session(s, opts, cache_path=path)
        assert again == best and none is None
        tau, st = s.solve_batch(opts)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        assert rel_fro(tau.cpu().numpy(), ref).max() <= 1e-9
    finally:
        for k, v in old.items():
            B.must_tune_set(k, v)



def test_plans_in_flight_on_two_streams(B):
    """Two plans of the same batch (own workspace, inputs and outputs each)
    replayed at the same time on two streams, several times each, give the
    result of a plain batch call (to the tolerance the single-plan replay test
    uses: the norms of the refinement are summed with atomics): nothing is
    shared between plans in flight."""
    import torch
    from paper_2308_16317_gb300.runner import Session
    w = _uneven_workload()
    s = Session(w)
    opts = B.must_default_opts(1, residual=3)
    ref, st = s.solve_batch(opts)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    ref = ref.cpu().numpy()
    items = len(w.energies) * s.nspin
    nb = B.must_batch_workspace_bytes(s.lizs, items, opts)
    plans, outs, keep = [], [], []
    for _ in range(2):
        E, T = s.E.clone(), s.tinv.clone()
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        tau, sta = s.alloc_out(len(s.lizs))
        plans.append(B.must_plan_batch(s.lizs, E, T, s.n_species, s.nspin, opts, ws, nb, tau, sta))
        outs.append((tau, sta))
        keep.append((E, T, ws))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for _ in range(3):
        for p, x in zip(plans, streams):
            B.must_plan_launch(p, stream=x)
    torch.cuda.synchronize()
    for tau, sta in outs:
        assert (sta.cpu().numpy() == 0).all()
        assert np.abs(tau.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
