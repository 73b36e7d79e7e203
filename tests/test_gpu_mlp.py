"""The warm-start MLP's hand-written GPU kernels (products on the tcgen05
tensor cores in 3xTF32) against the CPU reference (oracle/mlp.py): gradients
on the same BF16-rounded weights within 1e-3 relative per tensor, training reduces the loss, checkpoints round-trip, and
the feature / target / apply kernels invert each other."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _split(p, I, H, O):
    sizes = [("W1", (H, I)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,))]
    out, o = {}, 0
    for name, shp in sizes:
        k = int(np.prod(shp))
        out[name] = p[o:o + k].reshape(shp)
        o += k
    return out


@pytest.mark.parametrize("I,H,O,Bn", [(37, 24, 10, 16), (1302, 256, 512, 200)])
def test_gradients_match_cpu_reference(B, I, H, O, Bn):
    """Small widths (every product a single padded tile) and the warm start's
    own widths (1302 -> 256 -> 256 -> 512, a ragged batch of 200: several
    row, column and K tiles of the tensor-core products)."""
    import torch
    from oracle import mlp
    net = B.Mlp(I, H, O, max(64, Bn), seed=3)
    rng = np.random.default_rng(0)
    p = (rng.standard_normal(net.param_count()) * 0.3 / np.sqrt(I / 37.0)).astype(np.float32)
    B.must_mlp_set_params(net, torch.tensor(p, device="cuda"))
    x = rng.standard_normal((Bn, I)).astype(np.float32)
    t = rng.standard_normal((Bn, O)).astype(np.float32)
    g = torch.zeros(net.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.must_mlp_gradients(net, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), g, loss)
    torch.cuda.synchronize()
    P = _split(p.astype(np.float64), I, H, O)
    for w in ("W1", "W2", "W3"):
        P[w] = mlp.bf16_round(P[w].astype(np.float32))
    y, cache = mlp.forward(P, x.astype(np.float64))
    L, dy = mlp.mse_loss(y, t.astype(np.float64))
    ref = mlp.backward(P, cache, dy)
    got = _split(g.cpu().numpy().astype(np.float64), I, H, O)
    assert abs(loss.item() - L) <= 1e-4 * L
    for name in ref:
        err = np.linalg.norm(got[name] - ref[name]) / np.linalg.norm(ref[name])
        assert err <= 1e-3, (name, err)
    y_gpu = torch.zeros((Bn, O), dtype=torch.float32, device="cuda")
    B.must_mlp_forward(net, torch.tensor(x, device="cuda"), y_gpu)
    torch.cuda.synchronize()
    assert np.linalg.norm(y_gpu.cpu().numpy() - y) <= 1e-4 * np.linalg.norm(y)


def test_training_reduces_loss_and_checkpoint_roundtrips(B, tmp_path):
    import torch
    I, H, O, Bn = 20, 32, 8, 64
    net = B.Mlp(I, H, O, Bn, seed=1)
    rng = np.random.default_rng(1)
    W = rng.standard_normal((I, O)).astype(np.float32) * 0.5
    x = torch.tensor(rng.standard_normal((Bn, I)).astype(np.float32), device="cuda")
    t = torch.tensor(np.tanh(x.cpu().numpy() @ W), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    B.must_mlp_train_step(net, x, t, 0.0, loss)
    torch.cuda.synchronize()
    first = loss.item()
    for _ in range(400):
        B.must_mlp_train_step(net, x, t, 3e-3, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.05 * first
    path = str(tmp_path / "net.bin")
    B.must_mlp_save(net, path)
    other = B.Mlp(I, H, O, Bn, seed=99)
    B.must_mlp_load(other, path)
    ya = torch.zeros((Bn, O), dtype=torch.float32, device="cuda")
    yb = torch.zeros_like(ya)
    B.must_mlp_forward(net, x, ya)
    B.must_mlp_forward(other, x, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    with pytest.raises(B.MustError):
        B.must_mlp_load(B.Mlp(I + 1, H, O, Bn), path)


def test_feature_target_apply_roundtrip(B):
    import torch
    rng = np.random.default_rng(2)
    n, kap, n_occ = 5, 16, 270
    c = lambda *s: torch.tensor(rng.standard_normal(s) + 1j * rng.standard_normal(s), device="cuda")
    tm, tp, tk = c(n, kap, kap), c(n, kap, kap), c(n, kap, kap)
    E3 = c(n, 3)
    spin = torch.tensor([1.0, -1.0, 1.0, -1.0, 1.0], dtype=torch.float32, device="cuda")
    occ = torch.tensor((rng.random((n, n_occ)) < 0.5).astype(np.float32), device="cuda")
    n_in = 4 * kap * kap + n_occ + 8
    x = torch.zeros((n, n_in), dtype=torch.float32, device="cuda")
    scale = torch.zeros(n, dtype=torch.float32, device="cuda")
    interp = torch.zeros((n, kap, kap), dtype=torch.complex128, device="cuda")
    B.must_mlp_features(kap, tm, tp, E3, spin, occ, n_in, x, scale, interp)
    y = torch.zeros((n, 2 * kap * kap), dtype=torch.float32, device="cuda")
    B.must_mlp_targets(kap, tk, scale, interp, y)
    pred = torch.zeros_like(tk)
    B.must_mlp_apply(kap, y, scale, interp, pred)
    torch.cuda.synchronize()
    assert torch.allclose(interp, 0.5 * (tm + tp))
    assert (torch.abs(pred - tk).max() / torch.abs(tk).max()).item() < 1e-6
    xs = x.cpu().numpy()
    assert np.array_equal(xs[:, 4 * kap * kap:4 * kap * kap + n_occ], occ.cpu().numpy())
    assert np.allclose(xs[:, -2], spin.cpu().numpy())


def test_trained_network_beats_linear_interpolation(B):
    """Train on tau_00 generated by the method for seeded random 135-site LIZs
    and compare, on held-out LIZs, the network's prediction of the odd contour
    points with the linear interpolation of their neighbours (the method's
    own cheapest guess).  The gain is reported as the ratio of median errors."""
    import torch
    from paper_2308_16317_gb300 import warmstart as ws
    opts = B.must_default_opts(1, residual=1)
    train_w = ws.random_liz_workload(100000, 24)
    test_w = ws.random_liz_workload(200000, 6)
    tau_tr = ws.solve_all(train_w, opts)
    tau_te = ws.solve_all(test_w, opts)
    model = ws.WarmStart(max_batch=512)
    tp, tn, tt, E3, sp, oc = ws.samples_from_solution(tau_tr, train_w)
    x, scale, interp = model.features(tp, tn, E3, sp, oc)
    y = model.targets(tt, scale, interp)
    hist = model.train(x, y, epochs=40, batch=128, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0]
    tp2, tn2, tt2, E32, sp2, oc2 = ws.samples_from_solution(tau_te, test_w)
    pred, interp2 = model.predict(tp2, tn2, E32, sp2, oc2)
    e_mlp = ws.rel_err(pred, tt2).median().item()
    e_lin = ws.rel_err(interp2, tt2).median().item()
    print("held-out median relative error: network %.3e, linear interpolation %.3e (gain %.2fx)"
          % (e_mlp, e_lin, e_lin / e_mlp))
    assert e_mlp < e_lin


def _seeded(B, s, opts, seed, mask):
    import torch
    items = len(s.w.energies) * s.nspin
    nb = B.must_workspace_bytes(s.lizs[0], items, opts)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    tau, st = s.alloc_out(1)
    used = torch.full_like(st[0], -1)
    B.must_tau00_solve_seeded(s.lizs[0], s.E, s.tinv, s.n_species, s.nspin, opts, ws, nb, seed, mask, tau[0], st[0],
                              used)
    torch.cuda.synchronize()
    return tau[0], st[0], used


def test_seeded_solve_accepts_good_seeds_and_falls_back_on_bad(B, orc):
    """Weak wells (V ~ -0.02 Ry), where single scattering is accurate: the exact
    tau_00 as seed passes the residual gate and the refined result still
    matches the oracle; NaN seeds are rejected and the plain solve takes over."""
    import torch
    from helpers import oracle_tau, rel_fro
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    pos, _ = wl.fcc_cluster(1)
    liz = wl.Liz(pos, (np.arange(13) % 2).astype(np.int32))
    w = wl.Workload("weak", 2, [liz], wl.semicircle_contour(6), np.array([[-0.02, -0.03], [-0.01, -0.025]]), wl.R_MT)
    s = Session(w)
    opts = B.must_default_opts(1, residual=1)
    plain, st0 = s.solve(opts)
    torch.cuda.synchronize()
    assert (st0.cpu().numpy() == 0).all()
    mask = torch.ones_like(st0)
    tau, st, used = _seeded(B, s, opts, plain.clone(), mask)
    assert (st.cpu().numpy() == 0).all() and (used.cpu().numpy() == 1).all()
    ref, _ = oracle_tau(orc, w)
    assert rel_fro(blocks_to_numpy(tau).reshape(-1, 9, 9), ref).max() <= 1e-9
    bad = torch.full_like(plain, float("nan"))
    tau2, st2, used2 = _seeded(B, s, opts, bad, mask)
    assert (used2.cpu().numpy() == 0).all() and (st2.cpu().numpy() == 0).all()
    assert rel_fro(blocks_to_numpy(tau2).reshape(-1, 9, 9), ref).max() <= 1e-9
    none = torch.zeros_like(st0)
    tau3, _, used3 = _seeded(B, s, opts, bad, none)
    assert (used3.cpu().numpy() == 0).all()
    assert rel_fro(blocks_to_numpy(tau3), blocks_to_numpy(plain)).max() <= 1e-12
