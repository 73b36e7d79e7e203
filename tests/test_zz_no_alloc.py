"""The allocation-free entry point (must_tau00_solve_static) against the
workspace entry point (must_tau00_solve), through the C ABI.

must_tau00_solve_static serves callers that cannot allocate device memory
while they run; it solves in a scratch array compiled into the library.  The
check: two calls in a row (the second finds the first call's data still in
the shared scratch) give the same tau_00 as the ordinary FP64 solve, within
the FP64 tolerance of the parity tests; an LIZ too large for the scratch is
rejected with a clear error; the second call leaves the device's free memory
unchanged (it allocates nothing).  Collected last so that a failure here does not
hide the other GPU tests.
"""
import numpy as np
import pytest

from paper_2308_16317_gb300 import workload as wl

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module")
def B():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a GPU"
    from paper_2308_16317_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _rel(a, b):
    return (np.linalg.norm(a - b, axis=(-2, -1)) / np.linalg.norm(b, axis=(-2, -1))).max()


@pytest.mark.parametrize("make", [lambda: wl.first_shell_small(),
                                  lambda: wl.Workload("ragged304", 3, [wl.Liz(wl.fcc_cluster(2)[0],
                                                      np.random.default_rng(1).integers(0, 2, 19).astype(np.int32))],
                                                      wl.semicircle_contour(5), wl.spin_depths(2), wl.R_MT)])
def test_static_scratch_solve_matches_workspace_solve(B, make):
    import torch
    from paper_2308_16317_gb300.runner import Session
    w = make()
    s = Session(w)
    ref, st_ref = s.solve(B.must_default_opts(B.MUST_FP64))
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert (st_ref.cpu().numpy() == 0).all()
    outs = [(torch.full((s.n_out, len(w.energies), s.kap, s.kap), float("nan"), dtype=torch.complex128,
                        device="cuda"),
             torch.full((s.n_out, len(w.energies)), -1, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    for call, (tau, st) in enumerate(outs):      # two calls in a row share the scratch
        # the first call on the device looks up the scratch address and loads
        # the kernels; the second must leave the device's free memory unchanged
        free0 = torch.cuda.mem_get_info()[0]
        B.must_tau00_solve_static(s.lizs[0], s.E, s.tinv, s.n_species, s.nspin, tau, st)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:
            assert free1 == free0, "the allocation-free solve changed free device memory by %d bytes" % (free0 - free1)
        assert (st.cpu().numpy() == 0).all()
        assert _rel(tau.cpu().numpy(), ref) <= TOL64


def test_static_scratch_rejects_oversized_and_host_buffers(B):
    import torch
    # 249-site LIZ at lmax = 4: n = 6225, one energy of two spins needs ~1.2 GB
    pos, _ = wl.fcc_cluster(12)
    liz = B.must_liz_build(pos, np.zeros(pos.shape[0], np.int32), 4)
    E = torch.zeros(1, dtype=torch.complex128, device="cuda")
    tinv = torch.ones((2, 1, 1, 5), dtype=torch.complex128, device="cuda")
    tau = torch.empty((2, 1, 25, 25), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.MustError) as ei:
        B.must_tau00_solve_static(liz, E, tinv, 1, 2, tau)
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
    small = B.must_liz_build(np.zeros((1, 3)), np.zeros(1, np.int32), 2)
    with pytest.raises(B.MustError) as ei:
        B.must_tau00_solve_static(small, np.zeros(1, np.complex128), np.ones((1, 1, 1, 3), np.complex128), 1, 1,
                                  np.zeros((1, 1, 9, 9), np.complex128))
    assert ei.value.code == 1
    assert B.must_static_scratch_bytes() == 160 << 20
