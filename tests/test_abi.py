"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/must.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "must.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(must_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_16317_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_three_path_calls():
    names = declared_functions()
    for n in ("must_liz_build", "must_tau00_solve", "must_tau00_batch"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2308_16317_gb300 import binding
    assert set(declared_functions()) <= set(binding.exported_symbols())
    lib = binding.load()
    s = lib.must_status_string(4)
    assert s == b"MUST_ESINGULAR"


def test_host_side_argument_errors_need_no_gpu(lib):
    """Arguments are validated on the host before any device call."""
    from paper_2308_16317_gb300 import binding as B
    B.load()
    out = ctypes.c_void_p()
    assert B.load().must_liz_build(None, None, 3, 3, None, None, ctypes.byref(out)) == 1
    assert b"NULL" in B.load().must_last_error()
    import numpy as np
    pos = np.zeros((2, 3))
    sp = np.zeros(2, np.int32)
    r = B.load().must_liz_build(pos.ctypes.data_as(ctypes.c_void_p), sp.ctypes.data_as(ctypes.c_void_p), 2, 7,
                                None, None, ctypes.byref(out))
    assert r == 1 and b"lmax" in B.load().must_last_error()
    assert B.load().must_tau00_solve(None, 1, None, None, 1, 1, None, None, 0, None, None, None) == 1


def test_bench_traffic_profile_matches_current_kernel_source():
    """profiles/tc_update_kernel_fcc135.txt carries the sha256 of the code
    (comments stripped) of the kernel source it was captured from and the
    ratio of DRAM bytes to algorithmic bytes over a captured step; bench.py
    reports roofline.traffic (that ratio times the algorithmic bytes per
    launch) only while the sha matches (a stale capture reads as null)."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    t = bench.traffic_from_profiles("tc_update_kernel_fcc135", "paper_2308_16317_gb300/csrc/tc_gemm.cu", 7e8)
    assert t is not None and 0.95 * 7e8 < t < 1.1 * 7e8
    assert bench.traffic_from_profiles("tc_update_kernel_fcc135", "paper_2308_16317_gb300/csrc/mixed.cu", 7e8) is None


def test_contour_weights_are_computed_on_the_host():
    """must_contour_weights needs no GPU: the library's Gauss-Legendre nodes
    (its own Newton iteration) agree with numpy's, and the weights integrate
    polynomials along the semicircle."""
    import numpy as np
    from paper_2308_16317_gb300 import binding as B
    for n in (1, 5, 32):
        E, w = B.must_contour_weights(n)
        x, W = np.polynomial.legendre.leggauss(n)
        th = 0.5 * np.pi * (1.0 - x)
        assert np.abs(E - (0.2 + 0.5 * np.exp(1j * th))).max() <= 1e-14
    E, w = B.must_contour_weights(24)
    for m in range(4):
        assert abs(np.sum(w * E ** m) - (0.7 ** (m + 1) - (-0.3) ** (m + 1)) / (m + 1)) <= 1e-13
    with pytest.raises(B.MustError):
        B.must_contour_weights(8, 0.7, -0.3)


def test_site_charge_rejects_host_arrays():
    import numpy as np
    from paper_2308_16317_gb300 import binding as B
    E, w = B.must_contour_weights(4)
    tau = np.zeros((1, 4, 16, 16), np.complex128)
    V = np.array([-1.0])
    N = np.zeros(1)
    with pytest.raises(B.MustError):
        B.must_site_charge(3, E, w, V, 2.5, tau, None, N)


def test_code_digest_ignores_comments_only(tmp_path):
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text("// header\nint f(int x) {\n  return x + 1;  // add\n}\n")
    b.write_text("/* another\n   header */\n\nint f(int x) {\n  return x + 1;\n}\n")
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.code_sha256(str(a)) == bench.code_sha256(str(b))
    assert bench.code_sha256(str(a)) != bench.code_sha256(str(c))


def test_site_density_rejects_host_arrays():
    import numpy as np
    from paper_2308_16317_gb300 import binding as B
    E, w = B.must_contour_weights(4)
    tau = np.zeros((1, 4, 16, 16), np.complex128)
    V = np.array([-1.0])
    r = np.array([0.5, 1.0])
    out = np.zeros((1, 2))
    with pytest.raises(B.MustError):
        B.must_site_density(3, E, w, V, 2.5, tau, r, out)


def test_bench_algorithmic_work_of_the_update():
    """The roofline numerators of bench.py: the mixed path's trailing update
    moves 16 B per trailing-block element per panel step (7.905e8 B per launch
    of the 64-item n = 2160 workload, 65 launches per step); the FP64 path's
    update does 8 flops per complex MAC, which for r = n - kap eliminated
    columns approaches the unblocked 8/3 (n^3 - kap^3) minus the panels' share."""
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    n, kap, nb, items = 2160, 16, 64, 64
    byts = bench.phase_work("trailing_update", n, kap, nb, items, "bf16x3")[0]
    steps = [(k0, min(nb, n - kap - k0)) for k0 in range(0, n - kap, nb)]
    assert len(steps) == 34
    ref = sum(16 * (n - k0 - w) ** 2 for k0, w in steps) * items
    assert byts == ref
    assert abs(byts / 65 - 7.905e8) < 0.001e8
    # paired steps: step k's update of panel k+1's 64 columns and 64 rows, then
    # one pass for both; pairing every step roughly halves the C traffic
    b1 = bench.update_bytes(n, n - kap, nb, 1)
    k0, ref1 = 0, 0
    while k0 < n - kap:
        if k0 + 2 * nb <= n - kap and n - (k0 + 2 * nb) >= 1:
            m1, m2 = n - k0 - nb, n - k0 - 2 * nb
            ref1 += 16 * (m1 * nb + nb * m2 + m2 * m2)
            k0 += 2 * nb
        else:
            ref1 += 16 * (n - k0 - min(nb, n - kap - k0)) ** 2
            k0 += nb
    assert b1 == ref1 and 0.5 < b1 / (byts / items) < 0.6
    assert bench.update_bytes(n, n - kap, nb, 10 ** 6) * items == byts
    flops = bench.phase_work("trailing_update", n, kap, nb, 1, "fp64")[0]
    unblocked = 8.0 * sum((n - j - 1) ** 2 for j in range(n - kap))
    # the blocked update leaves out the work inside each panel (about nb/2 columns of width m)
    assert 0.9 * unblocked < flops < unblocked


def test_tuning_knobs_validate_and_round_trip():
    """Tuning knobs are process-wide host settings: valid values round-trip,
    invalid ones are rejected with MUST_EINVAL and leave the setting as it was
    (no GPU needed)."""
    from paper_2308_16317_gb300 import binding as B
    cases = {6: ([0, 1], [2, -1]), 7: ([2, 4, 8], [3, 16]), 8: ([0, 4, 8, 16], [2, 32]), 5: ([0, 2, 4, 8], [3]),
             9: ([0, 1], [2]), 10: ([0, 1, 2], [3, -1]), 11: ([0, 1, 1024], [-1]), 12: ([0, 204, 404, 816], [1, 304, 405]), 13: ([2, 3], [0, 1, 4])}
    for knob, (good, bad) in cases.items():
        old = B.must_tune_get(knob)
        try:
            for v in good:
                B.must_tune_set(knob, v)
                assert B.must_tune_get(knob) == v
            for v in bad:
                with pytest.raises(B.MustError) as ei:
                    B.must_tune_set(knob, v)
                assert ei.value.code == 1
                assert B.must_tune_get(knob) == good[-1]
        finally:
            B.must_tune_set(knob, old)
    with pytest.raises(B.MustError):
        B.must_tune_set(99, 1)


def test_kkr_build_rejects_bad_arguments_on_the_host():
    """must_kkr_build validates its arguments before any CUDA call."""
    import numpy as np
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import workload as wl
    c = wl.l12_crystal()
    bad = [
        (c.lattice, np.vstack([c.basis, c.basis[:1] + c.lattice[0]]), 1, 4),   # sites coincide modulo the lattice
        (c.lattice, c.basis, 4, 4),                                            # 4 x 25 > 64
        (np.zeros((3, 3)), c.basis, 1, 4),                                     # degenerate lattice
        (c.lattice, c.basis, 3, 0),                                            # n_k < 1
        (c.lattice, c.basis, 5, 4),                                            # lmax > 4
    ]
    for lat, bas, lmax, nk in bad:
        with pytest.raises(B.MustError) as ei:
            B.must_kkr_build(lat, bas, lmax, nk)
        assert ei.value.code == 1
    with pytest.raises(B.MustError):
        B.must_kkr_build(c.lattice, c.basis, 3, 4, eta=-1.0)


def test_bench_kkr_work_counts():
    """bench.kkr_work: 4 flops per real-by-complex multiply-add of the lattice
    sums (a pair group's stored point counting for both displacements) and 8 n^3
    per inverted k point; checked against a direct count for a fake handle."""
    import types
    import bench
    from paper_2308_16317_gb300 import workload as wl
    c = wl.l12_crystal(lmax=2)
    h = types.SimpleNamespace(n_kK=1000, n_disp=13, n_kpts=35, n_pts=3000, n_pts0=200, n=36)
    w = bench.kkr_work(h, c, 64)
    nL2 = 25
    assert w["kkr_recip"] == 4.0 * 64 * 1000 * 13 * nL2
    # 200 points of x = 0 (one displacement each), 2800 of the six pair groups (two each)
    assert w["kkr_realsum"] == 4.0 * 64 * 35 * nL2 * (200 + 2 * 2800)
    assert w["kkr_invert"] == 8.0 * 64 * 35 * 36 ** 3


def test_binding_constants_match_the_header():
    """The Python binding's copies of the header's enumerators and #define
    flags (precisions, status codes, full-KKR flags) carry the same values,
    and the library names each status code as the header does."""
    from paper_2308_16317_gb300 import binding as B
    text = open(os.path.join(ROOT, "include", "must.h")).read()
    text_nc = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    enums = {}
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", text_nc, flags=re.S):
        nxt = 0
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            if "=" in item:
                name, val = (x.strip() for x in item.split("="))
                nxt = int(val)
            else:
                name = item
            enums[name] = nxt
            nxt += 1
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(MUST_\w+)\s+(\d+)", text)}
    for name in ("MUST_FP64", "MUST_MIXED_BF16X3", "MUST_MIXED_TF32X3"):
        assert getattr(B, name) == enums[name], name
    for code, name in B.STATUS.items():
        assert enums[name] == code, name
        assert B.load().must_status_string(code).decode() == name
    for name in ("MUST_KKR_NO_SYMMETRY", "MUST_KKR_NO_TABLE"):
        assert getattr(B, name) == defines[name], name
