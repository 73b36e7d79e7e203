"""ctypes binding of the C ABI in include/must.h (argument marshalling only).

Every function has the name of its C entry point.  Array arguments may be
torch tensors (host or CUDA; their data pointer is passed) or numpy arrays
(host).  All computation happens in the CUDA library; if it has not been
built, ``load()`` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmust.so")
_lib = None

MUST_FP64, MUST_MIXED_BF16X3, MUST_MIXED_TF32X3 = 0, 1, 2
STATUS = {0: "MUST_OK", 1: "MUST_EINVAL", 2: "MUST_ENOMEM", 3: "MUST_ECUDA", 4: "MUST_ESINGULAR",
          5: "MUST_ENOCONV", 6: "MUST_ENONFINITE", 7: "MUST_ETIMEOUT", 8: "MUST_EUNSUPPORTED"}


class MustError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class must_solve_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("deterministic", ctypes.c_int32), ("equilibrate", ctypes.c_int32),
                ("residual", ctypes.c_int32)]


def load():
    """Load the built library (``paper_2308_16317_gb300/build.py``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmust.so is not built (run paper_2308_16317_gb300/build.py); "
                          "there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    sig = {
        "must_default_opts": (None, [ctypes.POINTER(must_solve_opts)]),
        "must_liz_build": (I32, [P, P, I32, I32, P, P, ctypes.POINTER(P)]),
        "must_liz_free": (None, [P]),
        "must_liz_order": (I32, [P]),
        "must_liz_kappa": (I32, [P]),
        "must_workspace_bytes": (SZ, [P, I32, ctypes.POINTER(must_solve_opts)]),
        "must_batch_workspace_bytes": (SZ, [I32, P, I32, ctypes.POINTER(must_solve_opts)]),
        "must_tinv_square_well": (I32, [I32, P, I32, P, D, I32, P, P]),
        "must_tau00_solve": (I32, [P, I32, P, P, I32, I32, ctypes.POINTER(must_solve_opts), P, SZ, P, P, P]),
        "must_tau00_batch": (I32, [I32, P, I32, P, P, I32, I32, ctypes.POINTER(must_solve_opts), P, SZ, P, P, P]),
        "must_tau00_solve_static": (I32, [P, I32, P, P, I32, I32, P, P, P]),
        "must_plan_batch": (I32, [I32, P, I32, P, P, I32, I32, ctypes.POINTER(must_solve_opts), P, SZ, P, P,
                                  ctypes.POINTER(P)]),
        "must_plan_launch": (I32, [P, P]),
        "must_plan_free": (None, [P]),
        "must_tune_set": (I32, [I32, I32]),
        "must_tau00_solve_seeded": (I32, [P, I32, P, P, I32, I32, ctypes.POINTER(must_solve_opts), P, SZ, P, P, P,
                                          P, P, P]),
        "must_mlp_create": (I32, [I32, I32, I32, I32, ctypes.c_uint64, ctypes.POINTER(P)]),
        "must_mlp_free": (None, [P]),
        "must_mlp_param_count": (SZ, [P]),
        "must_mlp_get_params": (I32, [P, P, P]),
        "must_mlp_set_params": (I32, [P, P, P]),
        "must_mlp_forward": (I32, [P, I32, P, P, P]),
        "must_mlp_gradients": (I32, [P, I32, P, P, P, P, P]),
        "must_mlp_train_step": (I32, [P, I32, P, P, ctypes.c_float, P, P]),
        "must_mlp_save": (I32, [P, ctypes.c_char_p]),
        "must_mlp_load": (I32, [P, ctypes.c_char_p]),
        "must_mlp_features": (I32, [I32, I32, P, P, P, P, P, I32, I32, P, P, P, P]),
        "must_mlp_apply": (I32, [I32, I32, P, I32, P, P, P, P]),
        "must_mlp_targets": (I32, [I32, I32, P, P, P, P, I32, P]),
        "must_tune_get": (I32, [I32]),
        "must_contour_weights": (I32, [I32, D, D, P, P]),
        "must_site_charge": (I32, [I32, I32, P, P, I32, P, D, P, P, P, P]),
        "must_site_density": (I32, [I32, I32, P, P, I32, P, D, P, I32, P, P, P]),
        "must_static_scratch_bytes": (SZ, []),
        "must_kkr_build": (I32, [P, P, P, I32, I32, I32, D, I32, P, ctypes.POINTER(P)]),
        "must_kkr_free": (None, [P]),
        "must_kkr_workspace_bytes": (SZ, [P, I32]),
        "must_kkr_tau": (I32, [P, I32, P, P, P, SZ, P, P, P]),
        "must_kkr_info": (I32, [P, P]),
        "must_kkr_eta": (D, [P]),
        "must_kkr_geometry": (I32, [P, P, P, I32, I32, I32, D, I32, P, P]),
        "must_kkr_table_bytes": (SZ, [P]),
        "must_profile_enable": (None, [ctypes.c_int]),
        "must_profile_read": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "must_launch_count": (ctypes.c_longlong, []),
        "must_peak_probe": (I32, [I32, I32, ctypes.c_int64, P, ctypes.POINTER(D), P]),
        "must_phase_name": (ctypes.c_char_p, [ctypes.c_int]),
        "must_status_string": (ctypes.c_char_p, [I32]),
        "must_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [n for n in ("must_default_opts", "must_liz_build", "must_liz_free", "must_liz_order", "must_liz_kappa",
                        "must_workspace_bytes", "must_batch_workspace_bytes", "must_tinv_square_well",
                        "must_tau00_solve", "must_tau00_batch", "must_status_string", "must_last_error",
                        "must_profile_enable", "must_profile_read", "must_launch_count", "must_phase_name",
                        "must_tau00_solve_static", "must_static_scratch_bytes", "must_plan_batch",
                        "must_plan_launch", "must_plan_free", "must_tune_set", "must_tune_get",
                        "must_mlp_create", "must_mlp_free", "must_mlp_param_count", "must_mlp_get_params",
                        "must_mlp_set_params", "must_mlp_forward", "must_mlp_gradients", "must_mlp_train_step",
                        "must_mlp_save", "must_mlp_load", "must_mlp_features", "must_mlp_apply", "must_mlp_targets",
                        "must_tau00_solve_seeded", "must_contour_weights", "must_site_charge", "must_site_density",
                        "must_peak_probe", "must_kkr_build", "must_kkr_free", "must_kkr_workspace_bytes",
                        "must_kkr_tau", "must_kkr_info", "must_kkr_eta", "must_kkr_geometry", "must_kkr_table_bytes")]


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(code: int):
    if code != 0:
        raise MustError(code, load().must_last_error().decode(errors="replace"))


def must_profile_enable(on: bool):
    load().must_profile_enable(1 if on else 0)


def must_profile_read():
    """{phase name: (milliseconds, launches, items)} since the last read."""
    n = 16
    ms = (ctypes.c_double * n)()
    la = (ctypes.c_longlong * n)()
    it = (ctypes.c_longlong * n)()
    k = load().must_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(la, ctypes.c_void_p),
                                 ctypes.cast(it, ctypes.c_void_p), n)
    return {load().must_phase_name(p).decode(): (ms[p], la[p], it[p]) for p in range(k)}


def must_launch_count() -> int:
    return int(load().must_launch_count())


def must_peak_probe(kind: int, blocks: int, iters: int, sink, stream=None) -> float:
    """Launch one arithmetic peak probe (0 DFMA, 1 DMMA, 2 FFMA); returns its flop count."""
    fl = ctypes.c_double(0.0)
    _check(load().must_peak_probe(kind, blocks, iters, _ptr(sink), ctypes.byref(fl), _stream(stream)))
    return fl.value


def must_default_opts(precision: int = MUST_FP64, **kw) -> must_solve_opts:
    o = must_solve_opts()
    load().must_default_opts(ctypes.byref(o))
    o.precision = precision
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Liz:
    """Owning wrapper of a must_liz handle."""

    def __init__(self, handle, n_sites, lmax, canted):
        self.handle = handle
        self.n_sites, self.lmax, self.canted = n_sites, lmax, canted
        self.n = load().must_liz_order(handle)
        self.kappa = load().must_liz_kappa(handle)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.must_liz_free(self.handle)
            self.handle = None


def must_liz_build(pos, species, lmax: int, spin_dirs=None, stream=None) -> Liz:
    pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    species = np.ascontiguousarray(np.asarray(species, dtype=np.int32))
    dirs = None if spin_dirs is None else np.ascontiguousarray(np.asarray(spin_dirs, dtype=np.float64))
    out = ctypes.c_void_p()
    _check(load().must_liz_build(_ptr(pos), _ptr(species), int(pos.shape[0]), int(lmax), _ptr(dirs),
                                 _stream(stream), ctypes.byref(out)))
    return Liz(out, int(pos.shape[0]), int(lmax), dirs is not None)


def must_workspace_bytes(liz: Liz, n_items: int, opts: must_solve_opts | None = None) -> int:
    return int(load().must_workspace_bytes(liz.handle, int(n_items), ctypes.byref(opts) if opts else None))


def must_batch_workspace_bytes(lizs, n_items_per_liz: int, opts: must_solve_opts | None = None) -> int:
    arr = (ctypes.c_void_p * len(lizs))(*[z.handle.value for z in lizs])
    return int(load().must_batch_workspace_bytes(len(lizs), arr, int(n_items_per_liz),
                                                 ctypes.byref(opts) if opts else None))


def must_tinv_square_well(E, V, r_mt: float, lmax: int, tinv, stream=None):
    """E: [nE] complex128 (as float64 pairs), V: [n_pot] float64, tinv: [n_pot][nE][lmax+1] complex128."""
    nE = _numel_complex(E)
    n_pot = V.numel() if hasattr(V, "numel") else int(np.asarray(V).size)
    _check(load().must_tinv_square_well(nE, _ptr(E), n_pot, _ptr(V), float(r_mt), int(lmax), _ptr(tinv),
                                        _stream(stream)))
    return tinv


def _numel_complex(a):
    if hasattr(a, "numel"):
        return a.numel() if a.is_complex() else a.numel() // 2
    a = np.asarray(a)
    return a.size if np.iscomplexobj(a) else a.size // 2


def must_tau00_solve(liz: Liz, E, tinv, n_species: int, nspin: int, opts: must_solve_opts | None, workspace,
                     ws_bytes: int, tau00, status=None, stream=None):
    _check(load().must_tau00_solve(liz.handle, _numel_complex(E), _ptr(E), _ptr(tinv), int(n_species), int(nspin),
                                   ctypes.byref(opts) if opts else None, _ptr(workspace), int(ws_bytes), _ptr(tau00),
                                   _ptr(status), _stream(stream)))
    return tau00


def must_tau00_batch(lizs, E, tinv, n_species: int, nspin: int, opts: must_solve_opts | None, workspace,
                     ws_bytes: int, tau00, status=None, stream=None):
    arr = (ctypes.c_void_p * len(lizs))(*[z.handle.value for z in lizs])
    _check(load().must_tau00_batch(len(lizs), arr, _numel_complex(E), _ptr(E), _ptr(tinv), int(n_species), int(nspin),
                                   ctypes.byref(opts) if opts else None, _ptr(workspace), int(ws_bytes), _ptr(tau00),
                                   _ptr(status), _stream(stream)))
    return tau00


def must_tau00_solve_static(liz: Liz, E, tinv, n_species: int, nspin: int, tau00, status=None, stream=None):
    """FP64 solve in the library's own static scratch: for callers that cannot
    allocate a workspace.  All arrays must be device memory; calls that overlap
    on the GPU share (and race on) the one scratch array."""
    _check(load().must_tau00_solve_static(liz.handle, _numel_complex(E), _ptr(E), _ptr(tinv), int(n_species),
                                          int(nspin), _ptr(tau00), _ptr(status), _stream(stream)))
    return tau00


def must_static_scratch_bytes() -> int:
    return int(load().must_static_scratch_bytes())


class Plan:
    """Owning wrapper of a must_plan (a captured batched launch)."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep          # buffers the graph refers to

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.must_plan_free(self.handle)
            self.handle = None


def must_plan_batch(lizs, E, tinv, n_species: int, nspin: int, opts, workspace, ws_bytes: int, tau00,
                    status=None) -> Plan:
    arr = (ctypes.c_void_p * len(lizs))(*[z.handle.value for z in lizs])
    out = ctypes.c_void_p()
    _check(load().must_plan_batch(len(lizs), arr, _numel_complex(E), _ptr(E), _ptr(tinv), int(n_species),
                                  int(nspin), ctypes.byref(opts) if opts else None, _ptr(workspace), int(ws_bytes),
                                  _ptr(tau00), _ptr(status), ctypes.byref(out)))
    return Plan(out, (lizs, E, tinv, workspace, tau00, status))


def must_plan_launch(plan: Plan, stream=None):
    _check(load().must_plan_launch(plan.handle, _stream(stream)))


def must_tune_set(knob: int, value: int):
    _check(load().must_tune_set(int(knob), int(value)))


def must_tune_get(knob: int) -> int:
    return int(load().must_tune_get(int(knob)))


class Mlp:
    """Owning wrapper of a must_mlp (the warm-start network)."""

    def __init__(self, n_in: int, hidden: int, n_out: int, max_batch: int, seed: int = 0):
        h = ctypes.c_void_p()
        _check(load().must_mlp_create(int(n_in), int(hidden), int(n_out), int(max_batch), int(seed), ctypes.byref(h)))
        self.handle, self.n_in, self.hidden, self.n_out, self.max_batch = h, n_in, hidden, n_out, max_batch

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.must_mlp_free(self.handle)
            self.handle = None

    def param_count(self) -> int:
        return int(load().must_mlp_param_count(self.handle))


def must_mlp_get_params(net: Mlp, out, stream=None):
    _check(load().must_mlp_get_params(net.handle, _ptr(out), _stream(stream)))
    return out


def must_mlp_set_params(net: Mlp, params, stream=None):
    _check(load().must_mlp_set_params(net.handle, _ptr(params), _stream(stream)))


def must_mlp_forward(net: Mlp, x, y, stream=None):
    _check(load().must_mlp_forward(net.handle, int(x.shape[0]), _ptr(x), _ptr(y), _stream(stream)))
    return y


def must_mlp_gradients(net: Mlp, x, target, grads=None, loss=None, stream=None):
    _check(load().must_mlp_gradients(net.handle, int(x.shape[0]), _ptr(x), _ptr(target), _ptr(grads), _ptr(loss),
                                     _stream(stream)))


def must_mlp_train_step(net: Mlp, x, target, lr: float, loss=None, stream=None):
    _check(load().must_mlp_train_step(net.handle, int(x.shape[0]), _ptr(x), _ptr(target), float(lr), _ptr(loss),
                                      _stream(stream)))


def must_mlp_save(net: Mlp, path: str):
    _check(load().must_mlp_save(net.handle, path.encode()))


def must_mlp_load(net: Mlp, path: str):
    _check(load().must_mlp_load(net.handle, path.encode()))


def must_mlp_features(kap: int, tau_prev, tau_next, E3, spin, occ, n_in: int, x, scale, interp, stream=None):
    n = int(tau_prev.shape[0])
    n_occ = int(occ.shape[1]) if occ is not None else 0
    _check(load().must_mlp_features(n, int(kap), _ptr(tau_prev), _ptr(tau_next), _ptr(E3), _ptr(spin), _ptr(occ),
                                    n_occ, int(n_in), _ptr(x), _ptr(scale), _ptr(interp), _stream(stream)))


def must_mlp_apply(kap: int, y, scale, interp, tau_pred, stream=None):
    _check(load().must_mlp_apply(int(y.shape[0]), int(kap), _ptr(y), int(y.shape[1]), _ptr(scale), _ptr(interp),
                                 _ptr(tau_pred), _stream(stream)))


def must_mlp_targets(kap: int, tau, scale, interp, y, stream=None):
    _check(load().must_mlp_targets(int(y.shape[0]), int(kap), _ptr(tau), _ptr(scale), _ptr(interp), _ptr(y),
                                   int(y.shape[1]), _stream(stream)))


def must_tau00_solve_seeded(liz: Liz, E, tinv, n_species: int, nspin: int, opts, workspace, ws_bytes: int, tau_seed,
                            seed_mask, tau00, status=None, seed_used=None, stream=None):
    _check(load().must_tau00_solve_seeded(liz.handle, _numel_complex(E), _ptr(E), _ptr(tinv), int(n_species),
                                          int(nspin), ctypes.byref(opts) if opts else None, _ptr(workspace),
                                          int(ws_bytes), _ptr(tau_seed), _ptr(seed_mask), _ptr(tau00), _ptr(status),
                                          _ptr(seed_used), _stream(stream)))
    return tau00


def must_contour_weights(n_e: int, e_bot: float = -0.3, e_f: float = 0.7):
    """(E, w): complex nodes and weights of int_{e_bot}^{e_f} f dE on the upper semicircle (host)."""
    E = np.zeros(n_e, np.complex128)
    w = np.zeros(n_e, np.complex128)
    _check(load().must_contour_weights(int(n_e), float(e_bot), float(e_f), _ptr(E.view(np.float64)),
                                       _ptr(w.view(np.float64))))
    return E, w


def must_site_charge(lmax: int, E, w, V, r_mt: float, tau00, n_of_E, N, stream=None):
    """Site charge of the centre (device tensors): tau00 [n_out][nE][kap][kap] complex128,
    E, w [nE] complex128, V [n_out] float64, n_of_E [n_out][nE] float64 or None, N [n_out] float64."""
    n_out, nE = int(tau00.shape[0]), int(tau00.shape[1])
    _check(load().must_site_charge(int(lmax), nE, _ptr(E), _ptr(w), n_out, _ptr(V), float(r_mt), _ptr(tau00),
                                   _ptr(n_of_E), _ptr(N), _stream(stream)))


def must_site_density(lmax: int, E, w, V, r_mt: float, tau00, r, n_of_r, stream=None):
    """Radial density inside the centre sphere (device tensors): tau00 [n_out][nE][kap][kap]
    complex128, E, w [nE] complex128, V [n_out] float64, r [n_r] float64, n_of_r [n_out][n_r]."""
    n_out, nE = int(tau00.shape[0]), int(tau00.shape[1])
    n_r = int(r.shape[0])
    _check(load().must_site_density(int(lmax), nE, _ptr(E), _ptr(w), n_out, _ptr(V), float(r_mt), _ptr(tau00),
                                    n_r, _ptr(r), _ptr(n_of_r), _stream(stream)))


class Kkr:
    """Owning wrapper of a must_kkr handle (full KKR of a periodic crystal)."""

    def __init__(self, handle, n_basis, lmax):
        self.handle = handle
        self.n_basis, self.lmax = n_basis, lmax
        self.kap = (lmax + 1) ** 2
        info = np.zeros(9, np.int32)   # see must_kkr_info
        _check(load().must_kkr_info(handle, _ptr(info)))
        (self.n, self.n_kpts, self.n_disp, self.n_pts, self.n_kK, self.n_kg, self.n_mesh,
         self.n_pts0, self.n_ops) = (int(v) for v in info)
        self.eta = float(load().must_kkr_eta(handle))
        self.table_bytes = int(load().must_kkr_table_bytes(handle))   # 0: no reciprocal-term table

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.must_kkr_free(self.handle)
            self.handle = None


MUST_KKR_NO_SYMMETRY = 1
MUST_KKR_NO_TABLE = 2


def must_kkr_build(lattice, basis, lmax: int, n_k: int, eta: float = 0.0, flags: int = 0, site_class=None,
                   stream=None) -> Kkr:
    lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(3, 3))
    bas = np.ascontiguousarray(np.asarray(basis, dtype=np.float64).reshape(-1, 3))
    cls = None if site_class is None else np.ascontiguousarray(np.asarray(site_class, dtype=np.int32))
    out = ctypes.c_void_p()
    _check(load().must_kkr_build(_ptr(lat), _ptr(bas), _ptr(cls), int(bas.shape[0]), int(lmax), int(n_k),
                                 float(eta), int(flags), _stream(stream), ctypes.byref(out)))
    return Kkr(out, int(bas.shape[0]), int(lmax))


KKR_INFO_FIELDS = ("n", "n_kpts", "n_disp", "n_pts", "n_kK", "n_kg", "n_mesh", "n_pts0", "n_ops")


def must_kkr_geometry(lattice, basis, lmax: int, n_k: int, eta: float = 0.0, flags: int = 0,
                      site_class=None) -> dict:
    """Host half of must_kkr_build (no device): the sizes must_kkr_info would
    report, keyed by KKR_INFO_FIELDS, plus 'eta'."""
    lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(3, 3))
    bas = np.ascontiguousarray(np.asarray(basis, dtype=np.float64).reshape(-1, 3))
    cls = None if site_class is None else np.ascontiguousarray(np.asarray(site_class, dtype=np.int32))
    info = np.zeros(9, np.int32)
    eta_used = np.zeros(1, np.float64)
    _check(load().must_kkr_geometry(_ptr(lat), _ptr(bas), _ptr(cls), int(bas.shape[0]), int(lmax), int(n_k),
                                    float(eta), int(flags), _ptr(info), _ptr(eta_used)))
    out = {k: int(v) for k, v in zip(KKR_INFO_FIELDS, info)}
    out["eta"] = float(eta_used[0])
    return out


def must_kkr_workspace_bytes(kkr: Kkr, n_items: int) -> int:
    return int(load().must_kkr_workspace_bytes(kkr.handle, int(n_items)))


def must_kkr_tau(kkr: Kkr, E, tinv, workspace, tau, status=None, stream=None):
    """E [n_items] complex128; tinv [n_items][n_basis][lmax+1] complex128;
    tau [n_items][n_basis][kap][kap] complex128 (column-major blocks); status [n_items] int32 or None."""
    n_items = _numel_complex(E)
    ws_bytes = int(workspace.numel() * workspace.element_size()) if hasattr(workspace, "numel") else workspace.nbytes
    _check(load().must_kkr_tau(kkr.handle, n_items, _ptr(E), _ptr(tinv), _ptr(workspace), ws_bytes, _ptr(tau),
                               _ptr(status), _stream(stream)))
    return tau
