"""Convenience layer over the C ABI for workloads from ``workload``: builds the
handles, puts energies and t^{-1} on the device (t^{-1} by the library's own
square-well kernel), sizes the workspace and calls ``must_tau00_solve`` /
``must_tau00_batch``.  Marshalling only; every step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .workload import Workload


class Session:
    def __init__(self, w: Workload, device: str = "cuda", lizs=None):
        self.w = w
        self.device = torch.device(device)
        idx = range(len(w.lizs)) if lizs is None else lizs
        self.lizs = [B.must_liz_build(w.lizs[i].pos, w.lizs[i].species, w.lmax,
                                      w.lizs[i].dirs if w.canted else None) for i in idx]
        self.E = torch.tensor(np.asarray(w.energies, np.complex128), device=self.device)
        V = torch.tensor(np.asarray(w.v_species, np.float64).reshape(-1), device=self.device)
        self.n_species = int(w.v_species.shape[1])
        self.nspin = int(w.v_species.shape[0])
        self.tinv = torch.empty((self.nspin * self.n_species, len(w.energies), w.lmax + 1), dtype=torch.complex128,
                                device=self.device)
        B.must_tinv_square_well(self.E, V, w.r_mt, w.lmax, self.tinv)
        self.n_out = 1 if w.canted else self.nspin
        self.kap = self.lizs[0].kappa
        self._ws = None

    def workspace(self, n_bytes: int):
        if self._ws is None or self._ws.numel() < n_bytes:
            self._ws = None
            self._ws = torch.empty(n_bytes, dtype=torch.uint8, device=self.device)
        return self._ws

    def alloc_out(self, n_liz: int = 1):
        nE = len(self.w.energies)
        tau = torch.empty((n_liz, self.n_out, nE, self.kap, self.kap), dtype=torch.complex128, device=self.device)
        st = torch.zeros((n_liz, self.n_out, nE), dtype=torch.int32, device=self.device)
        return tau, st

    def solve(self, opts=None, liz_index: int = 0, ws_bytes: int | None = None, out=None, stream=None):
        """tau_00 for every energy/spin of one LIZ -> (tau [n_out][nE][kap][kap] torch, status)."""
        liz = self.lizs[liz_index]
        nE = len(self.w.energies)
        items = nE * (1 if self.w.canted else self.nspin)
        if ws_bytes is None:
            ws_bytes = B.must_workspace_bytes(liz, items, opts)
        ws = self.workspace(ws_bytes)
        tau, st = out if out is not None else self.alloc_out(1)
        B.must_tau00_solve(liz, self.E, self.tinv, self.n_species, self.nspin, opts, ws, ws_bytes, tau[0], st[0],
                           stream=stream)
        return tau[0], st[0]

    def solve_batch(self, opts=None, ws_bytes: int | None = None, out=None, stream=None):
        nE = len(self.w.energies)
        items = nE * (1 if self.w.canted else self.nspin)
        if ws_bytes is None:
            ws_bytes = B.must_batch_workspace_bytes(self.lizs, items, opts)
        ws = self.workspace(ws_bytes)
        tau, st = out if out is not None else self.alloc_out(len(self.lizs))
        B.must_tau00_batch(self.lizs, self.E, self.tinv, self.n_species, self.nspin, opts, ws, ws_bytes, tau, st,
                           stream=stream)
        return tau, st


def blocks_to_numpy(tau: torch.Tensor) -> np.ndarray:
    """Column-major kap x kap blocks -> numpy arrays indexed [..., row, col]."""
    return tau.detach().cpu().numpy().swapaxes(-1, -2).copy()
