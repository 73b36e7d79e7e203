"""Learned warm start: data, training and prediction around the library's MLP
kernels (marshalling only; features, targets, training steps and
predictions run in the CUDA library).

Schedule along a contour of nE energies: the even points and the last one
are solved cold; every odd k in 1..nE-3 is predicted from tau_00(E_{k-1}) and
tau_00(E_{k+1}) (both solved), the three energies, the spin and the LIZ's
species occupancy.  The network predicts the correction to linear
interpolation in units of the neighbours' half-difference.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as B
from .runner import Session
from .workload import Workload, random_liz, semicircle_contour, spin_depths, R_MT

N_OCC_SITES = 135


def n_inputs(kap: int, n_occ: int = 2 * N_OCC_SITES) -> int:
    return 4 * kap * kap + n_occ + 8


def occupancy(liz, n_sites: int = N_OCC_SITES) -> np.ndarray:
    """One-hot species per LIZ site (site order of the LIZ, centre first)."""
    occ = np.zeros(2 * n_sites, np.float32)
    for j, s in enumerate(liz.species[:n_sites]):
        occ[2 * j + int(s)] = 1.0
    return occ


def predicted_points(nE: int):
    return list(range(1, nE - 2, 2))


def samples_from_solution(tau: torch.Tensor, w: Workload, liz_index_offset: int = 0):
    """Gather (tau_prev, tau_next, tau_target, E3, spin, occ) for every LIZ, spin
    and predicted point of a batch solution tau [n_liz][n_out][nE][kap][kap]."""
    n_liz, n_out, nE = tau.shape[0], tau.shape[1], tau.shape[2]
    ks = predicted_points(nE)
    li, si, ki = np.meshgrid(np.arange(n_liz), np.arange(n_out), np.array(ks), indexing="ij")
    li, si, ki = li.ravel(), si.ravel(), ki.ravel()
    dev = tau.device
    lt, st, kt = (torch.tensor(a, device=dev) for a in (li, si, ki))
    tprev, tnext, ttgt = tau[lt, st, kt - 1], tau[lt, st, kt + 1], tau[lt, st, kt]
    E = torch.tensor(np.asarray(w.energies), device=dev)
    E3 = torch.stack([E[kt - 1], E[kt], E[kt + 1]], dim=1).contiguous()
    spin = torch.tensor(np.where(si == 0, 1.0, -1.0).astype(np.float32), device=dev)
    occ = torch.tensor(np.stack([occupancy(w.lizs[j]) for j in li]), device=dev)
    return tprev.contiguous(), tnext.contiguous(), ttgt.contiguous(), E3, spin, occ


class WarmStart:
    """The network plus feature/target marshalling."""

    def __init__(self, kap: int = 16, hidden: int = 256, max_batch: int = 1024, seed: int = 16322):
        self.kap = kap
        self.n_in = n_inputs(kap)
        self.n_out = 2 * kap * kap
        self.net = B.Mlp(self.n_in, hidden, self.n_out, max_batch, seed)
        self.max_batch = max_batch

    def features(self, tprev, tnext, E3, spin, occ):
        n = tprev.shape[0]
        dev = tprev.device
        x = torch.empty((n, self.n_in), dtype=torch.float32, device=dev)
        scale = torch.empty(n, dtype=torch.float32, device=dev)
        interp = torch.empty((n, self.kap, self.kap), dtype=torch.complex128, device=dev)
        B.must_mlp_features(self.kap, tprev, tnext, E3, spin, occ, self.n_in, x, scale, interp)
        return x, scale, interp

    def targets(self, ttgt, scale, interp):
        y = torch.empty((ttgt.shape[0], self.n_out), dtype=torch.float32, device=ttgt.device)
        B.must_mlp_targets(self.kap, ttgt, scale, interp, y)
        return y

    def predict(self, tprev, tnext, E3, spin, occ):
        x, scale, interp = self.features(tprev, tnext, E3, spin, occ)
        n = x.shape[0]
        y = torch.empty((n, self.n_out), dtype=torch.float32, device=x.device)
        for b0 in range(0, n, self.max_batch):
            b1 = min(n, b0 + self.max_batch)
            B.must_mlp_forward(self.net, x[b0:b1], y[b0:b1])
        pred = torch.empty_like(tprev)
        B.must_mlp_apply(self.kap, y, scale, interp, pred)
        return pred, interp

    def train(self, x, y, epochs: int = 30, batch: int = 512, lr: float = 1e-3, seed: int = 0):
        """Adam with cosine decay over shuffled mini-batches; returns the mean
        loss of each epoch."""
        n = x.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        steps = epochs * max(1, n // batch)
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        hist = []
        s = 0
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g).to(x.device)
            tot, cnt = 0.0, 0
            for b0 in range(0, n - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                xb, yb = x[idx].contiguous(), y[idx].contiguous()
                lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
                B.must_mlp_train_step(self.net, xb, yb, lr_s, loss)
                tot += loss.item()
                cnt += 1
                s += 1
            hist.append(tot / max(1, cnt))
        return hist


def random_liz_workload(first_seed: int, count: int, n_e: int = 32, lmax: int = 3) -> Workload:
    """`count` random 50/50 135-site LIZs (seeds first_seed ..), the benchmark
    contour and two spins (the training set of the warm start)."""
    lizs = [random_liz(first_seed + i) for i in range(count)]
    return Workload("random135", lmax, lizs, semicircle_contour(n_e, im_min=0.005), spin_depths(2), R_MT)


def solve_all(w: Workload, opts=None, chunk: int = 16):
    """tau [n_liz][n_out][nE][kap][kap] (row, col) for every LIZ of w, solved by
    the library's batched call in groups of `chunk` LIZs."""
    out = []
    for c0 in range(0, len(w.lizs), chunk):
        sub = Workload(w.name, w.lmax, w.lizs[c0:c0 + chunk], w.energies, w.v_species, w.r_mt, w.canted)
        s = Session(sub)
        tau, st = s.solve_batch(opts)
        torch.cuda.synchronize()
        if not bool((st == 0).all()):
            raise RuntimeError("a training solve did not converge")
        out.append(tau.transpose(-1, -2).contiguous())
    return torch.cat(out, 0)


def rel_err(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    return torch.linalg.norm((a - b).reshape(a.shape[0], -1), dim=1) / torch.linalg.norm(b.reshape(b.shape[0], -1),
                                                                                          dim=1)
