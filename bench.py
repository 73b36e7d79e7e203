#!/usr/bin/env python3
"""Throughput benchmark of the LSMS tau_00 hot path on GB300.

One step = every (energy, spin) tau_00 of a 135-site fcc LIZ at lmax = 3
(n = 2160): 32 contour energies x 2 spins = 64 solves, each covering device
assembly of M = t^{-1} - g0, elimination of the leading n - 16 columns and
tau_00 (plus FP64 refinement on the mixed path).  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--precision bf16x3|tf32x3|fp64]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

Multi-GPU (torchrun): every rank solves its own LIZ (independent problems,
weak scaling, no collective on the data path); the barrier and the max over
ranks are for timing only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "τ_00 solves/sec at N_LIZ=135,l_max=3 (n=2160) vs plain FP64; % tensor peak"

TUNE = {}   # knob -> value set through --tune (library defaults otherwise)


def emit(line):
    """Print one JSON result line; non-default library knobs are recorded in it."""
    if TUNE and isinstance(line, dict):
        line = dict(line, tune={str(k): v for k, v in TUNE.items()})
    print(json.dumps(line))

UNIT = "solves/s"
PREC = {"fp64": 0, "bf16x3": 1, "tf32x3": 2}
RES = {"fp64": 0, "df": 1, "int": 2, "tc": 3}
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 (profiling recipe); DFMA/DMMA microbenchmark: 1.01-1.05
FP32_PEAK_TFLOPS = 80.5      # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (measured FFMA: 75)
FP32_INSTR_PEAK = 40.3       # T FP32 instructions/s: 152 SMs x 128 lanes x 2.07 GHz


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def code_sha256(path: str) -> str:
    """sha256 of a C/CUDA source with its comments and blank lines removed, so
    that a capture stays valid across comment-only edits of the kernel file."""
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    lines = [ln.rstrip() for ln in text.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def traffic_from_profiles(kernel_key: str, source: str, algorithmic_per_launch: float | None = None):
    """DRAM bytes per launch from profiles/<kernel_key>.txt, if the code of the
    kernel source it was captured from is unchanged (code_sha256 line); else
    None.  The file gives either the bytes per launch or the ratio of DRAM
    bytes to algorithmic bytes over a captured step, which is applied to
    algorithmic_per_launch."""
    path = os.path.join(ROOT, "profiles", kernel_key + ".txt")
    if not os.path.exists(path):
        return None
    sha = code_sha256(os.path.join(ROOT, source))
    vals = {}
    for ln in open(path):
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("code_sha256") != sha:
        return None
    try:
        if "dram_to_algorithmic" in vals:
            return None if algorithmic_per_launch is None else float(vals["dram_to_algorithmic"]) * algorithmic_per_launch
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def update_bytes(n: int, r: int, nb: int, pair_rows: int = 0) -> int:
    """C bytes the mixed path's trailing update reads and writes per matrix
    (16 B per complex-FP32 element per pass): one pass over the m x m
    trailing block per panel step, or, for paired steps (knob 11), step k's
    update of panel k+1's columns and rows plus one pass for both steps."""
    byts, k0 = 0, 0
    while k0 < r:
        nbe = min(nb, r - k0)
        k1 = k0 + nbe
        if pair_rows > 0 and nbe == nb and k1 + nb <= r and n - (k1 + nb) >= pair_rows:
            k2 = k1 + nb
            byts += 16 * (n - k1) * nb + 16 * nb * (n - k2) + 16 * (n - k2) ** 2
            k0 = k2
        else:
            byts += 16 * (n - k1) ** 2
            k0 = k1
    return byts


def phase_work(phase: str, n: int, kap: int, nb: int, items: int, precision: str, residual: str = "df",
               pair_rows: int = 0):
    """Algorithmic work of `items` matrices in one phase of one step:
    (amount, unit, bound, kernel source, profile key)."""
    r = n - kap
    if phase == "trailing_update":
        if precision != "fp64":
            # HBM-bound on the mixed path: the trailing block read and written once per pass
            return float(update_bytes(n, r, nb, pair_rows)) * items, "byte", "hbm", \
                "paper_2308_16317_gb300/csrc/tc_gemm.cu", "tc_update_kernel_fcc135"
        macs = 0
        for k0 in range(0, r, nb):
            nbe = min(nb, r - k0)
            m = n - k0 - nbe
            macs += m * m * nbe
        return macs * 8 * items, "flop", "alu", "paper_2308_16317_gb300/csrc/lu64.cu", "gemm64_kernel_fcc135"
    if phase == "residual":
        if residual == "tc":
            # tensor-core digit split: bound by one read of M's double-float copy (16 B per element)
            return 16.0 * n * n * items, "byte", "hbm", "paper_2308_16317_gb300/csrc/tc_residual.cu", \
                "residual_tc_kernel_fcc135"
        return 8.0 * n * n * kap * items, "flop", "alu", "paper_2308_16317_gb300/csrc/mixed.cu", \
            {"df": "residual_df_kernel_fcc135", "int": "residual_int_kernel_fcc135"}.get(residual,
                                                                                       "residual64_kernel_fcc135")
    if phase == "correction":
        return 8.0 * n * n * kap * items, "flop", "alu", "paper_2308_16317_gb300/csrc/mixed.cu", \
            "correct_kernel_fcc135"
    if phase == "assemble":
        bpe = 16 + (8 if precision != "fp64" else 0)
        return float(n) * n * bpe * items, "byte", "hbm", "paper_2308_16317_gb300/csrc/assemble.cu", \
            "assemble_kernel_fcc135"
    if phase == "panel":
        fl = 0
        for k0 in range(0, r, nb):
            nbe = min(nb, r - k0)
            fl += 8 * (n - k0) * nbe * nbe / 2
        return fl * items, "flop", "alu", "paper_2308_16317_gb300/csrc/mixed.cu", "panel32_kernel_fcc135"
    return None


class InflightPlans:
    """depth captured plans of the same solve, each with its own workspace,
    input copies (E, t^-1) and outputs; step i runs plan i % depth on stream
    i % depth, all streams forked from and joined back into the caller's."""

    def __init__(self, B, s, opts, items, depth, dev):
        import torch
        self.B, self.depth = B, depth
        nb = B.must_batch_workspace_bytes(s.lizs, items, opts)
        self.plans, self.outs, self.inputs, self.ws = [], [], [], []
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(depth)]
        for _ in range(depth):
            E, T = s.E.clone(), s.tinv.clone()
            w = torch.empty(nb, dtype=torch.uint8, device=dev)
            o = s.alloc_out(1)
            self.plans.append(B.must_plan_batch(s.lizs, E, T, s.n_species, s.nspin, opts, w, nb, o[0], o[1]))
            self.outs.append(o)
            self.inputs.append((E, T))
            self.ws.append(w)
        self.host_out = None

    def _fork(self, stream):
        for x in self.streams:
            x.wait_stream(stream)

    def _join(self, stream):
        for x in self.streams:
            stream.wait_stream(x)

    def launch(self, steps, stream):
        self._fork(stream)
        for i in range(steps):
            j = i % self.depth
            self.B.must_plan_launch(self.plans[j], stream=self.streams[j])
        self._join(stream)

    def e2e(self, steps, E_h, T_h, stream):
        import torch
        if self.host_out is None:
            self.host_out = [(torch.empty(o[0][0].shape, dtype=o[0].dtype).pin_memory(),
                              torch.empty(o[1][0].shape, dtype=o[1].dtype).pin_memory()) for o in self.outs]
        self._fork(stream)
        for i in range(steps):
            j = i % self.depth
            with torch.cuda.stream(self.streams[j]):
                E, T = self.inputs[j]
                E.copy_(E_h, non_blocking=True)
                T.copy_(T_h, non_blocking=True)
                self.B.must_plan_launch(self.plans[j], stream=self.streams[j])
                self.host_out[j][0].copy_(self.outs[j][0][0], non_blocking=True)
                self.host_out[j][1].copy_(self.outs[j][1][0], non_blocking=True)
        self._join(stream)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    libbuild.build()
    B.load()
    w = wl.liz135(seed=wl.SEED_BASE + 2 + rank, n_e=args.n_energies)
    s = Session(w, device="cuda:%d" % local)
    n, kap = s.lizs[0].n, s.kap
    items = len(w.energies) * s.nspin
    prec = args.precision
    opts = B.must_default_opts(PREC[prec], residual=RES[args.residual])
    nb = 64 if prec != "fp64" else 32

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    stream = torch.cuda.current_stream(dev)
    out = s.alloc_out(1)
    for _ in range(args.warmup):
        s.solve(opts, out=out)
    torch.cuda.synchronize(dev)
    st0 = out[1].cpu().numpy()
    # the step as a captured plan (must_plan_batch / must_plan_launch): the
    # whole launch sequence of the call replayed as one CUDA graph, recomputing
    # everything from E and t^-1 every time.  With --inflight D, D plans (own
    # workspace, inputs and outputs each) take the steps in turn on D streams,
    # so that D independent solves are in flight: one solve's latency-bound
    # panel chain and refinement leave the GPU room for the next one's work.
    plan = None
    pset = None
    if not args.no_plan:
        pset = InflightPlans(B, s, opts, items, max(1, args.inflight), dev)
        plan = pset.plans[0]
        pset.launch(args.warmup * pset.depth, stream)
        torch.cuda.synchronize(dev)
    plan_out = pset.outs[0] if pset else None

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    def timed_region(profiled: bool, use_plan: bool = False):
        # K steps between a barrier + synchronize on both sides, CUDA events on
        # the launching stream; the headline region replays the plan with the
        # library's per-phase instrumentation off, a second region of direct
        # calls with it on gives the phase split and the dominant kernel's
        # launch times
        barrier()
        torch.cuda.synchronize(dev)
        B.must_profile_enable(profiled)
        B.must_profile_read()
        l0 = B.must_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if use_plan:
            pset.launch(args.steps, stream)
        else:
            for _ in range(args.steps):
                s.solve(opts, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        l1 = B.must_launch_count()
        prof = B.must_profile_read() if profiled else None
        B.must_profile_enable(False)
        return max_over_ranks(e0.elapsed_time(e1)), l1 - l0, prof

    ms_total, n_launches, _ = timed_region(False, use_plan=plan is not None)
    clocks = sampler.stop() if rank == 0 else None
    ms_step = ms_total / args.steps
    value = items * ws * args.steps / (ms_total / 1e3)
    hout = plan_out if plan is not None else out
    tau_fast = blocks_to_numpy(hout[0][0])
    status = hout[1].cpu().numpy()
    direct = None
    one_in_flight = None
    if plan is not None:
        ms_direct, _, _ = timed_region(False)
        direct = {"value": items * ws * args.steps / (ms_direct / 1e3), "ms_per_step": ms_direct / args.steps,
                  "identical_to_plan": bool(np.array_equal(blocks_to_numpy(out[0][0]), tau_fast))}
        if pset.depth > 1:
            # the same plan replays, one solve at a time on the caller's stream
            barrier()
            torch.cuda.synchronize(dev)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for _ in range(args.steps):
                B.must_plan_launch(plan, stream=stream)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            ms1 = max_over_ranks(g0.elapsed_time(g1))
            one_in_flight = {"value": items * ws * args.steps / (ms1 / 1e3), "ms_per_step": ms1 / args.steps}
    ms_prof_total, _, prof = timed_region(True)
    status_prof = out[1].cpu().numpy()

    # roofline of the dominant phase (largest measured share of the step)
    peaks, peak_kind = load_peaks()
    dom = max((k for k in prof if k not in ("other",)), key=lambda k: prof[k][0])
    roofline = None
    pw = phase_work(dom, n, kap, nb, 1, prec, args.residual, B.must_tune_get(11))
    if pw is not None:
        per_item, unit, bound, src, key = pw
        ms_d, launches_d, items_d = prof[dom]
        if dom in ("residual", "correction"):
            total = per_item * items_d                      # items actually processed (device counted)
        else:
            total = per_item * items * args.steps           # whole-step work of this phase
        achieved = total / (ms_d / 1e3)
        if bound == "tensor":
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")) * 1e12
            punit, scale = "TFLOP/s", 1e12
        elif bound == "hbm":
            peak = peaks["hbm_gbs"] * 1e9
            punit, scale = "GB/s", 1e9
        elif dom == "residual" and args.residual == "int":
            # split-integer residual: per complex MAC 3 64-bit integer multiply-adds (a quarter of the FP32
            # rate, 4 issue slots each) + 8 FFMA + ~3 for splitting M: ~23 FP32-slot equivalents
            achieved = achieved / 8.0 * 23.0
            peak = FP32_INSTR_PEAK * 1e12
            punit, scale = "Tslots/s (FP32-equivalent)", 1e12
        elif dom == "residual" and args.residual == "df":
            # double-float residual: 48 FP32 instructions per complex MAC (8 FP64-equivalent flops)
            achieved = achieved / 8.0 * 48.0
            peak = FP32_INSTR_PEAK * 1e12
            punit, scale = "Tinstr/s (FP32)", 1e12
        else:
            peak = (FP64_PEAK_TFLOPS if dom == "residual" or prec == "fp64" else FP32_PEAK_TFLOPS) * 1e12
            punit, scale = "TFLOP/s", 1e12
        traffic = traffic_from_profiles(key, src, total / max(launches_d, 1))
        tensor_view = None
        if dom == "trailing_update" and prec != "fp64":
            # the same launches seen as tensor-core work: 24 tensor flops per complex MAC
            # (4 real MACs x 3 split products x 2)
            macs = 0
            for k0 in range(0, n - kap, nb):
                nbe = min(nb, n - kap - k0)
                m = n - k0 - nbe
                macs += m * m * nbe
            tf = macs * 24.0 * items * args.steps / (ms_d / 1e3)
            tp = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")) * 1e12
            tensor_view = {"achieved": tf / 1e12, "peak": tp / 1e12, "unit": "TFLOP/s", "frac": tf / tp}
        roofline = {"kernel_phase": dom, "bound": bound, "achieved": achieved / scale, "peak": peak / scale,
                    "unit": punit, "frac": achieved / peak, "traffic": traffic,
                    "peak_source": (peak_kind + " (MEASURED_PEAKS)") if bound in ("tensor", "hbm")
                    else "nominal FP64/FP32 from unit counts and clocks",
                    "algorithmic_per_launch": total / max(launches_d, 1),
                    "avg_launch_ms": ms_d / max(launches_d, 1), "launches": launches_d,
                    "share_of_step": ms_d / ms_prof_total, "tensor_view": tensor_view,
                    "timed_in": "a second %d-step region with per-phase CUDA events on (%.3f ms/step)"
                                % (args.steps, ms_prof_total / args.steps)}
    phases = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
              for k, v in prof.items() if v[1] > 0}

    # plain FP64 path on the same workload (the comparison the metric names)
    fp64 = None
    max_err = None
    if prec != "fp64" and args.fp64_steps > 0:
        o64 = B.must_default_opts(0)
        out64 = s.alloc_out(1)
        s.solve(o64, out=out64)
        torch.cuda.synchronize(dev)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.fp64_steps):
            s.solve(o64, out=out64)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = max_over_ranks(f0.elapsed_time(f1)) / args.fp64_steps
        fp64 = {"value": items * ws / (fms / 1e3), "ms_per_step": fms}
        t64 = blocks_to_numpy(out64[0][0])
        max_err = float((np.linalg.norm(tau_fast - t64, axis=(-2, -1)) / np.linalg.norm(t64, axis=(-2, -1))).max())

    # end to end through the C ABI with pinned host buffers
    E_h = torch.tensor(np.asarray(w.energies), dtype=torch.complex128).pin_memory()
    T_h = s.tinv.cpu().pin_memory()
    tau_h = torch.empty((s.n_out, len(w.energies), kap, kap), dtype=torch.complex128).pin_memory()
    sta_h = torch.empty((s.n_out, len(w.energies)), dtype=torch.int32).pin_memory()
    wsb = B.must_workspace_bytes(s.lizs[0], items, opts)
    wsp = s.workspace(wsb)
    B.must_tau00_solve(s.lizs[0], E_h, T_h, s.n_species, s.nspin, opts, wsp, wsb, tau_h, sta_h)
    barrier()
    t0 = time.perf_counter()
    e_steps = max(1, min(args.steps, 5))
    for _ in range(e_steps):
        B.must_tau00_solve(s.lizs[0], E_h, T_h, s.n_species, s.nspin, opts, wsp, wsb, tau_h, sta_h)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": items * ws * e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(E_h.numel() * 16 + T_h.numel() * 16),
           "d2h_bytes_per_step": int(tau_h.numel() * 16 + sta_h.numel() * 4),
           "path": "must_tau00_solve with pinned host buffers (staged by the library)"}
    if plan is not None:
        # the same through the plans: every step copies E and t^-1 from pinned
        # host memory into its plan's input buffers, replays the plan and reads
        # tau_00 and the status back into pinned host memory; the region ends
        # when every stream is done
        pset.e2e(pset.depth, E_h, T_h, stream)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        pset.e2e(e_steps, E_h, T_h, stream)
        torch.cuda.synchronize(dev)
        e2e_p = max_over_ranks(time.perf_counter() - t0)
        e2e_direct = e2e
        e2e = {"value": items * ws * e_steps / e2e_p, "unit": UNIT,
               "h2d_bytes_per_step": int(E_h.numel() * 16 + T_h.numel() * 16),
               "d2h_bytes_per_step": int(tau_h.numel() * 16 + sta_h.numel() * 4),
               "path": "plan replays (must_plan_launch, %d solves in flight) with the inputs copied from and "
                       "tau_00 read back to pinned host memory every step" % pset.depth, "direct_call": e2e_direct}

    cpu = None
    per_energy = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, o_items, o_tau = cpu_baseline(w, args.cpu_sample)
        # the headline's tau_00 against the oracle on the sampled (spin, energy) items
        errs = [float(np.linalg.norm(tau_fast[sp, e] - o_tau[q]) / np.linalg.norm(o_tau[q]))
                for q, (sp, e) in enumerate(o_items)]
        per_energy = {"max": max(errs), "items": [
            {"spin": sp, "e": e, "E": [float(w.energies[e].real), float(w.energies[e].imag)], "rel_err": er}
            for (sp, e), er in sorted(zip(o_items, errs), key=lambda t: (t[0][1], t[0][0]))]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "%s+f32 factors, %s residual, f64 solution" % (
                prec, {"fp64": "f64", "df": "double-float", "int": "split-integer",
                       "tc": "tensor-core digit-split"}[args.residual]),
            "data": "synthetic (seeded fcc 50/50 random alloy, square-well t-matrices)",
            "config": {"workload": "fcc135 LIZ, lmax=3, n=2160, 32 contour energies x 2 spins = 64 tau_00 solves/step",
                       "n": n, "n_liz": int(w.lizs[0].n_sites), "lmax": w.lmax, "solves_per_step": items,
                       "precision": prec, "residual": args.residual if prec != "fp64" else None, "l2": "inputs larger than L2 (%.1f GB of matrices per step)" % (
                           items * n * n * (24 if prec != "fp64" else 16) / 1e9)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(n_launches),
            "clocks": clocks, "plain_fp64": fp64, "max_rel_err_vs_fp64": max_err,
            "rel_err_vs_oracle_per_energy": per_energy,
            "status_ok": bool((status == 0).all() and (st0 == 0).all() and (status_prof == 0).all()),
            "phases": phases, "profiled_ms_per_step": ms_prof_total / args.steps,
            "timed": ("plan replays (the call captured once by must_plan_batch, replayed by must_plan_launch), "
                      "%d independent solves in flight on %d streams" % (pset.depth, pset.depth))
                     if plan is not None else "direct must_tau00_solve calls",
            "direct_calls": direct, "one_solve_in_flight": one_in_flight,
        }
        emit(line)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_supercell(args):
    """Batched uneven LIZs (per-site LIZs of the 256-site supercell, n 688..2160),
    one captured plan per precision, replayed every step."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import shard
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    libbuild.build()
    B.load()
    full = wl.batched_supercell()
    if args.shard == "balanced":
        # strong scaling: the first n_lizs LIZs split over the ranks by cost (sum of n^3)
        pool = full.lizs[:args.n_lizs]
        orders = [full.n_of(z) for z in pool]
        lizs = [pool[i] for i in shard.balanced_shards(orders, ws)[rank]]
    else:
        # weak scaling: every rank its own n_lizs LIZs
        lizs = full.lizs[rank * args.n_lizs:(rank + 1) * args.n_lizs]
    w = wl.Workload(full.name, full.lmax, lizs, wl.semicircle_contour(args.n_energies, im_min=0.005), full.v_species,
                    full.r_mt)
    s = Session(w, device="cuda:%d" % local)
    items = len(w.energies) * s.nspin * len(lizs)

    def max_over_ranks(x: float) -> float:
        if ws == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_plan(opts, steps, warm, parts=1):
        # the minimum holds one LIZ's items at the largest order; a multiple lets
        # that many LIZs share every launch.  parts > 1: the LIZs split into that
        # many cost-balanced parts (sum of n^3), each captured as its own plan with
        # its own workspace and outputs (the inputs E, t^-1 are shared read-only)
        # and replayed on its own stream, so that independent chunks are in flight
        # at once; every step still covers the whole batch.
        idx_parts = shard.balanced_shards([z.n for z in s.lizs], parts) if parts > 1 else [list(range(len(s.lizs)))]
        idx_parts = [ix for ix in idx_parts if ix]
        stream = torch.cuda.current_stream(dev)
        streams = [torch.cuda.Stream(device=dev) for _ in idx_parts] if len(idx_parts) > 1 else [stream]
        plans, outs, keep = [], [], []
        for ix in idx_parts:
            sub = [s.lizs[i] for i in ix]
            nbytes = B.must_batch_workspace_bytes(sub, len(w.energies) * s.nspin, opts) * max(1, args.chunk_lizs)
            wsp = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            tau_p, st_p = s.alloc_out(len(sub))
            plans.append(B.must_plan_batch(sub, s.E, s.tinv, s.n_species, s.nspin, opts, wsp, nbytes, tau_p, st_p))
            outs.append((tau_p, st_p))
            keep.append(wsp)

        def launch_all():
            if len(plans) == 1:
                B.must_plan_launch(plans[0], stream=stream)
                return
            for x in streams:
                x.wait_stream(stream)
            for pl, x in zip(plans, streams):
                B.must_plan_launch(pl, stream=x)
            for x in streams:
                stream.wait_stream(x)

        for _ in range(warm):
            launch_all()
        barrier()
        torch.cuda.synchronize(dev)
        l0 = B.must_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            launch_all()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        # outputs back in the batch's LIZ order
        tau, st = s.alloc_out(len(lizs))
        for ix, (tau_p, st_p) in zip(idx_parts, outs):
            for k, i in enumerate(ix):
                tau[i].copy_(tau_p[k])
                st[i].copy_(st_p[k])
        del keep
        return max_over_ranks(e0.elapsed_time(e1)), B.must_launch_count() - l0, tau, st

    prec = args.precision
    opts = B.must_default_opts(PREC[prec], residual=RES[args.residual])
    tuned = None
    if args.autotune:
        # grid search of the library's knobs on this batch (timed apart from the steps below)
        from paper_2308_16317_gb300 import autotune
        t0 = time.perf_counter()
        best, results = autotune.tune_session(s, opts, reps=2, workspace_lizs=max(1, args.chunk_lizs))
        tuned = {"best": best, "points": len(results or []), "seconds": time.perf_counter() - t0}
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    ms, launches, tau, st = timed_plan(opts, args.steps, args.warmup, parts=max(1, args.sc_parts))
    clocks = sampler.stop() if rank == 0 else None
    total_items = items
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([items], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        total_items = int(t.item())
    fp64 = None
    err = None
    if prec != "fp64" and args.fp64_steps > 0:
        ms64, _, tau64, _ = timed_plan(B.must_default_opts(0), args.fp64_steps, 1)
        fp64 = {"value": total_items * args.fp64_steps / (ms64 / 1e3), "ms_per_step": ms64 / args.fp64_steps}
        a, b = blocks_to_numpy(tau), blocks_to_numpy(tau64)
        err = float((np.linalg.norm(a - b, axis=(-2, -1)) / np.linalg.norm(b, axis=(-2, -1))).max())
    sizes = [z.n for z in s.lizs]
    # algorithmic work of the step (8/3 n^3 real flops per solve): LIZ mixes of
    # different sizes compare by this rate, not by solves/s
    work = sum(8.0 / 3.0 * float(n) ** 3 for n in sizes) * len(w.energies) * s.nspin
    line = {"metric": "tau_00 solves/sec, batched uneven LIZs (supercell, n %d..%d)" % (min(sizes), max(sizes)),
            "tflops_8_3_n3": work * args.steps / (ms / 1e3) / 1e12,
            "value": total_items * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.shard == "balanced" else "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": "supercell256 per-site LIZs with vacancies, lmax=3", "lizs_per_rank": len(lizs),
                       "shard": args.shard,
                       "workspace_lizs": max(1, args.chunk_lizs),
                       "energies": len(w.energies), "spins": s.nspin, "solves_per_step": items,
                       "n_min": min(sizes), "n_max": max(sizes), "precision": prec, "residual": args.residual,
                       "launch": "captured CUDA graph (must_plan_batch), replayed per step",
                       "parts_in_flight": max(1, args.sc_parts),
                       "bucket_sites": B.must_tune_get(0), "tile_n": B.must_tune_get(1)},
            "gpu_launches": int(launches), "clocks": clocks, "plain_fp64_batched": fp64,
            "max_rel_err_vs_fp64": err, "status_ok": bool((st.cpu().numpy() == 0).all()), "autotune": tuned}
    if rank == 0:
        emit(line)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_warmstart(args):
    """Learned warm start end to end: tau_00 training data from the method on
    seeded random 135-site LIZs, training with the library's kernels, then on
    the supercell's per-site LIZs: prediction error of the network vs linear
    interpolation, residual-gate acceptance of the seeds, and the throughput
    of the seeded schedule (even points cold, odd points seeded) vs solving
    every point cold."""
    import torch
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import warmstart as wsm
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session
    libbuild.build()
    B.load()
    opts = B.must_default_opts(PREC[args.precision], residual=RES[args.residual])
    t0 = time.perf_counter()
    train_w = wsm.random_liz_workload(100000, args.train_lizs)
    tau_tr = wsm.solve_all(train_w, opts)
    t_gen = time.perf_counter() - t0
    model = wsm.WarmStart(max_batch=1024)
    tp, tn, tt, E3, sp, oc = wsm.samples_from_solution(tau_tr, train_w)
    x, scale, interp = model.features(tp, tn, E3, sp, oc)
    y = model.targets(tt, scale, interp)
    t0 = time.perf_counter()
    hist = model.train(x, y, epochs=30, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del tau_tr, x, y
    full = wl.batched_supercell()
    ev = wl.Workload(full.name, full.lmax, full.lizs[:args.n_lizs], wl.semicircle_contour(32, im_min=0.005),
                     full.v_species, full.r_mt)
    nE = len(ev.energies)
    even = [k for k in range(nE) if k not in wsm.predicted_points(nE)]
    odd = wsm.predicted_points(nE)
    e_net, e_lin, used_all, t_cold, t_seed, n_solves, max_dev = [], [], [], 0.0, 0.0, 0, 0.0

    def ev_sub(lizs, ks):
        return wl.Workload(ev.name, ev.lmax, lizs, ev.energies[ks], ev.v_species, ev.r_mt)

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    for j, liz in enumerate(ev.lizs):
        s_all = Session(ev_sub([liz], list(range(nE))))
        ms_c, (tau_c, st_c) = timed(lambda: s_all.solve(opts))
        s_even = Session(ev_sub([liz], even))
        s_odd = Session(ev_sub([liz], odd))
        ms_e, (tau_e, _) = timed(lambda: s_even.solve(opts))
        # predict the odd points from their solved neighbours
        te = tau_e.transpose(-1, -2)                      # [n_out][len(even)][kap][kap] (row, col)
        pos = {k: i for i, k in enumerate(even)}
        prev = torch.stack([te[s_, pos[k - 1]] for s_ in range(2) for k in odd])
        nxt = torch.stack([te[s_, pos[k + 1]] for s_ in range(2) for k in odd])
        Et = torch.tensor(np.asarray(ev.energies), device=prev.device)
        E3 = torch.stack([torch.stack([Et[k - 1], Et[k], Et[k + 1]]) for _ in range(2) for k in odd]).contiguous()
        spin = torch.tensor([1.0] * len(odd) + [-1.0] * len(odd), dtype=torch.float32, device=prev.device)
        occ = torch.tensor(np.stack([wsm.occupancy(liz)] * (2 * len(odd))), device=prev.device)
        ms_p, (pred, interp) = timed(lambda: model.predict(prev.contiguous(), nxt.contiguous(), E3, spin, occ))
        seed = pred.reshape(2, len(odd), 16, 16).transpose(-1, -2).contiguous()   # column-major blocks
        mask = torch.ones((2, len(odd)), dtype=torch.int32, device=prev.device)
        items = 2 * len(odd)
        nb = B.must_workspace_bytes(s_odd.lizs[0], items, opts)
        wsp = torch.empty(nb, dtype=torch.uint8, device=prev.device)
        tau_o, st_o = s_odd.alloc_out(1)
        used = torch.zeros((2, len(odd)), dtype=torch.int32, device=prev.device)
        ms_o, _ = timed(lambda: B.must_tau00_solve_seeded(s_odd.lizs[0], s_odd.E, s_odd.tinv, s_odd.n_species,
                                                          s_odd.nspin, opts, wsp, nb, seed, mask, tau_o[0], st_o[0],
                                                          used))
        truth = tau_c.transpose(-1, -2)[:, odd].reshape(items, 16, 16)     # [spin][odd k] order
        e_net += wsm.rel_err(pred, truth).tolist()
        e_lin += wsm.rel_err(interp, truth).tolist()
        used_all += used.flatten().tolist()
        got = tau_o[0].transpose(-1, -2).reshape(items, 16, 16)
        max_dev = max(max_dev, float(wsm.rel_err(got, truth).max()))
        t_cold += ms_c
        t_seed += ms_e + ms_p + ms_o
        n_solves += 2 * nE
    line = {"metric": "learned warm start on batched supercell LIZs", "impl": "gb300",
            "train": {"lizs": args.train_lizs, "samples": int(tp.shape[0]), "generate_s": t_gen, "train_s": t_train,
                      "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]},
            "eval": {"lizs": len(ev.lizs), "predicted_points": len(e_net),
                     "median_rel_err_network": float(np.median(e_net)),
                     "median_rel_err_interpolation": float(np.median(e_lin)),
                     "p95_rel_err_network": float(np.percentile(e_net, 95)),
                     "p95_rel_err_interpolation": float(np.percentile(e_lin, 95)),
                     "prediction_gain": float(np.median(e_lin) / np.median(e_net)),
                     "seed_acceptance": float(np.mean(used_all)),
                     "seeded_vs_cold_max_rel_diff": max_dev,
                     "solves_per_s_cold": n_solves / (t_cold / 1e3),
                     "solves_per_s_seeded_schedule": n_solves / (t_seed / 1e3)},
            "precision": args.precision, "residual": args.residual}
    emit(line)


def run_canted(args):
    """Spin-canted 135-site LIZ (M of order 2n = 4320), 32 energies down to
    Im E = 0.00215: mixed-precision throughput, and per-energy error of the
    mixed path against the plain FP64 path on the same GPU."""
    import torch
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    libbuild.build()
    B.load()
    w = wl.canted135(n_e=args.n_energies)
    s = Session(w)
    opts = B.must_default_opts(PREC[args.precision], residual=RES[args.residual])
    out = s.alloc_out(1)
    for _ in range(args.warmup):
        s.solve(opts, out=out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.solve(opts, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tau = blocks_to_numpy(out[0][0])
    st = out[1].cpu().numpy()
    out64 = s.alloc_out(1)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    s.solve(B.must_default_opts(0), out=out64)
    f1.record()
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1)
    t64 = blocks_to_numpy(out64[0][0])
    err = np.linalg.norm(tau - t64, axis=(-2, -1)) / np.linalg.norm(t64, axis=(-2, -1))
    nE = len(w.energies)
    emit({"metric": "tau_00 solves/sec, spin-canted 135-site LIZ (order 2n = 4320)",
                      "value": nE / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": args.steps,
                      "precision": args.precision, "residual": args.residual,
                      "plain_fp64": {"value": nE / (ms64 / 1e3), "ms_per_step": ms64},
                      "status_ok": bool((st == 0).all()),
                      "per_energy_rel_err_vs_fp64": [float(x) for x in err.ravel()],
                      "im_E": [float(e.imag) for e in w.energies]})


def run_paper_shapes(args):
    """The paper's own ranks (Sec. 4.1, lmax = 4): a Ni30Au70-shaped 249-site LIZ
    (n = 6225, two spins), a CoCrFeMnNi-shaped canted 135-site LIZ (n = 6750)
    and the NiAu-shaped canted 249-site LIZ (n = 12450), 8 contour energies
    each; mixed-precision and plain FP64 throughput, and the mixed path's
    error against the FP64 path."""
    import torch
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session, blocks_to_numpy
    libbuild.build()
    B.load()
    res = {}
    shapes = [("niau249_n6225", wl.niau249(n_e=8)), ("cocrfemnni135_canted_n6750", wl.cocrfemnni135_canted(n_e=8)),
              ("niau249_canted_n12450", wl.niau249_canted(n_e=8))]
    for name, w in shapes:
        s = Session(w)
        items = len(w.energies) * (1 if w.canted else s.nspin)
        out = s.alloc_out(1)
        opts = B.must_default_opts(PREC[args.precision], residual=RES[args.residual])
        for _ in range(max(1, args.warmup)):
            s.solve(opts, out=out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            s.solve(opts, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        tau = blocks_to_numpy(out[0][0])
        ok = bool((out[1].cpu().numpy() == 0).all())
        out64 = s.alloc_out(1)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        s.solve(B.must_default_opts(0), out=out64)
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        t64 = blocks_to_numpy(out64[0][0])
        err = np.linalg.norm(tau - t64, axis=(-2, -1)) / np.linalg.norm(t64, axis=(-2, -1))
        n = s.lizs[0].n
        res[name] = {"n": int(n), "solves_per_step": items, "mixed_solves_per_s": items / (ms / 1e3),
                     "mixed_ms_per_step": ms, "fp64_solves_per_s": items / (ms64 / 1e3), "fp64_ms_per_step": ms64,
                     "fp64_lu_tflops": items * 8.0 / 3.0 * n ** 3 / (ms64 / 1e3) / 1e12,
                     "max_rel_err_vs_fp64": float(err.max()), "status_ok": ok}
        del s, out, out64
        torch.cuda.empty_cache()
    emit({"metric": "tau_00 solves/sec at the paper's ranks (lmax = 4)", "unit": UNIT,
                      "precision": args.precision, "residual": args.residual, "steps": args.steps,
                      "results": res})


def run_site_charge(args):
    """The step after the path: the charge inside the centre's sphere, the
    contour integral (Eq. 2) of the site Green's function (Eq. 3), from the
    tau_00 of the 135-site workload on the unclamped 32-node semicircle.
    Reports N per spin, the solve throughput and the charge kernel's time."""
    import torch
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import workload as wl
    from paper_2308_16317_gb300.runner import Session
    libbuild.build()
    B.load()
    w = wl.liz135(n_e=args.n_energies, im_min=None)
    s = Session(w)
    nE = len(w.energies)
    E, wt = B.must_contour_weights(nE)
    dev = torch.device("cuda")
    Ed = torch.tensor(E, device=dev)
    wd = torch.tensor(wt, device=dev)
    V = torch.tensor([w.site_depths(w.lizs[0], sp)[0] for sp in range(s.nspin)], dtype=torch.float64, device=dev)
    n_of_E = torch.zeros((s.nspin, nE), dtype=torch.float64, device=dev)
    N = torch.zeros(s.nspin, dtype=torch.float64, device=dev)
    opts = B.must_default_opts(PREC[args.precision], residual=RES[args.residual])
    out = s.alloc_out(1)
    for _ in range(args.warmup):
        s.solve(opts, out=out)
        B.must_site_charge(w.lmax, Ed, wd, V, w.r_mt, out[0][0], n_of_E, N)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t_solve = t_charge = 0.0
    for _ in range(args.steps):
        e0.record()
        s.solve(opts, out=out)
        e1.record()
        B.must_site_charge(w.lmax, Ed, wd, V, w.r_mt, out[0][0], n_of_E, N)
        e2.record()
        torch.cuda.synchronize()
        t_solve += e0.elapsed_time(e1)
        t_charge += e1.elapsed_time(e2)
    items = nE * s.nspin
    emit({"metric": "site charge inside the centre sphere from tau_00 (contour integral of Eq. 2-3)",
                      "N_per_spin": [float(x) for x in N.cpu().numpy()],
                      "n_of_E_per_spin": n_of_E.cpu().numpy().tolist(),
                      "solves_per_s": items * args.steps / (t_solve / 1e3),
                      "charge_kernel_ms": t_charge / args.steps, "solve_ms": t_solve / args.steps,
                      "precision": args.precision, "residual": args.residual,
                      "status_ok": bool((out[1].cpu().numpy() == 0).all())})


def run_cusolver_context(args):
    """Context only: the paper's own method (LU + solve in complex128, Sec. 3.2)
    through PyTorch's vendor-library path on this GPU, at the benchmark's
    matrix order with 16 right-hand sides.  The cost of LU + solve depends
    only on n, so a random well-conditioned complex128 matrix stands in for M.
    Not the library's path; reported beside it."""
    import torch
    n = 2160
    batch = 8
    g = torch.Generator(device="cuda").manual_seed(0)
    A = (torch.randn(batch, n, n, dtype=torch.float64, device="cuda", generator=g)
         + 1j * torch.randn(batch, n, n, dtype=torch.float64, device="cuda", generator=g)
         + n * torch.eye(n, dtype=torch.complex128, device="cuda"))
    Bm = torch.zeros(batch, n, 16, dtype=torch.complex128, device="cuda")
    Bm[:, n - 16:, :] = torch.eye(16, dtype=torch.complex128, device="cuda")
    for _ in range(max(1, args.warmup)):
        torch.linalg.solve(A, Bm)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        torch.linalg.solve(A, Bm)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    emit({"metric": "context: vendor complex128 LU + solve (torch.linalg.solve), n=2160, 16 RHS",
                      "value": batch / (ms / 1e3), "unit": UNIT, "ms_per_batch": ms, "batch": batch,
                      "tflops_8_3_n3": batch * 8 / 3 * n ** 3 / (ms / 1e3) / 1e12})


def run_peaks(args):
    """Measured arithmetic peaks of this GPU (the denominators of the FP64 and
    FP32 roofline fractions): DFMA, DMMA (FP64 tensor, mma.sync m8n8k4) and
    FFMA probes of the library (must_peak_probe), each launch sized to about
    150 ms and timed with CUDA events, best of 5, clocks sampled meanwhile."""
    import torch
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    libbuild.build()
    B.load()
    res = {}
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    for kind, name in ((0, "dfma_f64"), (1, "dmma_f64_m8n8k4"), (2, "ffma_f32")):
        res[name] = {}
        for per_sm in (4, 8):
            blocks = 152 * per_sm
            sink = torch.zeros(blocks * 256, dtype=torch.float64, device="cuda")
            iters = 256
            best = 0.0
            for trial in range(7):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                fl = B.must_peak_probe(kind, blocks, iters, sink)
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                if trial < 2:   # calibrate the launch to ~150 ms
                    iters = max(256, int(iters * 150.0 / max(ms, 1e-3)))
                    continue
                best = max(best, fl / (ms / 1e3))
            res[name]["%d_ctas_per_sm" % per_sm] = {"tflops": best / 1e12, "iters": iters}
        res[name]["tflops"] = max(v["tflops"] for v in res[name].values() if isinstance(v, dict))
    clocks = sampler.stop()
    emit({"metric": "measured arithmetic peaks (probe kernels, CUDA events, best of 5 launches of ~150 ms)",
          "unit": "TFLOP/s", "dfma_f64": res["dfma_f64"]["tflops"], "dmma_f64": res["dmma_f64_m8n8k4"]["tflops"],
          "ffma_f32": res["ffma_f32"]["tflops"], "detail": res, "clocks": clocks})


FP64_DFMA_MEASURED = 1.058   # TFLOP/s, the library's DFMA probe on this GPU (profiles/fp64_peak.md)


def kkr_work(h, c, items):
    """Algorithmic FP64 flops of one must_kkr_tau call, per kernel, as the
    kernels compute them: 4 real flops per multiply-add of a real number into a
    complex sum -- the reciprocal sums (every (k, K) term, every displacement
    and L''), the real-space sums (every (k, point, L''), a pair (x, -x) counting
    for both) -- and 8 per complex multiply-add of the in-place Gauss-Jordan
    inversion (n^3 per evaluated k point)."""
    nL2 = (2 * c.lmax + 1) ** 2
    return {"kkr_recip": 4.0 * items * h.n_kK * h.n_disp * nL2,
            "kkr_realsum": 4.0 * items * h.n_kpts * nL2 * (h.n_pts0 + 2 * (h.n_pts - h.n_pts0)),
            "kkr_invert": 8.0 * items * h.n_kpts * h.n ** 3}


def run_kkr(args):
    """Full KKR of a periodic crystal (the paper's Sec. 5 target): the
    site-diagonal tau of every site for 32 contour energies x 2 spins per step,
    by must_kkr_tau (Ewald structure constants, M(k) = t^-1 - G(k) inverted
    per k point, Brillouin-zone average), on the 4-site L1_2 cell (M(k) of
    order 64, 8^3 k points) and the primitive fcc cell (order 16, 16^3 k
    points).  Reports tau solves/s (one (energy, spin) item = all sites of the
    cell), M(k) inversions/s, the per-kernel split with the FP64 roofline of
    the dominant kernel, an end-to-end figure from pinned host buffers, and the
    oracle on the host cores on a bounded sample (errors of the sampled items
    against it)."""
    import torch
    import oracle
    from paper_2308_16317_gb300 import binding as B
    from paper_2308_16317_gb300 import build as libbuild
    from paper_2308_16317_gb300 import workload as wl
    libbuild.build()
    B.load()
    oracle.build()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    cores = min(16, os.cpu_count() or 1)
    crystals = []
    if args.kkr_cells in ("both", "l12"):
        crystals.append(wl.l12_crystal(n_k=8, n_e=args.n_energies))
    if args.kkr_cells in ("both", "fcc1"):
        crystals.append(wl.fcc_crystal(n_k=16, n_e=args.n_energies))
    results = {}
    for c in crystals:
        eta = 0.0
        if args.kkr_eta_scale != 1.0:
            # a multiple of 4 pi / Omega^(2/3) (the library's default is 1.0 of it, 0.7 with one site)
            eta = args.kkr_eta_scale * 4.0 * np.pi / abs(np.linalg.det(c.lattice)) ** (2.0 / 3.0)
        h = B.must_kkr_build(c.lattice, c.basis, c.lmax, c.n_k, eta=eta, site_class=c.species)
        nE = len(c.energies)
        picks = [(sp, e) for sp in range(c.nspin) for e in range(nE)]
        items = len(picks)
        # t^-1 of every (spin, species) well from the library's fixture kernel, gathered per (item, site)
        Vs = np.array([c.v_species[sp][k] for sp in range(c.nspin) for k in range(c.v_species.shape[1])])
        Ed_all = torch.tensor(c.energies, dtype=torch.complex128, device=dev)
        Vd = torch.tensor(Vs, dtype=torch.float64, device=dev)
        tab = torch.zeros((len(Vs), nE, c.lmax + 1), dtype=torch.complex128, device=dev)
        B.must_tinv_square_well(Ed_all, Vd, c.r_mt, c.lmax, tab)
        n_sp = c.v_species.shape[1]
        pot = torch.tensor([[sp * n_sp + int(c.species[b]) for b in range(c.n_basis)] for sp, _ in picks],
                           device=dev)
        eidx = torch.tensor([e for _, e in picks], device=dev)
        tinv = tab[pot, eidx[:, None]].contiguous()                    # [items][N_b][lmax+1]
        E = Ed_all[eidx].contiguous()
        ws = torch.empty(B.must_kkr_workspace_bytes(h, items), dtype=torch.uint8, device=dev)
        tau = torch.zeros((items, c.n_basis, h.kap, h.kap), dtype=torch.complex128, device=dev)
        st = torch.zeros(items, dtype=torch.int32, device=dev)
        for _ in range(args.warmup):
            B.must_kkr_tau(h, E, tinv, ws, tau, st)
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        time.sleep(0.2)
        l0 = B.must_launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            B.must_kkr_tau(h, E, tinv, ws, tau, st)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        launches = B.must_launch_count() - l0
        ms = e0.elapsed_time(e1) / args.steps
        # per-kernel split from a second region with the phase events on
        B.must_profile_enable(True)
        B.must_profile_read()
        for _ in range(args.steps):
            B.must_kkr_tau(h, E, tinv, ws, tau, st)
        torch.cuda.synchronize()
        prof = B.must_profile_read()
        B.must_profile_enable(False)
        kern = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                for k, v in prof.items() if k.startswith("kkr_") and v[1] > 0}
        work = kkr_work(h, c, items)
        for k, f in work.items():
            if k in kern and kern[k]["ms_per_step"] > 0:
                kern[k]["tflops"] = f / (kern[k]["ms_per_step"] / 1e3) / 1e12
                kern[k]["frac_of_measured_dfma"] = kern[k]["tflops"] / FP64_DFMA_MEASURED
        dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
        # end to end: inputs from pinned host memory, tau and status back, every step
        E_h = E.cpu().pin_memory()
        T_h = tinv.cpu().pin_memory()
        tau_h = torch.empty(tau.shape, dtype=tau.dtype).pin_memory()
        st_h = torch.empty(st.shape, dtype=st.dtype).pin_memory()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            E.copy_(E_h, non_blocking=True)
            tinv.copy_(T_h, non_blocking=True)
            B.must_kkr_tau(h, E, tinv, ws, tau, st)
            tau_h.copy_(tau, non_blocking=True)
            st_h.copy_(st, non_blocking=True)
        g1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = g0.elapsed_time(g1) / args.steps
        # the oracle on the host cores, on a bounded sample of the same items
        if args.no_cpu_baseline:
            results[c.name] = {"value": items / (ms / 1e3), "unit": "tau solves/s", "ms_per_step": ms,
                               "kernels": kern, "gpu_launches": launches, "clocks": clocks}
            continue
        sample = [picks[(k * 11) % items] for k in range(cores if c.n_basis == 1 else max(2, cores // 4))]
        si = [picks.index(p) for p in sample]
        Es = np.array([c.energies[e] for _, e in sample])
        Ts = tinv.cpu().numpy()[si]
        t0 = time.perf_counter()
        ref, used = oracle.kkr_tau(c.lmax, c.lattice, c.basis, Es, Ts, c.n_k, h.eta, nthreads=cores)
        dt = time.perf_counter() - t0
        got = np.swapaxes(tau.cpu().numpy()[si], -1, -2)
        err = np.linalg.norm(got - ref, axis=(-2, -1)) / np.linalg.norm(ref, axis=(-2, -1))
        results[c.name] = {
            "value": items / (ms / 1e3), "unit": "tau solves/s (all sites of the cell per (E, spin))",
            "ms_per_step": ms, "items_per_step": items, "n": h.n, "k_points": h.n_mesh,
            "k_points_evaluated": h.n_kpts, "point_group_ops": h.n_ops,
            "reciprocal_table_bytes": h.table_bytes,
            "inversions_per_s": items * h.n_kpts / (ms / 1e3),
            "gpu_launches": launches, "kernels": kern,
            "roofline": {"kernel_phase": dom, "bound": "alu", "unit": "TFLOP/s",
                         "achieved": kern[dom].get("tflops"), "peak": FP64_DFMA_MEASURED,
                         "peak_source": "measured DFMA probe (profiles/fp64_peak.md)",
                         "frac": kern[dom].get("frac_of_measured_dfma")},
            "e2e": {"value": items / (ms_e2e / 1e3), "unit": "tau solves/s",
                    "h2d_bytes_per_step": int(E.numel() * 16 + tinv.numel() * 16),
                    "d2h_bytes_per_step": int(tau.numel() * 16 + st.numel() * 4)},
            "cpu_baseline": {"value": len(sample) / dt, "unit": "tau solves/s", "cores": int(used), "kind": "oracle",
                             "sample": "%d of the %d items, one per thread, %.1f s" % (len(sample), items, dt)},
            "max_rel_err_vs_oracle": float(err.max()),
            "status_ok": bool((st.cpu().numpy() == 0).all()), "clocks": clocks, "eta": h.eta}
    emit({"metric": "full KKR (periodic crystal): site-diagonal tau solves/s, FP64", "data": "synthetic "
          "(square wells on the fcc lattice: L1_2 Ni3Au-like 4-site cell and a pure element's primitive cell)",
          "dtype": "f64", "steps": args.steps, "warmup": args.warmup, "crystals": results})


def cpu_baseline(w, sample: int):
    """The oracle on the host cores: `sample` (energy, spin) solves of the same
    LIZ, one per thread, timed end to end."""
    import oracle
    oracle.build()
    cores = sample if sample > 0 else min(16, os.cpu_count() or 1)
    nE = len(w.energies)
    items = [((k % 2), (k * 7) % nE) for k in range(cores)]
    liz = w.lizs[0]
    E = np.array([w.energies[e] for _, e in items])
    ti = np.array([oracle.site_tinv(w.lmax, w.energies[e], w.site_depths(liz, s), w.r_mt) for s, e in items])
    t0 = time.perf_counter()
    tau, _, used = oracle.tau00_batch(liz.pos, w.lmax, E, ti, nthreads=cores)
    dt = time.perf_counter() - t0
    return ({"value": len(items) / dt, "unit": UNIT, "cores": int(used), "kind": "oracle",
             "sample": "%d of the 64 (energy, spin) solves of the n=2160 LIZ, one per thread, %.1f s"
                       % (len(items), dt)}, items, tau)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2308_16317_gb300 import workload as wl
    w = wl.liz135()
    cores = args.cpu_sample if args.cpu_sample > 0 else min(16, os.cpu_count() or 1)
    for _ in range(args.warmup):
        cpu_baseline(w, max(1, cores // 4))
    times = []
    solves = 0
    for _ in range(args.steps):
        c = cpu_baseline(w, cores)[0]
        solves += cores
        times.append(cores / c["value"])
    total = sum(times)
    value = solves / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded fcc 50/50 random alloy, square-well t-matrices)",
            "config": {"workload": "fcc135 LIZ, lmax=3, n=2160, 32 contour energies x 2 spins = 64 tau_00 solves/step",
                       "n": 2160, "n_liz": 135, "lmax": 3, "solves_per_step": cores,
                       "note": "each step is a bounded sample: %d solves, one per host thread" % cores},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d steps x %d solves of the n=2160 LIZ" % (args.steps, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=list(PREC))
    ap.add_argument("--residual", default="tc", choices=list(RES),
                    help="refinement residual: FP64 (DFMA), double-float FP32 pairs, split-integer, or the "
                         "tensor-core digit split (default)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plan", action="store_true",
                    help="time direct must_tau00_solve calls instead of replays of the captured plan")
    ap.add_argument("--inflight", type=int, default=3,
                    help="independent solves in flight: captured plans taking the steps in turn on their own "
                         "streams (1: one plan, one stream)")
    ap.add_argument("--cpu-sample", type=int, default=0)
    ap.add_argument("--workload", default="liz135",
                    choices=["liz135", "supercell", "warmstart", "cusolver", "canted", "paper", "charge", "peaks",
                             "kkr"],
                    help="liz135: the benchmark workload; supercell: per-site LIZs of the 256-site supercell "
                         "with vacancies (uneven n), batched and replayed as a captured plan")
    ap.add_argument("--n-lizs", type=int, default=32, help="supercell / warmstart mode: evaluation LIZs")
    ap.add_argument("--kkr-eta-scale", type=float, default=1.0,
                    help="kkr mode: Ewald splitting parameter as a multiple of 4 pi / Omega^(2/3) (1.0: the "
                         "library's default)")
    ap.add_argument("--kkr-cells", default="both", choices=["both", "l12", "fcc1"],
                    help="kkr mode: the L1_2 4-site cell, the primitive fcc cell, or both")
    ap.add_argument("--sc-parts", type=int, default=1,
                    help="supercell: split the batch into this many cost-balanced parts, each a captured plan "
                         "with its own workspace replayed on its own stream (independent chunks in flight)")
    ap.add_argument("--chunk-lizs", type=int, default=2,
                    help="supercell: workspace for this many LIZs per launch (more LIZs share launches; "
                         "2 measured 5%% faster than 1, 4 no faster than 2)")
    ap.add_argument("--train-lizs", type=int, default=1667,
                    help="warmstart mode: random 135-site training LIZs (x 2 spins x 15 predicted points; "
                         "1667 LIZs give 50k training samples)")
    ap.add_argument("--shard", default="slices", choices=["slices", "balanced"],
                    help="supercell mode under torchrun: every rank its own n-lizs LIZs (weak scaling), or the "
                         "first n-lizs LIZs split over the ranks by the cost sum n^3 (shard.py, strong scaling)")
    ap.add_argument("--autotune", action="store_true",
                    help="supercell mode: grid-search the library's knobs on the batch first (autotune.py)")
    ap.add_argument("--tune", action="append", default=[], metavar="KNOB=VALUE",
                    help="set a library knob (must_tune_set) before the run; recorded in the JSON line")
    ap.add_argument("--n-energies", type=int, default=32,
                    help="contour energies per step (32 = the benchmark workload; fewer for ncu captures)")
    args = ap.parse_args()
    if args.tune and args.impl != "reference":
        from paper_2308_16317_gb300 import binding as B
        B.load()
        for kv in args.tune:
            k, v = (int(x) for x in kv.split("="))
            B.must_tune_set(k, v)   # raises if the library rejects it
            TUNE[k] = v
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "supercell":
        run_supercell(args)
    elif args.workload == "warmstart":
        run_warmstart(args)
    elif args.workload == "cusolver":
        run_cusolver_context(args)
    elif args.workload == "canted":
        run_canted(args)
    elif args.workload == "paper":
        run_paper_shapes(args)
    elif args.workload == "charge":
        run_site_charge(args)
    elif args.workload == "peaks":
        run_peaks(args)
    elif args.workload == "kkr":
        run_kkr(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
