"""Autotuner for the batched tau_00 path.

Times every combination of the library's tuning knobs (must_tune_set) on a
sample batch and keeps the fastest, caching the choice in a JSON file keyed
by GPU, precision and workload shape so later runs apply it without
re-measuring.  Knobs:
  bucket_sites  sites per padding quantum when LIZs of uneven size are
                grouped into shared launches (padding costs flops, finer
                quanta cost launches);
  tile_n        complex columns per tensor-core tile of the trailing update;
  run_tiles     longest run of row tiles per CTA of the streamed update;
  cluster_ctas  CTAs per cluster of the correction solve.
"""
from __future__ import annotations

import itertools
import json
import os

KNOBS = {"bucket_sites": 0, "tile_n": 1, "run_tiles": 3, "cluster_ctas": 7}
CANDIDATES = {"bucket_sites": [1, 2, 4, 8], "tile_n": [128, 256], "run_tiles": [16, 32, 64], "cluster_ctas": [2, 4]}


def search(run, set_knob, candidates=None, reps: int = 2):
    """Grid search: for each combination, set the knobs, run once to warm up,
    then `reps` timed runs (run() returns milliseconds).  Returns
    (best_setting, [(setting, ms), ...])."""
    candidates = candidates or CANDIDATES
    names = sorted(candidates)
    results = []
    for combo in itertools.product(*(candidates[k] for k in names)):
        setting = dict(zip(names, combo))
        for k, v in setting.items():
            set_knob(KNOBS[k], v)
        run()
        ms = min(run() for _ in range(max(1, reps)))
        results.append((setting, ms))
    best = min(results, key=lambda x: x[1])[0]
    for k, v in best.items():
        set_knob(KNOBS[k], v)
    return best, results


def cache_key(gpu: str, precision: int, lmax: int, n_max: int, items: int) -> str:
    return "%s|prec%d|lmax%d|nmax%d|items%d" % (gpu, precision, lmax, n_max, items)


def load(path: str) -> dict:
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save(path: str, key: str, best: dict, results) -> None:
    data = load(path)
    data[key] = {"best": best, "measured_ms": [[s, ms] for s, ms in results]}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(path: str, key: str, set_knob) -> bool:
    entry = load(path).get(key)
    if not entry:
        return False
    for k, v in entry["best"].items():
        set_knob(KNOBS[k], v)
    return True


def tune_session(session, opts, cache_path: str | None = None, reps: int = 2, candidates=None,
                 workspace_lizs: int = 2):
    """Tune the knobs for the batched call on `session`'s LIZs: each setting
    is captured into a plan (must_plan_batch, the way a batch is run) and its
    replays are timed with CUDA events on the device, so host launch cost does
    not bias the choice; reuses a cached choice for the same key if present."""
    import torch

    from . import binding as B
    items = len(session.w.energies) * (1 if session.w.canted else session.nspin)
    n_max = max(z.n for z in session.lizs)
    key = cache_key(torch.cuda.get_device_name(), int(opts.precision) if opts else 0, session.w.lmax, n_max,
                    items * len(session.lizs))
    if cache_path and apply(cache_path, key, B.must_tune_set):
        return load(cache_path)[key]["best"], None
    tau, st = session.alloc_out(len(session.lizs))
    nbytes = B.must_batch_workspace_bytes(session.lizs, items, opts) * max(1, workspace_lizs)
    ws = session.workspace(nbytes)

    state = {"plan": None}

    def set_knob(k, v):
        B.must_tune_set(k, v)
        state["plan"] = None       # the next run captures a plan with the new setting

    def run():
        if state["plan"] is None:
            state["plan"] = B.must_plan_batch(session.lizs, session.E, session.tinv, session.n_species,
                                              session.nspin, opts, ws, nbytes, tau, st)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        B.must_plan_launch(state["plan"])
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    best, results = search(run, set_knob, candidates, reps)
    state["plan"] = None
    if cache_path:
        save(cache_path, key, best, results)
    return best, results
