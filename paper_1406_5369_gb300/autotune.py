"""Autotuner for solver settings that change speed but not the answer's tolerance.

Each tunable is a keyword of Solver (e.g. inner_cycles: inner V-cycles per
outer FP64 step of defect correction). tune() builds one solver per
candidate setting, times solves of the caller's problem to the caller's
tolerance with CUDA events, and keeps the fastest. Results are cached per
GPU model and problem signature in _build/autotune.json beside the library,
so a tuned configuration is measured once per machine.
"""
from __future__ import annotations

import json
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(_HERE, "_build", "autotune.json")
_lock = threading.Lock()


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(db):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def signature(dim, n, **params):
    items = ",".join(f"{k}={params[k]}" for k in sorted(params))
    return f"{_gpu_name()}|dim={dim}|n={n}|{items}"


def time_solve(solver, f, tol, reps=3, stat="median"):
    """Milliseconds of `reps` solves from zero (after one warm-up solve): their
    median, or with stat="min" the fastest, the candidate's cost when nothing
    else holds the GPU (the tuner's choice, so that one disturbed solve on a
    shared machine cannot decide it)."""
    import torch
    solver.set_rhs(f)
    solver.set_solution(None)
    solver.solve(tol)
    times = []
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        solver.set_solution(None)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it, rr, _ = solver.solve(tol)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    if stat == "min":
        return times[0], it
    m = len(times) // 2
    return (times[m] if len(times) % 2 else 0.5 * (times[m - 1] + times[m])), it


def tune(dim, n, f, tol, knobs, base=None, reps=3, use_cache=True):
    """Returns (best settings dict, table of {setting: ms}).

    knobs: {name: [candidate values]} searched one knob at a time (each knob
    is tuned with the others at their best value so far); base: fixed Solver
    keywords (precision, smoother, ...), part of the cache key.
    """
    from .solver import Solver
    base = dict(base or {})
    sig = signature(dim, n, tol=tol, **base)
    with _lock:
        db = _load() if use_cache else {}
    if use_cache and sig in db and all(k in db[sig]["best"] for k in knobs):
        return db[sig]["best"], db[sig]["table"]
    best = {k: v[0] for k, v in knobs.items()}
    table = {}
    for name, values in knobs.items():
        results = {}
        for v in values:
            trial = dict(best, **{name: v})
            s = Solver(dim, n, **base, **trial)
            ms, it = time_solve(s, f, tol, reps, stat="min")
            s.close()
            del s
            results[v] = ms
            table[json.dumps(trial, sort_keys=True)] = {"ms": ms, "iterations": it}
        best[name] = min(results, key=results.get)
    if use_cache:
        with _lock:
            db = _load()
            db[sig] = {"best": best, "table": table}
            _store(db)
    return best, table


def lfa_choice(dim, c=(1.0, 1.0, 1.0), tol=1e-10, smoothers=("rbgs", "jacobi"), omegas=None, nus=None,
               grid="node"):
    """The configuration (smoother, omega, nu1, nu2) that local Fourier
    analysis predicts to reach `tol` with the least operator-model traffic
    (lfa.choose); the rest of the ranking is returned under "ranking".
    Host-side only: the prediction replaces timing for the discrete choices
    the feature model leaves open (Sec. 2.3, Sec. 5)."""
    from . import lfa
    ranked = lfa.choose(dim, c=c, tol=tol, smoothers=smoothers, omegas=omegas, nus=nus, grid=grid)
    if not ranked:
        raise ValueError("no candidate converges according to LFA")
    best = dict(ranked[0])
    best["ranking"] = ranked
    return best
