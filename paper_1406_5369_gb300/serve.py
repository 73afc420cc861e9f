"""Continuous-batching solve server (host loop around the batch engine).

Requests (dim, n, tolerance, seed, arrival time) are admitted while the
device memory they need fits a budget, in arrival order. Each admitted
request gets a grid hierarchy resident on the device - reused from a pool
of idle hierarchies of the same size when one exists - and joins the 2D or
3D batch. Every loop iteration runs one batched solve step (a defect-
correction step: inner FP32 V-cycles and the FP64 outer update) for all
active requests of each batch, so requests that arrive while others are on
the GPU join at the next step and same-size levels of all requests run in
the same launches; requests whose relative residual reached their
tolerance retire, freeing their slot (the hierarchy goes back to the pool).

Latency = completion time - arrival time, on the host clock.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from .batch import BatchSolver
from .solver import Solver

# Per-dimension solver settings. 3 inner V-cycles per outer step and BF16
# storage for the 3D inner cycles measured fastest on the serving mix
# (838 vs 749 solves/s against 2 inner cycles and FP32 storage everywhere);
# every request still reaches its tolerance by the FP64 outer residual.
DEFAULT_PARAMS = {
    2: dict(smoother="rbgs", omega=1.0, nu1=2, nu2=1, precision="fp32_dc", inner_cycles=3),
    3: dict(smoother="jacobi", omega=6.0 / 7.0, nu1=2, nu2=2, precision="bf16_dc", inner_cycles=3),
}


class Server:
    def __init__(self, budget_bytes=150e9, max_active=2048, params=None, maxit=60, device="cuda"):
        self.budget = float(budget_bytes)
        self.params = {d: dict(DEFAULT_PARAMS[d], **((params or {}).get(d, {}))) for d in (2, 3)}
        self.maxit = maxit
        self.device = device
        self.max_active = int(max_active)
        self.batches = {d: BatchSolver(self.max_active) for d in (2, 3)}
        self.pool = collections.defaultdict(list)  # (dim, n) -> idle Solvers
        self.used = 0.0                            # bytes of every live hierarchy (active + pooled)
        self.active = {}                           # request id -> dict
        self.peak_used = 0.0
        self.steps = 0

    # ---- memory
    def _bytes(self, dim, n):
        from . import _capi as C
        import ctypes
        lib = C.load()
        p = self.params[dim]
        o = C.mg_options()
        lib.mg_default_options(ctypes.byref(o))
        o.smoother = 0 if p["smoother"] == "rbgs" else 1
        o.precision = {"fp64": 0, "fp32_dc": 1, "bf16_dc": 2}[p["precision"]]
        return float(lib.mg_workspace_bytes(dim, n, 0, ctypes.byref(o)))

    def _evict_for(self, need):
        # drop idle pooled hierarchies (largest first) until `need` bytes fit
        while self.used + need > self.budget:
            keys = [k for k, v in self.pool.items() if v]
            if not keys:
                return False
            k = max(keys, key=lambda kk: kk[1])
            s = self.pool[k].pop()
            self.used -= s.workspace_bytes
            s.close()
            del s
        return True

    def _acquire(self, dim, n):
        key = (dim, n)
        if self.pool[key]:
            return self.pool[key].pop(), False
        need = self._bytes(dim, n)
        if not self._evict_for(need):
            return None, False
        s = Solver(dim, n, maxit=self.maxit, **self.params[dim])
        self.used += s.workspace_bytes
        self.peak_used = max(self.peak_used, self.used)
        return s, True

    # ---- requests
    def _members(self, dim):
        return sum(1 for a in self.active.values() if a["req"]["dim"] == dim)

    def admit(self, req):
        """Returns True if the request got a hierarchy and joined its batch;
        False (the request keeps waiting) while its batch has no free slot or
        its hierarchy does not fit the memory budget."""
        import synth
        dim = req["dim"]
        if self._members(dim) >= self.max_active:
            return False
        s, _ = self._acquire(dim, req["n"])
        if s is None:
            return False
        try:
            f = synth.torch_uniform_rhs(dim, req["n"], req["seed"], device=self.device)
            s.set_rhs(f)
            s.set_solution(None)
            del f
            pid = self.batches[dim].add(s)
        except Exception:
            # the hierarchy goes back to the pool (still counted in self.used)
            self.pool[(dim, req["n"])].append(s)
            return False
        self.active[req["id"]] = {"req": req, "solver": s, "pid": pid, "steps": 0}
        return True

    def _retire(self, rid, now, done, keep_solution):
        a = self.active.pop(rid)
        d = a["req"]["dim"]
        self.batches[d].remove(a["pid"])
        rec = {"id": rid, "latency": now - a["req"]["t"], "steps": a["steps"], "relres": a["rho"],
               "dim": d, "n": a["req"]["n"], "tol": a["req"]["tol"]}
        if keep_solution:
            rec["u"] = a["solver"].get_solution()
        self.pool[(d, a["req"]["n"])].append(a["solver"])
        done.append(rec)

    def step(self, now_fn, done, keep_solutions=False):
        """One batched solve step for every active request; retires the converged."""
        for d in (2, 3):
            ids = [(rid, a["pid"]) for rid, a in self.active.items() if a["req"]["dim"] == d]
            if not ids:
                continue
            rho = self.batches[d].step([p for _, p in ids])
            now = now_fn()
            for (rid, _), r in zip(ids, rho):
                a = self.active[rid]
                a["steps"] += 1
                a["rho"] = float(r)
                if not (r > a["req"]["tol"]) or a["steps"] >= self.maxit:
                    self._retire(rid, now, done, keep_solutions)
        self.steps += 1

    def run(self, requests, keep_solutions=False, max_wall=None):
        """Serves a list of requests with arrival times req['t'] (seconds from
        the start). Returns (completed records, stats)."""
        pending = collections.deque(sorted(requests, key=lambda r: r["t"]))
        waiting = collections.deque()
        done = []
        rejected = []  # requests whose hierarchy alone exceeds the budget: they could never start
        t0 = time.perf_counter()
        now_fn = lambda: time.perf_counter() - t0  # noqa: E731
        queue_depth = []
        while pending or waiting or self.active:
            now = now_fn()
            if max_wall is not None and now > max_wall:
                break
            while pending and pending[0]["t"] <= now:
                req = pending.popleft()
                if self._bytes(req["dim"], req["n"]) > self.budget:
                    rejected.append(req["id"])
                else:
                    waiting.append(req)
            while waiting and self.admit(waiting[0]):
                waiting.popleft()
            queue_depth.append(len(waiting))
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(0.001, pending[0]["t"] - now_fn())))
                continue
            self.step(now_fn, done, keep_solutions)
        wall = now_fn()
        lat = np.array([d["latency"] for d in done]) if done else np.zeros(1)
        stats = {"completed": len(done), "submitted": len(requests), "wall_s": wall,
                 "solves_per_s": len(done) / wall if wall > 0 else 0.0,
                 "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "mean_ms": 1e3 * float(lat.mean()), "steps": self.steps,
                 "peak_hbm_gb": self.peak_used / 1e9, "max_queue_depth": int(max(queue_depth) if queue_depth else 0),
                 "unfinished": len(self.active) + len(waiting) + len(pending), "rejected": len(rejected)}
        return done, stats
