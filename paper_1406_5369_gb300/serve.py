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
The 2D and the 3D batch run on streams of their own: both steps are
enqueued (mg_batch_step_async), requests that have arrived meanwhile are
admitted while the GPU runs them, and only then does the loop wait for the
two steps' norms.

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


def _new_stream(device):
    """A stream of its own for one batch (None on a host without CUDA)."""
    try:
        import torch
        if device == "cuda" and torch.cuda.is_available():
            st = torch.cuda.Stream()
            return st.cuda_stream
    except ImportError:
        pass
    return None


class _RHSGraphs:
    """Each request's right-hand side (synth.torch_uniform_rhs, drawn on the
    device from the request's seed) through one CUDA graph per grid size: the
    generator's dozen torch operations are captured once, with the seed read
    from a device scalar, and every later request of that size is one graph
    replay into a fixed buffer instead of a dozen launches and allocations
    (the host's cost per request bounded the server's throughput). The values
    are bit-identical to the uncaptured generator's."""

    def __init__(self, device):
        self.device = device
        self.graphs = {}

    def draw(self, dim, n, seed):
        import torch
        import synth
        key = (dim, n)
        if key not in self.graphs:
            seed_t = torch.zeros((), dtype=torch.int64, device=self.device)
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):  # warm-up outside the capture
                synth.torch_uniform_rhs(dim, n, seed_t, device=self.device)
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                out = synth.torch_uniform_rhs(dim, n, seed_t, device=self.device)
            self.graphs[key] = (g, seed_t, out)
        g, seed_t, out = self.graphs[key]
        seed_t.fill_(synth.torch_seed(seed))
        g.replay()
        return out


class SlabAllocator:
    """Offsets into one device slab of `total` bytes for the hierarchies'
    arenas: best fit over a free list kept in address order, split on
    allocation, merged with free neighbours on release; every block starts on
    an `align`-byte boundary. The server allocates its whole memory budget
    once, so that admitting or evicting a hierarchy never allocates or frees
    device memory (a device free waits for every queued kernel)."""

    def __init__(self, total, align=256):
        self.align = int(align)
        self.total = int(total) // self.align * self.align
        self.free_list = [(0, self.total)] if self.total > 0 else []  # (offset, size), address order
        self.used = 0

    def _round(self, n):
        return (int(n) + self.align - 1) // self.align * self.align

    def alloc(self, nbytes):
        """Offset of a block of at least nbytes, or None if no free block fits."""
        need = self._round(nbytes)
        best = None
        for i, (off, size) in enumerate(self.free_list):
            if size >= need and (best is None or size < self.free_list[best][1]):
                best = i
        if best is None:
            return None
        off, size = self.free_list[best]
        if size == need:
            del self.free_list[best]
        else:
            self.free_list[best] = (off + need, size - need)
        self.used += need
        return off

    def free(self, off, nbytes):
        size = self._round(nbytes)
        fl = self.free_list
        lo, hi = 0, len(fl)
        while lo < hi:  # first free block above off
            mid = (lo + hi) // 2
            if fl[mid][0] < off:
                lo = mid + 1
            else:
                hi = mid
        if lo < len(fl) and off + size > fl[lo][0] or lo > 0 and fl[lo - 1][0] + fl[lo - 1][1] > off:
            raise ValueError("block overlaps a free block")
        fl.insert(lo, (off, size))
        if lo + 1 < len(fl) and off + size == fl[lo + 1][0]:  # merge with the next
            fl[lo] = (off, size + fl[lo + 1][1])
            del fl[lo + 1]
        if lo > 0 and fl[lo - 1][0] + fl[lo - 1][1] == off:  # merge with the previous
            fl[lo - 1] = (fl[lo - 1][0], fl[lo - 1][1] + fl[lo][1])
            del fl[lo]
        self.used -= size

    def largest_free(self):
        return max((sz for _, sz in self.free_list), default=0)

    def merged_size(self, off, nbytes):
        """Size of the free block that releasing (off, nbytes) would leave:
        the block plus the free blocks directly before and after it."""
        size = self._round(nbytes)
        total = size
        for foff, fsz in self.free_list:
            if foff + fsz == off or foff == off + size:
                total += fsz
        return total


class Server:
    def __init__(self, budget_bytes=150e9, max_active=2048, params=None, maxit=60, device="cuda"):
        self.budget = float(budget_bytes)
        self.params = {d: dict(DEFAULT_PARAMS[d], **((params or {}).get(d, {}))) for d in (2, 3)}
        self.maxit = maxit
        self.device = device
        self.max_active = int(max_active)
        self.streams = {d: _new_stream(device) for d in (2, 3)}
        self.batches = {d: BatchSolver(self.max_active, stream=self.streams[d]) for d in (2, 3)}
        self.pool = collections.defaultdict(list)  # (dim, n) -> idle Solvers
        self._sizes = {}                           # (dim, n) -> workspace bytes
        self._rhs = _RHSGraphs(device) if device == "cuda" else None
        self.freed = 0                             # retirements so far (admission retries wait for one)
        self.used = 0.0                            # bytes of every live hierarchy (active + pooled)
        self.slab_alloc = SlabAllocator(self.budget)
        self.slab = None                           # the device slab (allocated at the first admission)
        self.active = {}                           # request id -> dict
        self.peak_used = 0.0
        self.steps = 0

    # ---- memory
    def _bytes(self, dim, n):
        key = (dim, n)
        if key not in self._sizes:
            self._sizes[key] = self._workspace(dim, n)
        return self._sizes[key]

    def _workspace(self, dim, n):
        from . import _capi as C
        import ctypes
        lib = C.load()
        p = self.params[dim]
        o = C.mg_options()
        lib.mg_default_options(ctypes.byref(o))
        o.smoother = 0 if p["smoother"] == "rbgs" else 1
        o.precision = {"fp64": 0, "fp32_dc": 1, "bf16_dc": 2}[p["precision"]]
        return float(lib.mg_workspace_bytes(dim, n, 0, ctypes.byref(o)))

    def _drop(self, s):
        self.used -= s.workspace_bytes
        self.slab_alloc.free(s._slab_off, s.workspace_bytes)
        s.close()

    def _place(self, need):
        # a slab block for `need` bytes; while none fits, drop the idle pooled
        # hierarchy whose release leaves the largest free block (the larger
        # hierarchy on ties)
        while True:
            off = self.slab_alloc.alloc(need)
            if off is not None:
                return off
            idle = [(k, i, s) for k, v in self.pool.items() for i, s in enumerate(v)]
            if not idle:
                return None
            k, i, s = max(idle, key=lambda t: (self.slab_alloc.merged_size(t[2]._slab_off, t[2].workspace_bytes),
                                               t[2].workspace_bytes))
            self._drop(self.pool[k].pop(i))

    def _acquire(self, dim, n):
        key = (dim, n)
        if self.pool[key]:
            return self.pool[key].pop(), False
        need = self._bytes(dim, n)
        if need > self.slab_alloc.total:
            return None, False
        off = self._place(need)
        if off is None:
            return None, False
        arena = None
        if self.device == "cuda":
            import torch
            if self.slab is None:
                self.slab = torch.empty(self.slab_alloc.total, dtype=torch.uint8, device=self.device)
            arena = self.slab[off:off + int(need)]
        s = Solver(dim, n, maxit=self.maxit, arena=arena, **self.params[dim])
        s._slab_off = off
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
            if self._rhs is not None:
                f = self._rhs.draw(dim, req["n"], req["seed"])
            else:
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
               "dim": d, "n": a["req"]["n"], "tol": a["req"]["tol"], "t": a["req"]["t"], "done_at": now}
        if keep_solution:
            rec["u"] = a["solver"].get_solution()
        self.pool[(d, a["req"]["n"])].append(a["solver"])
        self.freed += 1
        done.append(rec)

    def step(self, now_fn, done, keep_solutions=False, meanwhile=None):
        """One batched solve step for every active request; retires the
        converged. Both batches' steps are enqueued first; `meanwhile` (e.g.
        admission of new arrivals) runs on the host while the GPU works."""
        launched = {}
        for d in (2, 3):
            ids = [(rid, a["pid"]) for rid, a in self.active.items() if a["req"]["dim"] == d]
            if ids:
                self.batches[d].step_async([p for _, p in ids])
                launched[d] = ids
        if meanwhile is not None:
            meanwhile()
        for d, ids in launched.items():
            rho = self.batches[d].step_wait()
            now = now_fn()
            for (rid, _), r in zip(ids, rho):
                a = self.active[rid]
                a["steps"] += 1
                a["rho"] = float(r)
                if not (r > a["req"]["tol"]) or a["steps"] >= self.maxit:
                    self._retire(rid, now, done, keep_solutions)
        self.steps += 1

    def run(self, requests, keep_solutions=False, max_wall=None, window=None):
        """Serves a list of requests with arrival times req['t'] (seconds from
        the start). Returns (completed records, stats). window = (t0, t1):
        the statistics cover requests arriving in [t0, t1) (latency) and
        completions in [t0, t1) (solves/s); the earlier ones warm the server
        up. None: every request, over the whole run."""
        pending = collections.deque(sorted(requests, key=lambda r: r["t"]))
        waiting = collections.deque()
        done = []
        rejected = []  # requests whose hierarchy alone exceeds the budget: they could never start
        t0 = time.perf_counter()
        now_fn = lambda: time.perf_counter() - t0  # noqa: E731
        queue_depth = []

        blocked_at = [-1]  # self.freed when the head of the queue last failed to get in

        def arrivals():
            now = now_fn()
            while pending and pending[0]["t"] <= now:
                req = pending.popleft()
                if self._bytes(req["dim"], req["n"]) > self.slab_alloc.total:
                    rejected.append(req["id"])
                else:
                    waiting.append(req)
            # a request that did not fit is retried only after a retirement
            # (memory and slots are freed by nothing else)
            if waiting and blocked_at[0] != self.freed:
                while waiting and self.admit(waiting[0]):
                    waiting.popleft()
                blocked_at[0] = self.freed if waiting else -1
            queue_depth.append(len(waiting))

        while pending or waiting or self.active:
            if max_wall is not None and now_fn() > max_wall:
                break
            if not self.active:
                blocked_at[0] = -1  # nothing runs: the head of the queue is tried again
                arrivals()
                if not self.active:
                    if waiting:
                        # nothing runs and every idle hierarchy could be dropped,
                        # so a request that still cannot be placed never will be
                        rejected.append(waiting.popleft()["id"])
                    elif pending:
                        time.sleep(max(0.0, min(0.001, pending[0]["t"] - now_fn())))
                    continue
            # arrivals are admitted while the step runs (they join the next one)
            self.step(now_fn, done, keep_solutions, meanwhile=arrivals)
        wall = now_fn()
        if window is None:
            w0, w1 = 0.0, wall
            sel = done
            finished = len(done)
        else:
            w0, w1 = window
            sel = [d for d in done if w0 <= d["t"] < w1]
            finished = sum(1 for d in done if w0 <= d["done_at"] < w1)
        lat = np.array([d["latency"] for d in sel]) if sel else np.zeros(1)
        span = max(min(w1, wall) - w0, 1e-9)
        stats = {"completed": len(done), "submitted": len(requests), "wall_s": wall,
                 "solves_per_s": finished / span,
                 "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                 "mean_ms": 1e3 * float(lat.mean()), "steps": self.steps,
                 "window_s": [w0, w1], "completed_in_window": finished, "latency_samples": len(sel),
                 "peak_hbm_gb": self.peak_used / 1e9, "max_queue_depth": int(max(queue_depth) if queue_depth else 0),
                 "unfinished": len(self.active) + len(waiting) + len(pending), "rejected": len(rejected)}
        return done, stats
