"""Host logic of the solve server (serve.Server) on CPU, with the device
solver and batch engine replaced by fakes: admission by the memory budget in
arrival order, reuse of pooled hierarchies of the same size, the slab
allocator that places arenas in the budget (best fit, coalescing), eviction of
the idle hierarchy whose release opens the largest free block when a new size
needs room, byte accounting, and rejection of a request whose hierarchy alone
exceeds the budget (it could never start). The arena sizes come from the real
mg_workspace_bytes.
"""
import numpy as np
import pytest

from paper_1406_5369_gb300 import serve


class FakeSolver:
    created = []

    def __init__(self, dim, n, maxit=60, arena=None, **params):
        self.dim, self.n = dim, n
        self.workspace_bytes = FakeSolver.bytes_of(dim, n)
        self.closed = False
        FakeSolver.created.append(self)

    bytes_of = None

    def set_rhs(self, f):
        pass

    def set_solution(self, u=None):
        pass

    def close(self):
        self.closed = True


class FakeBatch:
    fail_next_add = False

    def __init__(self, max_active, stream=None):
        self.max_active = max_active
        self.live = {}
        self.next = 0
        self.inflight = None

    def add(self, s):
        # like mg_batch_add: MG_ENOMEM (raised by the binding) when every slot is taken
        if len(self.live) >= self.max_active or FakeBatch.fail_next_add:
            FakeBatch.fail_next_add = False
            raise RuntimeError("batch is full")
        self.next += 1
        self.live[self.next] = [s, 0]
        return self.next

    def remove(self, pid):
        del self.live[pid]

    def step(self, pids):
        # every problem gains a factor 100 per step
        out = []
        for p in pids:
            self.live[p][1] += 1
            out.append(10.0 ** (-2 * self.live[p][1]))
        return np.array(out)

    def step_async(self, pids):
        assert self.inflight is None, "one step in flight per batch"
        self.inflight = list(pids)

    def step_wait(self):
        pids, self.inflight = self.inflight, None
        return self.step(pids)


@pytest.fixture
def server(monkeypatch):
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    monkeypatch.setattr(serve, "BatchSolver", FakeBatch)
    import synth
    monkeypatch.setattr(synth, "torch_uniform_rhs", lambda dim, n, seed, device=None: None)
    FakeSolver.created = []

    def make(budget, max_active=2048):
        srv = serve.Server(budget_bytes=budget, max_active=max_active, device="cpu")
        FakeSolver.bytes_of = srv._bytes
        return srv
    return make


def req(i, dim, n, tol=1e-6, t=0.0):
    return {"id": i, "t": t, "dim": dim, "n": n, "tol": tol, "seed": i}


def test_budget_admission_pool_reuse_and_eviction(server):
    b65 = serve.Server(1.0, device="cpu")._bytes(2, 65)
    b129 = serve.Server(1.0, device="cpu")._bytes(2, 129)
    srv = server(b65 + b129)
    assert srv.admit(req(0, 2, 65)) and srv.admit(req(1, 2, 65))
    assert not srv.admit(req(3, 2, 129))  # does not fit beside them, nothing idle to drop
    assert srv.used == 2 * b65 and len(FakeSolver.created) == 2
    done = []
    srv.step(lambda: 1.0, done)  # 1e-2: not yet
    srv.step(lambda: 2.0, done)  # 1e-4
    srv.step(lambda: 3.0, done)  # 1e-6 <= tol: both retire to the pool
    assert len(done) == 2 and not srv.active and srv.used == 2 * b65
    assert srv.admit(req(2, 2, 65))  # reuses a pooled hierarchy
    assert len(FakeSolver.created) == 2 and srv.used == 2 * b65
    srv.step(lambda: 4.0, done)
    srv.step(lambda: 5.0, done)
    srv.step(lambda: 6.0, done)
    # a larger size drops idle pooled hierarchies until a block fits: the one
    # next to the free tail suffices, the other stays pooled
    assert srv.admit(req(3, 2, 129))
    assert srv.used == b65 + b129 and FakeSolver.created[-1].n == 129
    assert sum(s.closed for s in FakeSolver.created) == 1 and len(srv.pool[(2, 65)]) == 1
    assert srv.peak_used >= srv.used
    assert srv.slab_alloc.used == srv.slab_alloc._round(b65) + srv.slab_alloc._round(b129)


def test_slab_allocator_best_fit_coalescing_and_alignment():
    a = serve.SlabAllocator(10_000, align=256)
    assert a.total == 9984
    x = a.alloc(1000)   # 1024
    y = a.alloc(2000)   # 2048
    z = a.alloc(300)    # 512
    assert (x, y, z) == (0, 1024, 3072) and a.used == 3584
    assert a.alloc(7000) is None  # 6400 left at the end
    a.free(y, 2000)
    w = a.alloc(500)    # best fit: the 2048 hole, not the 6400 tail
    assert w == 1024
    a.free(w, 500)
    assert a.merged_size(z, 300) == 2048 + 512 + 6400  # free on both sides of z
    a.free(x, 1000)     # merges with the 2048 hole: [0, 3072)
    assert a.free_list[0] == (0, 3072)
    a.free(z, 300)      # everything merges back
    assert a.free_list == [(0, 9984)] and a.used == 0
    with pytest.raises(ValueError):
        a.free(0, 256)  # already free


def test_run_serves_everything_and_rejects_what_can_never_fit(server):
    srv = server(3 * serve.Server(1.0, device="cpu")._bytes(2, 129))
    reqs = [req(i, 2, 65 if i % 2 else 129, t=0.001 * i) for i in range(12)]
    reqs.append(req(99, 2, 4097))  # far above the budget
    done, stats = srv.run(reqs, max_wall=30.0)
    assert stats["completed"] == 12 and stats["rejected"] == 1 and stats["unfinished"] == 0
    assert sorted(d["id"] for d in done) == list(range(12))
    assert all(d["latency"] >= 0 and d["relres"] <= d["tol"] for d in done)
    assert stats["peak_hbm_gb"] * 1e9 <= srv.budget


def test_admission_waits_for_a_free_slot(server):
    """More requests than batch slots: the surplus waits (no exception, no
    leaked hierarchy) and is admitted as retiring requests free their slots."""
    srv = server(1e15, max_active=3)
    assert all(srv.admit(req(i, 2, 65)) for i in range(3))
    n_created, used = len(FakeSolver.created), srv.used
    assert not srv.admit(req(3, 2, 65))  # batch full: waits, takes no hierarchy
    assert len(FakeSolver.created) == n_created and srv.used == used
    assert srv.admit(req(4, 3, 33))  # the other dimension's batch has room
    reqs = [req(10 + i, 2, 65 if i % 2 else 129, t=0.0) for i in range(20)]
    srv2 = server(1e15, max_active=4)
    done, stats = srv2.run(reqs, max_wall=30.0)
    assert stats["completed"] == 20 and stats["unfinished"] == 0
    assert sorted(d["id"] for d in done) == [10 + i for i in range(20)]


def test_failed_batch_add_returns_the_hierarchy_to_the_pool(server):
    srv = server(1e15, max_active=8)
    FakeBatch.fail_next_add = True
    assert not srv.admit(req(0, 2, 65))
    assert srv.pool[(2, 65)] and not srv.active
    n_created = len(FakeSolver.created)
    assert srv.admit(req(0, 2, 65))  # retried: reuses the pooled hierarchy
    assert len(FakeSolver.created) == n_created and srv.used == srv._bytes(2, 65)


def test_requests_admitted_during_a_step_join_the_next(server):
    """Arrivals admitted while a step is in flight (the `meanwhile` hook) are
    not part of that step: they take their first step with the next one."""
    srv = server(1e15, max_active=8)
    assert srv.admit(req(0, 2, 65))
    done = []
    srv.step(lambda: 1.0, done, meanwhile=lambda: srv.admit(req(1, 3, 33)))
    assert srv.active[0]["steps"] == 1 and srv.active[1]["steps"] == 0
    srv.step(lambda: 2.0, done)
    assert srv.active[0]["steps"] == 2 and srv.active[1]["steps"] == 1


def test_statistics_window_excludes_warm_up_requests(server):
    srv = server(1e15, max_active=64)
    reqs = [req(i, 2, 65, t=0.0 if i < 5 else 0.05) for i in range(10)]
    done, stats = srv.run(reqs, max_wall=30.0, window=(0.04, 10.0))
    assert stats["completed"] == 10 and stats["latency_samples"] == 5
    assert all("done_at" in d and d["done_at"] >= d["t"] for d in done)


def test_a_request_that_can_never_be_placed_is_rejected_not_waited_on(server):
    """With nothing running, every idle hierarchy could be dropped; a request
    whose hierarchy still does not fit is rejected instead of waiting (the run
    must end)."""
    srv = server(3 * serve.Server(1.0, device="cpu")._bytes(2, 65))
    srv.slab_alloc.total = srv.slab_alloc.used = 0  # as if the budget had no room at all
    srv.slab_alloc.free_list = []
    done, stats = srv.run([req(0, 2, 65), req(1, 2, 65, t=0.01)], max_wall=10.0)
    assert stats["rejected"] == 2 and stats["completed"] == 0 and stats["wall_s"] < 5.0
