"""Host logic of the solve server (serve.Server) on CPU, with the device
solver and batch engine replaced by fakes: admission by the memory budget in
arrival order, reuse of pooled hierarchies of the same size, eviction of idle
hierarchies (largest first) when a new size needs room, byte accounting, and
rejection of a request whose hierarchy alone exceeds the budget (it could
never start). The arena sizes come from the real mg_workspace_bytes.
"""
import numpy as np
import pytest

from paper_1406_5369_gb300 import serve


class FakeSolver:
    created = []

    def __init__(self, dim, n, maxit=60, **params):
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

    def __init__(self, max_active):
        self.max_active = max_active
        self.live = {}
        self.next = 0

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
    srv = server(1.0)
    b65 = srv._bytes(2, 65)
    srv.budget = 2.5 * b65
    assert srv.admit(req(0, 2, 65)) and srv.admit(req(1, 2, 65))
    assert not srv.admit(req(2, 2, 65))  # a third would exceed the budget
    assert srv.used == 2 * b65
    done = []
    srv.step(lambda: 1.0, done)  # 1e-2: not yet
    srv.step(lambda: 2.0, done)  # 1e-4
    srv.step(lambda: 3.0, done)  # 1e-6 <= tol: both retire to the pool
    assert len(done) == 2 and not srv.active and srv.used == 2 * b65
    n_created = len(FakeSolver.created)
    assert srv.admit(req(2, 2, 65))  # reuses a pooled hierarchy
    assert len(FakeSolver.created) == n_created and srv.used == 2 * b65
    # a larger size evicts the idle pooled one (the only idle hierarchy) first
    b129 = srv._bytes(2, 129)
    srv.budget = b65 + b129
    assert srv.admit(req(3, 2, 129))
    assert srv.used == b65 + b129 and FakeSolver.created[-1].n == 129
    assert sum(s.closed for s in FakeSolver.created) == 1
    assert srv.peak_used >= srv.used


def test_run_serves_everything_and_rejects_what_can_never_fit(server):
    srv = server(1.0)
    srv.budget = 3 * srv._bytes(2, 129)
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
