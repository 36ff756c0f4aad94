"""The server's admission and retirement logic on the host, with a stand-in
for the library (no GPU): requests are admitted first come, first served
while the HBM budget and the slots allow, never above either, each retires
once its solve reports completion, and a request larger than the whole
budget is refused up front."""
import numpy as np
import pytest

from paper_2008_02710_gb300 import serve, synth


class FakeChain:
    """Completes after `polls` queries; records the live contexts."""
    live = 0
    peak = 0
    order = []

    def __init__(self, csr, precision="mixed"):
        self.csr = csr
        self.polls = 1 + csr.n % 4
        FakeChain.live += 1
        FakeChain.peak = max(FakeChain.peak, FakeChain.live)
        FakeChain.order.append(csr.n)

    def set_params(self, **kw):
        assert kw.get("persistent") == 0  # solves share the GPU

    def solve_async(self, schedule, theta, tol, max_steps):
        self.tol = tol

    def query(self):
        self.polls -= 1
        return self.polls <= 0

    def wait(self, raise_on_noconv=True):
        return {"status": "RLGL_OK", "moves": 3, "edges_pushed": 7 * self.csr.n}

    def estimate(self):
        return np.full(self.csr.n, 1.0 / self.csr.n)

    def close(self):
        FakeChain.live -= 1


@pytest.fixture
def fake(monkeypatch):
    FakeChain.live = FakeChain.peak = 0
    FakeChain.order = []
    monkeypatch.setattr(serve.rlgl, "load", lambda *a, **k: None)
    monkeypatch.setattr(serve.rlgl, "Chain", FakeChain)
    monkeypatch.setattr(serve.rlgl, "release_retired", lambda: None)
    # footprint: 1000 bytes per node
    monkeypatch.setattr(serve.rlgl, "footprint", lambda n, nnz, weighted, precision: 1000 * n)
    return FakeChain


def _req(i, n, arrival):
    csr = synth.CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), None)
    return serve.Request(i, arrival, csr, 1e-6)


def test_budget_and_slots_are_never_exceeded(fake):
    sizes = [50, 300, 120, 700, 90, 410, 60, 250, 330, 80, 500, 40]
    reqs = [_req(i, n, 0.0) for i, n in enumerate(sizes)]
    srv = serve.Server(hbm_budget_bytes=1000 * 1000, max_active=3)
    res = srv.run(reqs, realtime=False)
    assert sorted(r.id for r in res) == list(range(len(sizes)))
    assert all(r.status == "RLGL_OK" and r.pi is not None for r in res)
    assert srv.stats["max_used_bytes"] <= 1000 * 1000
    assert srv.stats["max_active"] <= 3 and fake.peak <= 3
    assert fake.live == 0
    # first come, first served: admission follows arrival (here: id) order
    assert fake.order == sizes


def test_arrivals_in_time_order_and_latencies(fake):
    reqs = [_req(i, 10 + i, 0.002 * i) for i in range(8)]
    srv = serve.Server(hbm_budget_bytes=1e9, max_active=32)
    res = srv.run(reqs, realtime=True)
    by_id = {r.id: r for r in res}
    for i in range(8):
        assert by_id[i].start >= by_id[i].arrival - 1e-9
        assert by_id[i].finish >= by_id[i].start
    s = serve.summary(res)
    assert s["requests"] == 8 and s["not_ok"] == 0 and s["p99_s"] >= s["p50_s"]


def test_request_above_the_whole_budget_is_refused(fake):
    srv = serve.Server(hbm_budget_bytes=1000 * 100)
    with pytest.raises(ValueError):
        srv.run([_req(0, 101, 0.0)], realtime=False)


class FakeBatch:
    """A batch context stand-in: completes after two queries."""
    made = []

    def __init__(self, csr, precision="mixed", node_ptr=None):
        self.csr = csr
        self.k = 1 if node_ptr is None else len(node_ptr) - 1
        self.polls = 2
        FakeBatch.made.append(self.k)

    def set_params(self, **kw):
        pass

    def set_chain_tol(self, tol):
        assert len(tol) == self.k

    def solve_async(self, schedule, theta, tol, max_steps):
        pass

    def query(self):
        self.polls -= 1
        return self.polls <= 0

    def wait(self, raise_on_noconv=True):
        return {"status": "RLGL_OK", "moves": 4, "edges_pushed": 0}

    def chains(self):
        return np.zeros(self.k, np.int32), np.full(self.k, 4, np.int64), np.zeros(self.k)

    def estimate(self):
        return np.ones(self.csr.n)

    def close(self):
        pass


def test_batch_server_budget_cap_and_batches(monkeypatch):
    FakeBatch.made = []
    monkeypatch.setattr(serve.rlgl, "load", lambda *a, **k: None)
    monkeypatch.setattr(serve.rlgl, "Chain", FakeBatch)
    monkeypatch.setattr(serve.rlgl, "release_retired", lambda: None)
    monkeypatch.setattr(serve.rlgl, "footprint", lambda n, nnz, weighted, precision: 1000 * n)
    sizes = [50, 300, 120, 700, 90, 410, 60, 250, 330, 80, 500, 40]
    reqs = [_req(i, n, 0.0) for i, n in enumerate(sizes)]
    srv = serve.BatchServer(hbm_budget_bytes=1000 * 1000, max_chains=4, alone_nodes=600)
    res = srv.run(reqs, realtime=False)
    assert sorted(r.id for r in res) == list(range(len(sizes)))
    assert all(r.status == "RLGL_OK" and len(r.pi) == sizes[r.id] for r in res)
    assert srv.stats["max_used_bytes"] <= 1000 * 1000 and srv.stats["max_chains"] <= 4
    # the oldest request decides: a large one (>= 600 nodes) runs alone; a
    # small one opens a batch of every queued small request that fits the
    # budget (1000 nodes) and the cap (4 chains), in arrival order
    assert FakeBatch.made == [4, 1, 4, 3]
    assert srv.stats["batches"] == 3 and srv.stats["alone"] == 1
    # a batch's requests retire together; the large request retires alone
    fin = {}
    for r in res:
        fin.setdefault(r.finish, []).append(sizes[r.id])
    assert sorted(sorted(v) for v in fin.values()) == [[40, 330, 500], [50, 90, 120, 300], [60, 80, 250, 410],
                                                        [700]]
