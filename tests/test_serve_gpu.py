"""Continuous-batching server: requests admitted under an HBM budget while
others run; each result equals the same request solved alone."""
import numpy as np
import pytest

from paper_2008_02710_gb300 import synth

pytestmark = pytest.mark.gpu


def _requests(k, seed=7):
    from paper_2008_02710_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(k):
        n = int(np.exp(rng.uniform(np.log(500), np.log(20000))))
        tol = float(rng.choice([1e-4, 1e-6, 1e-8]))
        reqs.append(Request(i, arrival=0.002 * i, csr=synth.rmat_chain_n(n, seed=100 + i), tol=tol))
    return reqs


def test_served_results_equal_alone_fp64():
    from paper_2008_02710_gb300 import rlgl
    from paper_2008_02710_gb300.serve import Server, summary
    reqs = _requests(24)
    # a budget that holds only a few chains at a time: later requests queue
    foot = sorted(rlgl.footprint(r.csr.n, r.csr.nnz, False, "fp64") for r in reqs)
    budget = sum(foot[-4:])
    srv = Server(budget, max_active=8, precision="fp64")
    res = srv.run(reqs, realtime=True)
    assert len(res) == len(reqs)
    assert srv.stats["max_used_bytes"] <= budget
    assert srv.stats["max_active"] >= 2          # solves overlapped on the device
    assert any(r.queue_wait > 0.0 for r in res)  # and some waited for memory
    s = summary(res)
    assert s["not_ok"] == 0 and s["p99_s"] >= s["p50_s"] > 0
    by_id = {r.id: r for r in res}
    for q in reqs:
        with rlgl.Chain(q.csr, precision="fp64") as ch:
            ch.set_params(theta_scale=0.5)
            info = ch.solve(q.schedule, 0.0, q.tol, q.max_steps)
            alone = ch.estimate()
        r = by_id[q.id]
        d = float(np.abs(r.pi - alone).sum())
        if r.moves == info["moves"]:
            assert d <= 1e-12, (q.id, d)
        else:  # the stop test fired a move apart (rounding at the tolerance)
            assert abs(r.moves - info["moves"]) <= 1 and d <= 10 * q.tol


def test_served_mixed_meets_tolerance():
    from paper_2008_02710_gb300.serve import Server
    import oracle
    reqs = _requests(10, seed=11)
    srv = Server(8 << 30, max_active=16, precision="mixed")
    res = srv.run(reqs, realtime=False)
    for r in res:
        q = reqs[r.id]
        assert r.status == "RLGL_OK"
        p = oracle.transition_probs(q.csr)
        ref, it, _ = oracle.power_iteration(q.csr, p, tol=1e-13, maxit=100000, nthreads=8)
        # a residual below tol bounds the error up to the chain's mixing
        # factor (Eq. convergence); these R-MAT chains mix fast
        assert np.abs(r.pi - ref).sum() <= max(100 * q.tol, 1e-6), (r.id, q.tol)


def test_batch_server_results_equal_alone_fp64():
    """Batching through the persistent batch solve: the queued requests form
    batches (a small budget forces several); every served result equals the
    same request solved alone."""
    from paper_2008_02710_gb300 import rlgl
    from paper_2008_02710_gb300.serve import BatchServer, summary
    reqs = _requests(24)
    foot = sorted(rlgl.footprint(r.csr.n, r.csr.nnz, False, "fp64") for r in reqs)
    srv = BatchServer(sum(foot[-6:]), max_chains=8, precision="fp64", theta_lag=0)
    res = srv.run(reqs, realtime=False)
    assert len(res) == len(reqs) and srv.stats["batches"] >= 3 and srv.stats["max_chains"] >= 2
    s = summary(res)
    assert s["not_ok"] == 0
    by_id = {r.id: r for r in res}
    for q in reqs:
        with rlgl.Chain(q.csr, precision="fp64") as ch:
            ch.set_params(theta_scale=0.5)
            info = ch.solve(q.schedule, 0.0, q.tol, q.max_steps)
            alone = ch.estimate()
        r = by_id[q.id]
        d = float(np.abs(r.pi - alone).sum())
        if r.moves == info["moves"]:
            assert d <= 1e-11, (q.id, d)
        else:  # the stop test fired a move apart (rounding at the tolerance)
            assert abs(r.moves - info["moves"]) <= 1 and d <= 10 * q.tol, (q.id, r.moves, info["moves"], d)


def test_batch_server_device_graphs_meet_tolerance():
    """Graphs drawn on the device (the serving bench's generator), served in
    MIXED precision, the small ones in a batch and the large ones alone:
    each estimate is within the tolerance's reach of the oracle's law for
    that graph."""
    import torch
    import oracle
    from paper_2008_02710_gb300.serve import BatchServer, Request
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(12):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(50000))))
        tol = float(rng.choice([1e-4, 1e-6, 1e-8]))
        reqs.append(Request(i, 0.0, synth.rmat_chain_n_device(n, seed=500 + i, device="cuda"), tol))
    # the four requests of 17000 nodes or more run alone (persistent sweep,
    # stale threshold), the other eight in one batch
    srv = BatchServer(8 << 30, max_chains=64, precision="mixed", alone_nodes=17000)
    res = srv.run(reqs, realtime=False)
    assert srv.stats["batches"] == 1 and srv.stats["alone"] == 4 and srv.stats["max_chains"] == 8
    for r in res:
        q = reqs[r.id]
        assert r.status == "RLGL_OK"
        host = synth.CSR(q.csr.n, q.csr.row_ptr.cpu().numpy(), q.csr.col.cpu().numpy(), None)
        p = oracle.transition_probs(host)
        ref, _, _ = oracle.power_iteration(host, p, tol=1e-13, maxit=100000, nthreads=8)
        assert np.abs(r.pi - ref).sum() <= max(100 * q.tol, 1e-6), (r.id, q.tol)
