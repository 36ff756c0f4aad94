"""The parameter autotuner: selection logic on a stand-in chain (CPU), and
one tuning run on the GPU."""
import numpy as np
import pytest

from paper_2008_02710_gb300 import autotune as at


class _FakeChain:
    """Records parameters; a solve 'takes' a time that depends on them."""

    def __init__(self, cost, converges):
        self.params = {}
        self.cost, self.converges = cost, converges
        self.now = 0.0
        self.resets = 0

    def set_params(self, **kw):
        self.params.update(kw)

    def reset(self, m0=None):
        self.resets += 1

    def solve(self, schedule, tol, max_steps, raise_on_noconv):
        self.now += self.cost(self.params)
        ok = self.converges(self.params)
        return {"status": "RLGL_OK" if ok else "RLGL_ENOCONV", "moves": 10 if ok else max_steps}

    def clock(self):
        return self.now


def test_candidates_is_the_product():
    c = at.candidates({"a": (1, 2), "b": (3,)})
    assert c == [{"a": 1, "b": 3}, {"a": 2, "b": 3}]
    assert len(at.candidates()) == 4 * 2 * 3


def test_picks_the_fastest_converging_setting():
    cost = lambda p: abs(p["theta_scale"] - 0.5) + 0.1 * p["r"] + p["pull_crossover"]
    conv = lambda p: p["pull_crossover"] != 0.1      # the cheapest ones fail
    ch = _FakeChain(cost, conv)
    res = at.autotune(ch, clock=ch.clock)
    assert res["best"] == {"theta_scale": 0.5, "r": 1, "pull_crossover": 0.25}
    assert ch.params == res["best"]
    assert len(res["trials"]) == 24
    assert all(t[1] is None for t in res["trials"] if t[0]["pull_crossover"] == 0.1)


def test_batch_grid_adds_the_block_size():
    cost = lambda p: abs(p["theta_scale"] - 0.5) + (0.0 if p["batch_block"] == 128 else 1.0)
    ch = _FakeChain(cost, lambda p: True)
    ch.nchains = 4
    res = at.autotune(ch, clock=ch.clock)
    assert len(res["trials"]) == 24 * 3
    assert res["best"]["batch_block"] == 128 and ch.params["batch_block"] == 128


def test_raises_when_nothing_converges():
    ch = _FakeChain(lambda p: 1.0, lambda p: False)
    with pytest.raises(RuntimeError):
        at.autotune(ch, grid={"theta_scale": (1.0,)}, clock=ch.clock)


@pytest.mark.gpu
def test_autotune_on_gpu():
    import oracle
    from paper_2008_02710_gb300 import synth
    from paper_2008_02710_gb300.rlgl import Chain
    csr = synth.rmat_chain(13, 16, seed=2)
    p = oracle.transition_probs(csr)
    ref, _, _ = oracle.power_iteration(csr, p, tol=1e-15, maxit=100000)
    with Chain(csr, precision="mixed") as ch:
        res = at.autotune(ch, tol=1e-9, grid={"theta_scale": (0.5, 1.0), "r": (1,),
                                               "pull_crossover": (0.25,)})
        pi = ch.estimate()
        prm = ch.get_params()
    assert res["best"]["theta_scale"] in (0.5, 1.0) and prm.theta_scale == res["best"]["theta_scale"]
    assert np.abs(pi - ref).sum() < 1e-6


@pytest.mark.gpu
def test_autotune_batch_block_size_on_gpu():
    """Tuning a batch picks a block size the library accepts and leaves the
    batch solved with it."""
    import oracle
    from paper_2008_02710_gb300 import synth
    from paper_2008_02710_gb300.rlgl import Chain
    parts = [synth.rmat_chain_n(n, 8, seed=s) for n, s in ((3000, 1), (500, 2), (12000, 3))]
    batch, node_ptr = synth.stack_chains(parts)
    with Chain(batch, node_ptr=node_ptr, precision="mixed") as ch:
        res = at.autotune(ch, tol=1e-9, grid={"theta_scale": (0.5,), "r": (1,), "pull_crossover": (0.25,),
                                               "batch_block": (128, 256, 512)})
        pi = ch.estimate()
        assert ch.get_params().batch_block == res["best"]["batch_block"]
    assert len(res["trials"]) == 3 and all(t[3] == "RLGL_OK" for t in res["trials"])
    for k, c in enumerate(parts):
        law, _, _ = oracle.power_iteration(c, oracle.transition_probs(c), tol=1e-15, maxit=100000)
        assert np.abs(pi[node_ptr[k]:node_ptr[k + 1]] - law).sum() < 1e-6
