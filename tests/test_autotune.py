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
