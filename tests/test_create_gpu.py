"""Edge cases of context creation and of the sweep's staged select, through
the C-ABI against the oracle (or the one-kernel-per-phase path):
- a weighted row longer than 65536 links, whose weight sum a whole block
  takes (non-integer weights, so the order of the FP64 additions differs
  from the oracle's by rounding only);
- a chain one node-range longer than the grid, so that exactly one block
  stages a second, ragged range;
- the stale threshold on the MIXED path through many re-derivations."""
import numpy as np
import pytest

import oracle
from paper_2008_02710_gb300 import synth

pytestmark = pytest.mark.gpu


def Chain(*a, **k):
    from paper_2008_02710_gb300.rlgl import Chain as C
    return C(*a, **k)


def _star_chain(n, seed):
    """Node 0 links to every node (one row of n links); node i >= 1 links to
    0, to itself and to i + 1 (mod n); weights U(0, 1]."""
    rng = np.random.default_rng(seed)
    cols = [np.arange(n, dtype=np.int32)]
    i = np.arange(1, n, dtype=np.int64)
    rest = np.stack([np.zeros(n - 1, np.int64), i, (i + 1) % n], axis=1).astype(np.int32)
    col = np.concatenate([cols[0], rest.reshape(-1)])
    row_ptr = np.concatenate([[0, n], n + 3 * np.arange(1, n, dtype=np.int64)]).astype(np.int64)
    w = (1.0 - rng.random(col.shape[0])).astype(np.float32)  # (0, 1]
    return synth.CSR(n, row_ptr, col, w)


def test_long_weighted_row_sum_by_a_block():
    csr = _star_chain(150001, seed=9)
    assert csr.row_ptr[1] - csr.row_ptr[0] > 65536
    pi_or, C, H, info_or = oracle.run(csr, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=1e-12,
                                      max_steps=100000)
    assert info_or["status"] == "OK"
    for prec, bound in (("fp64", 1e-11), ("mixed", 1e-6)):
        with Chain(csr, precision=prec) as ch:
            ch.set_params(theta_scale=0.5)
            info = ch.solve("link_threshold", tol=1e-12 if prec == "fp64" else 1e-9, max_steps=100000)
            pi = ch.estimate()
        assert info["status"] == "RLGL_OK"
        assert np.abs(pi - pi_or).sum() <= bound, prec


def test_one_block_stages_a_second_ragged_range():
    """608 blocks x 1024 nodes + 17: block 0 alone has a second range, of 17
    nodes. 25 MIXED moves of the sweep agree with the phase kernels."""
    csr = synth.rmat_chain_n(608 * 1024 + 17, 4, seed=21)
    res = []
    for persistent in (1, 0):
        with Chain(csr, precision="mixed") as ch:
            ch.set_params(theta_scale=0.5, persistent=persistent)
            info = ch.solve("link_threshold", tol=0.0, max_steps=25, raise_on_noconv=False)
            assert info["moves"] == 25 and ch.get_params().persistent == persistent
            res.append((ch.estimate(), ch.move_log(25)))
    (pa, la), (pb, lb) = res
    assert np.abs(pa - pb).sum() <= 2e-6
    for ra, rb in zip(la[:10], lb[:10]):
        assert abs(ra["green"] - rb["green"]) <= max(2, rb["green"] // 10000)


def test_stale_threshold_mixed_through_many_rederivations():
    csr = synth.rmat_chain(14, 16, seed=5, weighted=True)
    pi_or, C, H, info_or = oracle.run(csr, sched=oracle.LINK_THRESHOLD, theta_scale=0.5, tol=1e-12,
                                      max_steps=200000)
    with Chain(csr, precision="mixed") as ch:
        ch.set_params(theta_scale=0.5, theta_lag=1, refresh_factor=0.1)
        info = ch.solve("link_threshold", tol=1e-10, max_steps=200000)
        pi = ch.estimate()
        inv = ch.invariant_residual()
    assert info["status"] == "RLGL_OK"
    assert info["refreshes"] >= 5
    # the MIXED bound against the FP64 law (FP32 cash between re-derivations)
    assert np.abs(pi - pi_or).sum() <= 1e-6
    assert inv <= 1e-9
