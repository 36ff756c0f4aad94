"""Seeded input generators: determinism and the structure each workload
promises (these hold none of the method's arithmetic)."""
import hashlib

import numpy as np
import pytest

from paper_2008_02710_gb300 import synth


def _digest(csr):
    h = hashlib.sha256()
    for a in (csr.row_ptr, csr.col) + ((csr.w,) if csr.w is not None else ()):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def test_tiny_chain_structure_and_determinism():
    a, b = synth.tiny_chain(1000, 1), synth.tiny_chain(1000, 1)
    assert _digest(a) == _digest(b)
    assert _digest(a) != _digest(synth.tiny_chain(1000, 2))
    deg = a.degrees()
    assert deg.min() >= 3 and deg.max() <= 10
    for i in (0, 17, 999):
        row = a.col[a.row_ptr[i]:a.row_ptr[i + 1]]
        assert row[-1] == i and row[-2] == (i + 1) % 1000
    k = np.round(a.w.astype(np.float64) * (1 << 24))
    assert np.array_equal(k / (1 << 24), a.w.astype(np.float64))
    assert a.w.min() > 0 and a.w.max() <= 1


def test_rmat_structure():
    g = synth.rmat_chain(12, 16, seed=3)
    n = 1 << 12
    assert g.n == n and g.nnz == 16 * n + 2 * n and g.w is None
    assert g.col.min() >= 0 and g.col.max() < n
    # every row keeps its cycle edge and self-loop (appended after the R-MAT edges)
    for i in (0, 5, n - 1):
        row = g.col[g.row_ptr[i]:g.row_ptr[i + 1]]
        assert row[-2] == (i + 1) % n and row[-1] == i
    deg = g.degrees()
    assert deg.max() > 20 * deg.mean()  # heavy tail
    assert _digest(g) == _digest(synth.rmat_chain(12, 16, seed=3))


def test_rmat_undirected_is_symmetric():
    g = synth.rmat_chain(9, 4, seed=5, undirected=True)
    n = g.n
    rows = np.repeat(np.arange(n), g.degrees())
    A = np.zeros((n, n))
    np.add.at(A, (rows, g.col), 1.0)
    assert np.array_equal(A, A.T)


def test_weighted_rmat_weights_on_grid():
    g = synth.rmat_chain(10, 8, seed=4, weighted=True)
    w = g.w.astype(np.float64)
    assert np.array_equal(np.round(w * (1 << 24)) / (1 << 24), w)
    assert w.min() > 0 and w.max() <= 1


def test_counter_rng_is_position_only():
    assert synth.u64(7, 3, 12345) == synth.u64(7, 3, 12345)
    assert synth.u64(7, 3, 12345) != synth.u64(7, 4, 12345)
    u = np.array([synth.unit(1, 2, i) for i in range(4000)])
    assert 0 <= u.min() and u.max() < 1 and abs(u.mean() - 0.5) < 0.02


def test_powerlaw_chain():
    g = synth.powerlaw_chain(2000, 8.0, seed=11)
    deg = g.degrees() - 2
    assert abs(deg.mean() - 8.0) < 0.5
    assert g.col.max() < 2000


def test_device_rmat_generator_on_cpu_tensors():
    """The device R-MAT generator (run here on CPU tensors): a valid CSR of
    n nodes, 18 n links (16 n R-MAT + cycle + self-loops), every node with
    its cycle edge and self-loop, skewed in-degrees, seeded."""
    torch = pytest.importorskip("torch")
    n = 5000
    a = synth.rmat_chain_n_device(n, seed=3, device="cpu")
    b = synth.rmat_chain_n_device(n, seed=3, device="cpu")
    c = synth.rmat_chain_n_device(n, seed=4, device="cpu")
    rp, col = a.row_ptr.numpy(), a.col.numpy()
    assert a.n == n and rp[0] == 0 and rp[-1] == 18 * n and np.all(np.diff(rp) >= 2)
    assert col.dtype == np.int32 and col.min() >= 0 and col.max() < n
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(np.bincount(rows[col == rows], minlength=n) >= 1)  # self-loops
    assert np.all(np.bincount(rows[col == (rows + 1) % n], minlength=n) >= 1)  # cycle
    indeg = np.bincount(col, minlength=n)
    assert indeg.max() > 20 * indeg.mean() / 2
    assert np.array_equal(a.col.numpy(), b.col.numpy()) and not np.array_equal(a.col.numpy(), c.col.numpy())
    stacked, node_ptr = synth.stack_chains_device([a, c])
    assert stacked.n == 2 * n and int(stacked.row_ptr[-1]) == 36 * n
    assert list(node_ptr) == [0, n, 2 * n] and int(stacked.col[-1]) >= n
