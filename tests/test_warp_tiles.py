"""Host-side check of the warp-tile bookkeeping of the all-green sweep and the
FP64 residual pull (no GPU). Tiles split the merge path of the in-link
lists (row ends merged with in-links) at diagonals that are multiples of
the tile size, as the create step's partition does. A row whose merge items
all fall in one tile is summed and finished in that tile. Any other row
leaves a piece in every tile it touches. It is finished once, after the
barrier, by the split pass: its end item is in a tile whose first row is
that row and began in an earlier tile (t_ptr[r0] < e0). Checked here: every
row is finished exactly once, and the split pass finds exactly the rows that
cross a tile boundary."""
import numpy as np
import pytest


def partition(t_ptr, items):
    """(first row, first in-link) of every tile boundary: for diagonal d the
    smallest i with t_ptr[i + 1] >= d - i (rows ended before d)."""
    n, nnz = len(t_ptr) - 1, int(t_ptr[-1])
    ntiles = (n + nnz + items - 1) // items
    tr, te = [], []
    for b in range(ntiles + 1):
        d = min(b * items, n + nnz)
        lo, hi = max(0, d - nnz), min(d, n)
        while lo < hi:
            mid = (lo + hi) // 2
            if t_ptr[mid + 1] >= d - mid:
                hi = mid
            else:
                lo = mid + 1
        tr.append(lo)
        te.append(d - lo)
    return np.array(tr), np.array(te)


def rows_of(deg):
    return np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)


@pytest.mark.parametrize("items", [256, 384])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_every_row_finished_once(items, seed):
    rng = np.random.default_rng(seed)
    n = 3000
    # power-law in-degrees with empty rows and a few hubs spanning many tiles
    deg = np.minimum(rng.zipf(1.7, n), 5000)
    deg[rng.choice(n, 300, replace=False)] = 0
    deg[rng.choice(n, 3, replace=False)] = 3 * items + 17
    t_ptr = rows_of(deg)
    tr, te = partition(t_ptr, items)
    ntiles = len(tr) - 1
    finished = np.zeros(n, dtype=int)
    split_rows = set()
    for b in range(ntiles):
        r0, e0 = tr[b], te[b]
        nr = tr[b + 1] - r0
        first_split = t_ptr[r0] < e0 if r0 < n else False
        for k in range(nr):
            if k == 0 and first_split:
                continue
            finished[r0 + k] += 1  # in-tile epilogue
        # the split pass: this tile's first row ends here and began earlier
        if nr > 0 and t_ptr[r0] < e0:
            finished[r0] += 1
            split_rows.add(int(r0))
    assert np.all(finished == 1)
    # the rows whose merge items (in-links at t_ptr[j] + j .., end at
    # t_ptr[j + 1] + j) cross a tile boundary
    a = t_ptr[:-1] + np.arange(n)
    e = t_ptr[1:] + np.arange(n)
    crossing = {int(j) for j in np.nonzero((a // items != e // items) & (deg > 0))[0]}
    assert split_rows == crossing


def test_tile_bounds_cover_the_merge_path():
    rng = np.random.default_rng(5)
    deg = rng.integers(0, 40, 1000)
    t_ptr = rows_of(deg)
    for items in (256, 384):
        tr, te = partition(t_ptr, items)
        sizes = (tr[1:] - tr[:-1]) + (te[1:] - te[:-1])
        assert np.all(sizes[:-1] == items) and 0 < sizes[-1] <= items
        assert tr[-1] == len(deg) and te[-1] == t_ptr[-1]
