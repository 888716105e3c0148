"""The synthetic inputs are the recipe the design states: seeded generators
whose outputs have the stated sizes (after dropping self-loops and duplicate
undirected edges), so every number measured on them can be reproduced."""
import numpy as np
import pytest

import graphgen as gg


def _canonical_counts(g):
    n, s, d = g
    s = np.asarray(s, np.int64)
    d = np.asarray(d, np.int64)
    keep = s != d
    a, b = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    key = np.unique(a * n + b)
    deg = np.bincount(key // n, minlength=n) + np.bincount(key % n, minlength=n)
    return n, len(key), int(deg.max()), int((deg == 0).sum())


@pytest.mark.parametrize("name,expect", [
    ("grid32", (1024, 1984, 4, 0)),
    ("ba100k", (100000, 299991, 1153, 0)),
    ("dcsbm1m", (1000000, 3967668, 31142, 21741)),
])
def test_workload_sizes(name, expect):
    assert _canonical_counts(gg.workload(name)) == expect


def test_generators_are_seeded():
    a = gg.workload("ba100k")
    b = gg.workload("ba100k")
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_batch_mix():
    items = gg.batch_mix(256, 1000, 50000, 3)
    assert len(items) == 256
    kinds = {k for k, _ in items}
    assert kinds == {"grid", "tree", "ba"}
    sizes = np.array([g[0] for _, g in items])
    assert sizes.min() >= 900 and sizes.max() <= 50000   # grids round to r x c near n
    # log-uniform sizes: about half of them below the geometric mean of the range
    assert 0.35 < np.mean(sizes < np.sqrt(1000 * 50000)) < 0.65
