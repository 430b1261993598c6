"""Host-side logic without a GPU: the size buckets of PanelBatch, and the seeded
synthetic populations (determinism, prefixes, sizes, orientation, angles)."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_02166_gb300 import inputs

pytest.importorskip("torch")
from paper_1511_02166_gb300.solver import size_buckets  # noqa: E402


@pytest.mark.parametrize("width,min_count", [(64, 1), (64, 608), (192, 608), (192, 5), (1, 1)])
def test_size_buckets_partition_the_sorted_batch(width, min_count):
    rng = np.random.default_rng(width + min_count)
    sizes = np.sort(rng.integers(3, 700, 2500))[::-1]
    buckets = size_buckets(sizes, width, min_count)
    # contiguous, in order, every airfoil exactly once
    pos = 0
    for start, count, nmax in buckets:
        assert start == pos and count >= 1
        assert nmax == max(int(sizes[start]), 3) == int(sizes[start:start + count].max())
        pos += count
    assert pos == len(sizes)
    # no bucket below min_count unless the whole batch is
    if len(buckets) > 1:
        assert all(c >= min_count for _, c, _ in buckets)
    # without merging, one key ceil(n / width) per bucket
    if min_count == 1:
        for start, count, _ in buckets:
            keys = {-(-int(n) // width) for n in sizes[start:start + count]}
            assert len(keys) == 1


def test_size_buckets_small_batches():
    assert size_buckets(np.array([], dtype=np.int64), 64, 608) == []
    assert size_buckets(np.array([200, 150, 90]), 64, 608) == [(0, 3, 200)]


@pytest.mark.parametrize("name", sorted(inputs.SPECS))
def test_populations_are_seeded_prefix_stable_and_valid(name):
    spec = inputs.SPECS[name]
    a = inputs.make_population(name, batch=7)
    b = inputs.make_population(name, batch=7)
    c = inputs.make_population(name, batch=3)
    assert np.array_equal(a.nodes, b.nodes) and np.array_equal(a.alpha, b.alpha)
    # a smaller batch is a prefix of the same stream
    assert np.array_equal(c.nodes, a.nodes[:c.offsets[-1]]) and np.array_equal(c.alpha, a.alpha[:3])
    sizes = np.diff(a.offsets)
    assert np.all(sizes >= spec.n_min) and np.all(sizes <= spec.n_max)
    assert np.all(np.abs(a.alpha) <= math.radians(10.0) + 1e-12)
    for k in range(a.batch):
        xy = a.airfoil(k)
        assert np.all(np.isfinite(xy))
        assert oracle.signed_area(xy) > 0  # counter-clockwise (Section 2's node order)
        assert np.argmax(xy[:, 0]) == 0     # trailing edge first
