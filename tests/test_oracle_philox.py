"""Pins of the oracle's Philox4x32-10 generator and normal draws."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        got = philox.philox4x32_10(np.array(ctr), np.array(key))
        assert [int(g) for g in got] == out


def test_uniform_range_and_extremes():
    assert philox.uniform53(0, 0) == 2.0 ** -53
    assert philox.uniform53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0


def test_normal_moments():
    xi = philox.normals(seed=0, iteration=0, level=0, samples=np.arange(4096), n_modes=64)
    n = xi.size
    assert abs(xi.mean()) < 5.0 / np.sqrt(n)
    assert abs(xi.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    # fourth moment of N(0,1) is 3
    assert abs((xi ** 4).mean() - 3.0) < 5.0 * np.sqrt(96.0 / n)
    # even/odd modes (cos/sin halves of Box-Muller) uncorrelated
    c = np.corrcoef(xi[:, 0::2].ravel(), xi[:, 1::2].ravel())[0, 1]
    assert abs(c) < 5.0 / np.sqrt(n / 2)


def test_counter_fields_are_independent_streams():
    a = philox.normals(0, 0, 1, [5], 8)
    assert not np.allclose(a, philox.normals(0, 1, 1, [5], 8))  # iteration
    assert not np.allclose(a, philox.normals(0, 0, 2, [5], 8))  # level
    assert not np.allclose(a, philox.normals(0, 0, 1, [6], 8))  # sample
    assert not np.allclose(a, philox.normals(1, 0, 1, [5], 8))  # seed
    # a sample's draw does not depend on which batch it was drawn in
    b = philox.normals(0, 0, 1, [3, 4, 5], 8)
    assert np.array_equal(a[0], b[2])
