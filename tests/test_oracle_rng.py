"""Pins of the oracle's random-number layer: Philox-4x32-10 against the published
known-answer vectors, the 53-bit uniform map, and the distinct-pair index pick."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:2], v[2:6], v[6:10]))
    return rows


@pytest.mark.parametrize("key,ctr,out", _kat())
def test_philox_known_answers(oracle_mod, key, ctr, out):
    assert oracle_mod.philox(key[0], key[1], ctr) == tuple(out)


def test_u53_range_and_endpoints(oracle_mod):
    assert oracle_mod.u53(0, 0) == 0.0
    top = oracle_mod.u53(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == (2.0**53 - 1) / 2.0**53 and top < 1.0
    # the low word contributes only its top 21 bits
    assert oracle_mod.u53(0, 0x7FF) == 0.0
    assert oracle_mod.u53(0, 0x800) == 2.0**-53
    assert oracle_mod.u53(1, 0) == 2.0**-32


def test_u53_uniform_moments(oracle_mod):
    g = np.random.default_rng(7)
    w = g.integers(0, 2**32, size=(20000, 2), dtype=np.uint64)
    u = np.array([oracle_mod.u53(int(a), int(b)) for a, b in w])
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    assert abs(np.mean(u**2) - 1 / 3) < 4 * np.sqrt((1 / 5 - 1 / 9) / len(u))


@pytest.mark.parametrize("n", [2, 3, 7, 50])
def test_pick_pair_distinct_and_uniform(oracle_mod, n):
    g = np.random.default_rng(n)
    w = g.integers(0, 2**32, size=(8000, 2), dtype=np.uint64)
    counts = np.zeros((n, n))
    for a0, b0 in w:
        a, b = oracle_mod.pick_pair(int(a0), int(b0), n)
        assert 0 <= a < n and 0 <= b < n and a != b
        counts[a, b] += 1
    # every ordered pair (a != b) equally likely: chi-square over n(n-1) cells
    m = counts[~np.eye(n, dtype=bool)]
    e = len(w) / (n * (n - 1))
    chi2 = ((m - e) ** 2 / e).sum()
    dof = n * (n - 1) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_pick_pair_extreme_words(oracle_mod):
    # the multiply-shift map never reaches n, whatever the word
    for n in (2, 3, 1000, 2**31):
        a, b = oracle_mod.pick_pair(0xFFFFFFFF, 0xFFFFFFFF, n)
        assert (a, b) == (n - 1, n - 2)
        a, b = oracle_mod.pick_pair(0, 0, n)
        assert a == 0 and b == 1
