"""The OSPA metric against its definition (Schuhmacher, Vo and Vo 2008): brute force over
every injection on small sets, and the closed forms of the empty, cardinality-only and
single-pair cases."""
import itertools
import math

import numpy as np
import pytest

from paper_2604_19723_gb300.ospa import ospa


def brute(X, Y, c, p):
    X, Y = np.asarray(X, float), np.asarray(Y, float)
    if len(X) > len(Y):
        X, Y = Y, X
    m, n = len(X), len(Y)
    if n == 0:
        return 0.0
    if m == 0:
        return c
    best = min(sum(min(c, np.linalg.norm(X[i] - Y[q[i]])) ** p for i in range(m))
               for q in itertools.permutations(range(n), m))
    return ((best + c ** p * (n - m)) / n) ** (1.0 / p)


def test_closed_forms():
    c = 1.5
    assert ospa(np.zeros((0, 3)), np.zeros((0, 3)), c) == 0.0
    assert ospa(np.zeros((0, 3)), np.ones((2, 3)), c) == c
    Y = np.array([[0.0, 0, 0], [10.0, 0, 0]])
    # one point exactly on one of two: only the missing one costs, c^p / n
    assert ospa(Y[:1], Y, c, 2) == pytest.approx(c * math.sqrt(0.5))
    # one pair at distance 0.3 < c: |x - y|
    assert ospa(np.array([[0.3, 0, 0]]), np.array([[0.0, 0, 0]]), c, 2) == pytest.approx(0.3)
    # beyond the cut-off the distance saturates at c
    assert ospa(np.array([[5.0, 0, 0]]), np.array([[0.0, 0, 0]]), c, 2) == pytest.approx(c)


@pytest.mark.parametrize("m,n,p", [(3, 3, 2), (2, 4, 2), (4, 2, 1), (3, 5, 2)])
def test_matches_brute_force(m, n, p):
    r = np.random.default_rng(10 * m + n)
    X = r.normal(size=(m, 3))
    Y = r.normal(size=(n, 3))
    for c in (0.5, 2.0):
        assert ospa(X, Y, c, p) == pytest.approx(brute(X, Y, c, p), rel=1e-12)
    # symmetric and invariant under reordering
    assert ospa(X, Y, 1.0, p) == pytest.approx(ospa(Y[::-1], X[::-1], 1.0, p), rel=1e-12)
