"""Pins of the oracle's two-point W1 (Eq. (W1_vector), Algorithms "WassersteinDistance2" and
"WassersteinDistance2_vector"): the transport LP against brute force over permutations and the
assignment form, closed forms (translation, points on the diagonal), replication of atoms for
unequal sample counts, and the pair weighting of the aggregate."""
import itertools
import math

import numpy as np
import pytest

import ensemble_inputs as gen
from oracle import stats

pytest.importorskip("scipy")


def _cost(X, Y):
    return np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(axis=2))


@pytest.mark.parametrize("M,k", [(3, 2), (5, 2), (6, 6)])
def test_lp_and_assignment_equal_brute_force(M, k):
    X = gen.uniform(1 + M, (M, k))
    Y = gen.uniform(2 + M, (M, k)) + 0.3
    C = _cost(X, Y)
    brute = min(sum(C[m, s[m]] for m in range(M)) for s in itertools.permutations(range(M))) / M
    assert abs(stats.ot_w1_lp(X, Y) - brute) <= 1e-9 * brute
    assert abs(stats.ot_w1_assignment(X, Y) - brute) <= 1e-12 * brute


@pytest.mark.parametrize("k", [2, 6])
def test_translation_gives_the_shift_length(k):
    """W1(mu, mu + t) = |t|: the identity coupling costs |t| and the 1-Lipschitz function
    x . t / |t| shows no coupling costs less."""
    X = gen.uniform(7, (9, k))
    t = gen.uniform(8, (k,))
    for W in (stats.ot_w1_lp(X, X + t), stats.ot_w1_assignment(X, X + t)):
        assert abs(W - np.linalg.norm(t)) <= 1e-9 * np.linalg.norm(t)


def test_unequal_counts_equal_replicated_assignment():
    """M_A = 6, M_B = 3: the LP optimum equals the assignment between A and B with every atom
    of B repeated twice (uniform weights 1/6 on both sides)."""
    X = gen.uniform(11, (6, 2))
    Y = gen.uniform(12, (3, 2)) + 0.1
    lp = stats.ot_w1_lp(X, Y)
    rep = stats.ot_w1_assignment(X, np.repeat(Y, 2, axis=0))
    assert abs(lp - rep) <= 1e-9 * rep
    # the same law sampled with twice as many atoms is at distance 0
    assert stats.ot_w1_lp(np.repeat(Y, 2, axis=0), Y) <= 1e-12


def test_points_on_the_diagonal_reduce_to_one_dimension():
    """For a pair (x, x) the component-wise atoms are (a, a): the Euclidean cost is sqrt(2) |a - b|,
    so W1 is sqrt(2) times the one-dimensional W1 (sorted rearrangement / CDF distance), also for
    unequal counts."""
    a = gen.uniform(21, (8,))
    b = gen.uniform(22, (4,)) * 1.3
    X = np.stack([a, a], axis=1)
    Y = np.stack([b, b], axis=1)
    assert abs(stats.ot_w1(X, Y) - math.sqrt(2.0) * stats.w1_empirical(a, b)) <= 1e-9


def test_aggregate_weights_and_symmetry():
    M, G = 5, 3
    ua = gen.uniform(31, (M, G, 3))
    ub = gen.uniform(32, (M, G, 3)) + 0.05
    for vector in (True, False):
        total, D = stats.w1_two_point(ua, ub, vector=vector, per_pair=True)
        Dv = D if vector else D.sum(axis=1)
        manual = 0.0
        for i in range(G):
            for j in range(i, G):
                manual += (1.0 if i == j else 2.0) * Dv[stats.pair_index(i, j, G)]
        assert abs(total - manual / G**2) <= 1e-14
        assert abs(stats.w1_two_point(ub, ua, vector=vector) - total) <= 1e-9 * total
        assert stats.w1_two_point(ua, ua, vector=vector) <= 1e-12
    # diagonal pairs of the vector form: (u, u) in R^6 costs sqrt(2) |u - v| in R^3
    _, D = stats.w1_two_point(ua, ub, vector=True, per_pair=True)
    for i in range(G):
        assert abs(D[stats.pair_index(i, i, G)] - math.sqrt(2.0) * stats.ot_w1(ua[:, i, :], ub[:, i, :])) <= 1e-9
