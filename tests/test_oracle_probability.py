"""Oracle pins: success probabilities and the Golomb-Rice parameter.

* Appendix A lemma: the bound on the rotation-fitting success probability
  reproduces both panels of the paper's Figure "prob" (printed values).
* The bound equals the exact probability (computed here by enumerating
  bit masks, a different route) for prime m and is below it otherwise.
* Brute-force and split success probabilities equal exact rational values.
* Kiely's rule picks the Golomb-Rice parameter with the smallest expected
  code length for a geometric source (checked by direct summation).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from helpers import golden_pairs


def exact_rotation_success(m, a):
    """P(success of one k | |A| = a), by enumeration of all b-subsets of [0, m):
    P(A distinct) P(B distinct) E[#distinct rotations of S] / C(m, b)."""
    b = m - a
    full = (1 << m) - 1
    masks = np.array([x for x in range(1 << m) if bin(x).count("1") == b], dtype=np.int64)
    period = np.full(len(masks), m, dtype=np.int64)
    done = np.zeros(len(masks), bool)
    for r in range(1, m + 1):
        rot = ((masks << r) | (masks >> (m - r))) & full if r < m else masks
        hit = (rot == masks) & ~done
        period[hit] = r
        done |= hit
    p_a = math.perm(m, a) / m**a
    p_b = math.perm(m, b) / m**b
    return p_a * p_b * period.mean() / math.comb(m, b)


def test_figure_prob_left_panel(orc):
    for m, factor in golden_pairs("fig_prob_factor.txt"):
        m = int(m)
        got = orc.rotation_success_bound(m) / orc.plain_success(m)
        assert got == pytest.approx(factor, rel=2e-5, abs=1e-4), m


def test_figure_prob_right_panel(orc):
    for m, bits in golden_pairs("fig_prob_space.txt"):
        m = int(m)
        # expected stored number grows by m * E_a[1/P(R|a)] / (1/P(B))
        e_rot = sum(math.comb(m, a) * 2.0**-m / orc.rotation_bound_given_a(m, a)
                    for a in range(m + 1))
        got = math.log2(m * orc.plain_success(m) * e_rot) / m
        assert got == pytest.approx(bits, rel=2e-5, abs=1e-9), m


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7, 8, 9, 11, 12, 13])
def test_bound_against_exact_enumeration(orc, m):
    for a in range(m + 1):
        exact = exact_rotation_success(m, a)
        bound = orc.rotation_bound_given_a(m, a)
        assert bound <= exact * (1 + 1e-12)
        if math.gcd(a, m - a) == 1:
            assert bound == pytest.approx(exact, rel=1e-12)


def test_plain_success_is_m_factorial_over_m_to_the_m(orc):
    for m in range(1, 25):
        assert orc.plain_success(m) == pytest.approx(math.factorial(m) / m**m, rel=1e-13)
    # expected brute-force trials for the benchmark leaf sizes
    assert 1 / orc.plain_success(8) == pytest.approx(16777216 / 40320, rel=1e-12)
    assert 1 / orc.plain_success(16) == pytest.approx(881657.95, rel=1e-7)


def multinomial_success(parts):
    m = sum(parts)
    p = Fraction(math.factorial(m))
    for q in parts:
        p /= math.factorial(q)
        p *= Fraction(q, m) ** q
    return float(p)


@pytest.mark.parametrize("leaf,m", [(8, 32), (8, 96), (8, 20), (12, 60), (12, 240), (16, 112),
                                    (16, 560), (16, 320), (16, 2000), (16, 1120), (5, 11)])
def test_split_success_is_the_multinomial(orc, leaf, m):
    assert orc.split_success(leaf, m) == pytest.approx(multinomial_success(orc.parts(leaf, m)),
                                                       rel=1e-9)


def test_expected_split_trials_closed_forms(orc):
    # full lower-1 / lower-2 nodes for l = 8 and l = 16; a fanout-2 node of 2000 keys
    assert 1 / orc.split_success(8, 32) == pytest.approx(185.28, rel=1e-4)
    assert 1 / orc.split_success(8, 96) == pytest.approx(116.89, rel=1e-4)
    assert 1 / orc.split_success(16, 112) == pytest.approx(397978, rel=1e-5)
    assert 1 / orc.split_success(16, 560) == pytest.approx(222260, rel=1e-5)
    assert 1 / orc.split_success(16, 2000) == pytest.approx(55.65, rel=1e-3)


def geometric_rice_length(p, tau):
    """Expected Golomb-Rice length of X ~ Geometric(p) on {0, 1, ...}."""
    q = (1.0 - p) ** (2**tau)
    return tau + 1 + q / (1.0 - q)


def test_kiely_rule_is_optimal_for_geometric_sources(orc):
    for p in np.geomspace(1e-9, 0.99, 400):
        tau = orc.kiely_tau(float(p))
        lengths = [geometric_rice_length(float(p), t) for t in range(0, 40)]
        best = min(lengths)
        assert lengths[tau] <= best * (1 + 1e-9), (p, tau, int(np.argmin(lengths)))


@pytest.mark.parametrize("leaf,rotation", [(8, False), (8, True), (12, True), (16, True), (24, True)])
def test_tau_table_uses_the_node_probability(orc, leaf, rotation):
    tau = orc.tau_table(leaf, rotation, 600)
    assert tau[0] == 0 and tau[1] == 0
    for m in range(2, 601):
        if m <= leaf:
            p = orc.rotation_success_bound(m) / m if rotation else orc.plain_success(m)
        else:
            p = orc.split_success(leaf, m)
        assert tau[m] == orc.kiely_tau(p)
    # a full plain leaf of 8 keys takes about 416 trials: parameter 8
    if not rotation and leaf == 8:
        assert tau[8] == 8
