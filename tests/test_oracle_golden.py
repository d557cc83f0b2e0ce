"""The oracle against values the paper prints (fixtures in tests/golden/,
each citing its passage)."""
import os
from math import comb

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_monomial_order_of_the_worked_example():
    """Sec. 2, Eq. RBF_interp_poly: d = 2, k = 2 gives the six terms
    1, x, y, x^2, xy, y^2 as the columns of P, in that order."""
    want = np.loadtxt(os.path.join(GOLDEN, "monomials_d2_k2.txt"), dtype=np.int32)
    ax, ay = oracle.monomial_exponents(2)
    assert len(want) == comb(2 + 2, 2) == 6
    assert np.array_equal(np.stack([ax, ay], 1), want)


def test_monomial_order_is_graded_for_every_degree():
    """The same rule for the degrees the configurations use (2..6): every
    term of total degree <= k once, by total degree, the x power
    descending within a degree -- which for k = 2 is the printed order."""
    for k in range(7):
        ax, ay = oracle.monomial_exponents(k)
        assert len(ax) == comb(k + 2, k)
        terms = list(zip(ax.tolist(), ay.tolist()))
        assert len(set(terms)) == len(terms)
        assert all(a + b <= k for a, b in terms)
        assert terms == sorted(terms, key=lambda t: (t[0] + t[1], -t[0]))
