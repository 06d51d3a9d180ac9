"""Pins of the oracle's Butcher tableaux: the printed App. C entries and the
textbook rooted-tree order conditions."""
import json
import os
from math import factorial

import numpy as np
import pytest

from oracle.tableau import (butcher_rk5, default_tableau, ht112_explicit, rk4_classical,
                            ssp3_imex433_explicit)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "app_c_tableaux.json")


def order_conditions(A, b):
    """Residuals of the explicit RK order conditions up to order 5."""
    c = A.sum(axis=1)
    conds = [
        (1, b.sum() - 1),
        (2, b @ c - 1 / 2),
        (3, b @ c ** 2 - 1 / 3), (3, b @ A @ c - 1 / 6),
        (4, b @ c ** 3 - 1 / 4), (4, b @ (c * (A @ c)) - 1 / 8),
        (4, b @ A @ c ** 2 - 1 / 12), (4, b @ A @ A @ c - 1 / 24),
        (5, b @ c ** 4 - 1 / 5), (5, b @ (c ** 2 * (A @ c)) - 1 / 10),
        (5, b @ (A @ c) ** 2 - 1 / 20), (5, b @ (c * (A @ c ** 2)) - 1 / 15),
        (5, b @ (c * (A @ A @ c)) - 1 / 30), (5, b @ A @ c ** 3 - 1 / 20),
        (5, b @ A @ (c * (A @ c)) - 1 / 40), (5, b @ A @ A @ c ** 2 - 1 / 60),
        (5, b @ A @ A @ A @ c - 1 / 120),
    ]
    return conds


def order_of(A, b):
    p = 0
    for k in range(1, 6):
        if all(abs(r) < 1e-14 for o, r in order_conditions(A, b) if o == k):
            p = k
        else:
            break
    return p


def test_printed_app_c_tableaux():
    """The explicit tableaux equal those printed in App. C (golden file)."""
    with open(GOLDEN) as fh:
        g = json.load(fh)
    A, b = ht112_explicit()
    assert np.array_equal(A, np.array(g["ht112"]["A_explicit"]))
    assert np.array_equal(b, np.array(g["ht112"]["b_explicit"]))
    A, b = ssp3_imex433_explicit()
    assert np.allclose(A, np.array(g["ssp3_imex433"]["A_explicit"]), rtol=0, atol=1e-16)
    assert np.allclose(b, np.array(g["ssp3_imex433"]["b_explicit"]), rtol=0, atol=1e-16)


@pytest.mark.parametrize("fn,p", [(ht112_explicit, 2), (ssp3_imex433_explicit, 3),
                                  (rk4_classical, 4), (butcher_rk5, 5)])
def test_order(fn, p):
    A, b = fn()
    assert np.allclose(np.triu(A), 0.0)
    assert order_of(A, b) == p


@pytest.mark.parametrize("N", [0, 1, 2, 3, 4])
def test_time_average_polynomial_matches_lw(N):
    """sum_i b_i P_i(z) agrees with (e^z - 1)/z through z^N, the property that
    makes cRK-FR linearly equivalent to LWFR (Sec. 5, under Eq. time.step.2d):
    stage polynomials P_i(z) = 1 + z sum_j a_ij P_j(z)."""
    A, b = default_tableau(N)
    s = len(b)
    P = []
    for i in range(s):
        poly = np.zeros(s + 1)
        poly[0] = 1.0
        for j in range(i):
            poly[1:] += A[i, j] * P[j][:-1]
        P.append(poly)
    T = sum(bi * Pi for bi, Pi in zip(b, P))
    for k in range(N + 1):
        assert abs(T[k] - 1.0 / factorial(k + 1)) < 1e-15
