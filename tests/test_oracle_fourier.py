"""Pins of the von Neumann analysis that gives CFL(N) (Sec. 5, under
Eq. time.step.2d): the N = 0 upwind closed form, an independent closed form of
the amplification matrix for linear advection, the stored table, and the
behaviour of the actual scheme just below and above the limit."""
import json
import os
from math import factorial

import numpy as np
import pytest

from oracle import fourier
from oracle.basis import Basis
from oracle.crkfr import Scheme1D
from oracle.systems import VarCoeffAdvection

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_cfl.json")


def test_n0_is_upwind():
    """N = 0 is first-order upwind: G = 1 - nu (1 - e^{-i kappa}), limit 1."""
    for nu in (0.3, 0.9):
        k = fourier.kappa_grid(16)
        G = fourier.amplification(0, nu, k)[:, 0, 0]
        assert np.allclose(G, 1 - nu * (1 - np.exp(-1j * k)), atol=1e-15)
    assert fourier.cfl_number(0) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("family", ["gl", "gll"])
def test_amplification_closed_form(N, family):
    """For v_t + v_x = 0 the local stages give U = T(-nu D) v with
    T(z) = sum_{k<=N} z^k/(k+1)!, the face flux is upwind (lambda = a) and the
    non-conservative fluctuation cancels on the upwind side, so
    G = I - nu (D + g_L' (e^{-i kappa} l(1)^T - l(0)^T)) T(-nu D)."""
    bs = Basis(N, family)
    D = bs.D
    for nu in (0.05, 0.2):
        Z = -nu * D
        T = sum(np.linalg.matrix_power(Z, k) / factorial(k + 1) for k in range(N + 1))
        ks = fourier.kappa_grid(32)
        Go = fourier.amplification(N, nu, ks, family)
        for i, k in enumerate(ks):
            Op = D + np.outer(bs.gLp, np.exp(-1j * k) * bs.l1 - bs.l0)
            G = np.eye(N + 1) - nu * Op @ T
            assert np.max(np.abs(G - Go[i])) < 1e-12


def test_stored_cfl_table():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    for key, val in g["cfl"].items():
        N, family = key.split("_")
        assert fourier.cfl_number(int(N), family) == pytest.approx(val, rel=1e-12, abs=1e-14)


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2, 3])
def test_scheme_stable_below_and_unstable_above_limit(N):
    """Run the actual step on random periodic data: bounded at 0.97 CFL(N),
    growing at 1.05 CFL(N)."""
    cfl = fourier.cfl_number(N)
    E = 16
    rng = np.random.default_rng(N)
    v0 = rng.standard_normal((1, E, N + 1))
    a = np.ones((E, N + 1))
    sch = Scheme1D(VarCoeffAdvection(), N, 1.0 / E)
    out = {}
    for f in (0.97, 1.05):
        v = v0.copy()
        for _ in range(1500):
            v = sch.step(v, a, f * cfl / E)
        out[f] = np.max(np.abs(v))
    assert out[0.97] < 2.0 * np.max(np.abs(v0))
    assert out[1.05] > 1e3 * np.max(np.abs(v0))
