"""Pins of the oracle's subcell blending limiter (Sec. 4: Eqs.
blended.scheme, subcell.defn, low.order.update, numflux.args, Fblend;
Algorithms 1 and 2):

- alpha = 0 everywhere is the plain cRK-FR step, bit for bit;
- alpha = 1 everywhere is first-order finite volumes on the subcell grid
  (cells of width w_p dx, written out independently here with the fluxes of
  Eq. combined.num.flux);
- mass is conserved and h stays positive for a dam break onto a thin layer,
  where the unlimited step produces a negative depth;
- the smoothness indicator vanishes on smooth data and on polynomials of
  degree N - 2, and is near 1 at a jump;
- with the well-balanced form the limited step keeps a lake at rest to
  round-off.
"""
import numpy as np
import pytest

from oracle import fourier
from oracle.basis import Basis
from oracle.crkfr import Scheme1D
from oracle.limiter import Blending1D, hennemann_alpha
from oracle.systems import ShallowWater1D, ShallowWater1DWB, VarCoeffAdvection

G = 9.81


def grid(N, E, L=1.0, family="gl"):
    bs = Basis(N, family)
    dx = L / E
    return bs, (np.arange(E)[:, None] + bs.xi[None, :]) * dx, dx


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll"), (3, "gl"), (4, "gl")])
def test_alpha_zero_is_the_plain_step(N, family):
    bs, x, dx = grid(N, 12, family=family)
    b = 0.1 * np.sin(2 * np.pi * x) ** 2
    u = np.stack([1.0 + 0.1 * np.cos(2 * np.pi * x) - b, 0.3 * np.sin(2 * np.pi * x)])
    sch = Scheme1D(ShallowWater1D(G), N, dx, family=family)
    dt = sch.compute_dt(u, b, fourier.cfl_number(N, family, halvings=30), 0.5)
    assert np.array_equal(Blending1D(sch, alpha=0.0).step(u, b, dt), sch.step(u, b, dt))


def subcell_fv(sy, u, c, w, dx, dt):
    """First-order FV on the subcells of all elements, as one periodic row of
    cells of widths w_p dx: flux between cells i, i+1 by Eq. combined.num.flux,
    each side with B at its own state (Eq. non.cons.num.flux.basic)."""
    M = u.shape[0]
    U = u.reshape(M, -1)
    C = c.reshape(-1)
    W = np.tile(w, u.shape[1]) * dx
    K = U.shape[1]
    out = U.copy()
    for i in range(K):
        j = (i + 1) % K
        uL, uR, cL, cR = U[:, i], U[:, j], C[i], C[j]
        lam = max(sy.speed(uL, cL), sy.speed(uR, cR))
        f = 0.5 * (sy.flux(uL, cL) + sy.flux(uR, cR)) - 0.5 * lam * (uR - uL)
        un, cn = 0.5 * (uL + uR), 0.5 * (cL + cR)
        out[:, i] -= dt / W[i] * (f + sy.ncprod(uL, cL, un, cn))
        out[:, j] += dt / W[j] * (f + sy.ncprod(uR, cR, un, cn))
    return out.reshape(u.shape)


@pytest.mark.parametrize("N,family", [(1, "gl"), (3, "gl"), (3, "gll")])
def test_alpha_one_is_subcell_finite_volumes(N, family):
    bs, x, dx = grid(N, 7, family=family)
    b = 0.1 * np.sin(2 * np.pi * x) ** 2
    u = np.stack([1.0 + 0.1 * np.cos(2 * np.pi * x) - b, 0.3 * np.sin(2 * np.pi * x)])
    sy = ShallowWater1D(G)
    sch = Scheme1D(sy, N, dx, family=family)
    dt = 0.2 * dx * np.min(bs.w) / 4.0
    got = Blending1D(sch, alpha=1.0).step(u, b, dt)
    want = subcell_fv(sy, u, b, bs.w, dx, dt)
    assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("N,family", [(1, "gl"), (3, "gll")])
def test_alpha_one_with_friction_is_fv_then_backward_euler(N, family):
    """With Chezy friction and alpha = 1 the limited step is the subcell FV
    update followed by a backward-Euler friction step per node, in closed
    form here (|m| + dt C_f |m|^2 / h^2 = |r|, positive root) instead of the
    oracle's Newton iteration."""
    from oracle.sources import ChezyFriction
    bs, x, dx = grid(N, 7, family=family)
    b = 0.1 * np.sin(2 * np.pi * x) ** 2
    u = np.stack([1.0 + 0.1 * np.cos(2 * np.pi * x) - b, 0.3 * np.sin(2 * np.pi * x)])
    sy = ShallowWater1D(G)
    Cf = 3.0
    sch = Scheme1D(sy, N, dx, family=family, source=ChezyFriction(Cf))
    dt = 0.2 * dx * np.min(bs.w) / 4.0
    got = Blending1D(sch, alpha=1.0).step(u, b, dt)
    h, r = subcell_fv(sy, u, b, bs.w, dx, dt)
    k = dt * Cf / (h * h)
    # the positive root without cancellation: 2 |r| / (1 + sqrt(1 + 4 k |r|))
    m = 2.0 * r / (1.0 + np.sqrt(1.0 + 4.0 * k * np.abs(r)))
    assert np.max(np.abs(got - np.stack([h, m]))) < 1e-14


def dam_break(N, E, hR=1e-3, family="gll"):
    bs, x, dx = grid(N, E, family=family)
    h = np.where((x > 0.25) & (x < 0.75), 1.0, hR)
    return bs, np.stack([h, np.zeros_like(h)]), np.zeros_like(h), dx


def test_dam_break_positive_and_conservative():
    """GLL nodes, so that the face states of u^n (at which the wave speed is
    taken) are nodal values and admissible; C_s = 0.2, so that the
    first-order scheme on the smallest subcell (w_0 dx = dx / 12) is
    positive, which needs lam dt <= w_0 dx / 2."""
    N, E = 3, 40
    bs, u, b, dx = dam_break(N, E)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family="gll")
    lim = Blending1D(sch)
    cfl = fourier.cfl_number(N, "gll", halvings=30)
    assert 0.2 * cfl <= 0.5 * bs.w[0]
    mass0 = np.sum(bs.w * u[0]) * dx
    v = u.copy()
    for _ in range(60):
        v = lim.step(v, b, sch.compute_dt(v, b, cfl, 0.2))
        assert np.min(v[0]) > 0.0
    assert abs(np.sum(bs.w * v[0]) * dx - mass0) < 1e-13
    assert np.max(lim.last_alpha) > 0.5 and np.min(lim.last_alpha) == 0.0
    # the unlimited step loses positivity on the same problem
    w = u.copy()
    lost = False
    with np.errstate(all="ignore"):
        for _ in range(60):
            w = sch.step(w, b, sch.compute_dt(w, b, cfl, 0.2))
            if not np.all(w[0] > 0.0):
                lost = True
                break
    assert lost


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator(N):
    bs, x, dx = grid(N, 20)
    # smooth, positive (like a depth: the mean mode dominates)
    assert np.all(hennemann_alpha(bs, 1.0 + 0.2 * np.sin(2 * np.pi * x)) == 0.0)
    # degree N - 2: the two highest modes vanish
    assert np.all(hennemann_alpha(bs, 1.0 + 0.5 * x ** (N - 2)) == 0.0)
    # a jump inside element 10 (between its first two nodes)
    a = hennemann_alpha(bs, np.where(x < 0.515, 1.0, 0.0), smooth=False)
    assert a[10] > 0.9 and np.all(a[:8] == 0.0) and np.all(a[13:] == 0.0)


@pytest.mark.parametrize("alpha,family", [(None, "gll"), (1.0, "gl"), (1.0, "gll"), (0.3, "gll")])
def test_well_balanced_lake_at_rest_with_limiter(alpha, family):
    """The blended face flux mixes B(w) at the u^n trace (high order) with B
    at the end node (low order).  With GLL nodes the two coincide and the
    limited well-balanced step keeps a lake at rest over a discontinuous
    bottom to round-off for any alpha; with GL nodes only alpha = 0 or 1
    does."""
    N, E = 3, 16
    bs, x, dx = grid(N, E, family=family)
    b = 0.3 * np.exp(-((x - 0.4) ** 2) / (2 * 0.05 ** 2)) + np.where(x > 0.7, 0.2, 0.0)
    u0 = np.stack([1.0 - b, np.zeros_like(b)])
    sch = Scheme1D(ShallowWater1DWB(G), N, dx, family=family)
    lim = Blending1D(sch, alpha=alpha, indicator_var=0)
    u = u0.copy()
    for _ in range(20):
        u = lim.step(u, b, 2e-3)
    assert np.max(np.abs(u - u0)) < 1e-13
    if alpha is None:
        assert np.max(lim.last_alpha) > 0.5


def test_advection_has_no_constraint_and_blends():
    N, E = 3, 20
    bs, x, dx = grid(N, E)
    a = 1.0 + 0.5 * np.sin(2 * np.pi * x)
    v = np.where((x > 0.215) & (x < 0.515), 1.0, 0.0)[None]
    sch = Scheme1D(VarCoeffAdvection(), N, dx)
    lim = Blending1D(sch)
    out = lim.step(v, a, 0.2 * fourier.cfl_number(N, halvings=30) * dx / 1.5)
    assert np.all(np.isfinite(out))
    assert np.max(lim.last_alpha) > 0.5
    # the limited step stays within the data's bounds more tightly than the
    # unlimited one
    plain = sch.step(v, a, 0.2 * fourier.cfl_number(N, halvings=30) * dx / 1.5)
    assert np.max(np.abs(out - 0.5)) < np.max(np.abs(plain - 0.5))


@pytest.mark.parametrize("N,family", [(N, f) for N in (1, 2, 3, 4) for f in ("gl", "gll")])
def test_modal_coefficients_of_single_modes(N, family):
    """The nodal values of the orthonormal Legendre mode j (on [0, 1] mapped to
    [-1, 1]) have the coefficient vector e_j, and the coefficients of any
    nodal data satisfy Parseval against a 12-point Gauss-Legendre integral of
    its interpolant (independent of the inverse Vandermonde)."""
    from oracle.limiter import legendre_orthonormal, modal_coefficients
    bs = Basis(N, family)
    for j in range(N + 1):
        X = legendre_orthonormal(j, 2.0 * bs.xi - 1.0)
        m = modal_coefficients(bs, X)
        e = np.zeros(N + 1)
        e[j] = 1.0
        assert np.max(np.abs(m - e)) < 1e-13
    rng = np.random.default_rng(N)
    X = rng.standard_normal(N + 1)
    m = modal_coefficients(bs, X)
    g, w = np.polynomial.legendre.leggauss(12)
    # Lagrange interpolant of X at the quadrature points of [-1, 1]
    xi = 2.0 * bs.xi - 1.0
    P = np.ones((12, N + 1))
    for k in range(N + 1):
        for l in range(N + 1):
            if l != k:
                P[:, k] *= (g - xi[l]) / (xi[k] - xi[l])
    assert abs(np.sum(m * m) - np.sum(w * (P @ X) ** 2)) < 1e-12 * np.sum(m * m)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator_energy_and_logistic_centre(N):
    """Mode N alone has energy 1 (alpha 1); the mean plus mode N scaled so
    that its energy share is exactly the threshold T(N) sits at the centre of
    the logistic map (alpha 1/2); the mean plus mode N-1 with share T of the
    modes below N also gives 1/2 (the second energy of the indicator)."""
    from oracle.limiter import legendre_orthonormal
    bs = Basis(N)
    xi = 2.0 * bs.xi - 1.0
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    mode = lambda j: legendre_orthonormal(j, xi)
    a = hennemann_alpha(bs, mode(N)[None, :], smooth=False)
    assert a[0] == 1.0
    r = np.sqrt(T / (1.0 - T))
    a = hennemann_alpha(bs, (mode(0) + r * mode(N))[None, :], smooth=False)
    assert a[0] == pytest.approx(0.5, abs=1e-9)
    a = hennemann_alpha(bs, (mode(0) + r * mode(N - 1))[None, :], smooth=False)
    assert a[0] == pytest.approx(0.5, abs=1e-9)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator_2d_mode_classes(N):
    """Tensor-product modes: P_i(y) P_j(x) with max(i, j) = N has energy 1 in
    the first class (alpha 1); the mean plus a mode with max(i, j) = N - 1 of
    share T among the modes below N sits at alpha 1/2; a mode with both
    degrees below N - 1 leaves alpha 0."""
    from oracle.limiter import hennemann_alpha_2d, legendre_orthonormal
    bs = Basis(N)
    xi = 2.0 * bs.xi - 1.0
    T = 0.5 * 10.0 ** (-1.8 * (N + 1) ** 0.25)
    m2 = lambda i, j: np.outer(legendre_orthonormal(i, xi), legendre_orthonormal(j, xi))
    one = lambda X: X[None, None]
    assert hennemann_alpha_2d(bs, one(m2(N, 0)), smooth=False)[0, 0] == 1.0
    assert hennemann_alpha_2d(bs, one(m2(1, N)), smooth=False)[0, 0] == 1.0
    r = np.sqrt(T / (1.0 - T))
    X = m2(0, 0) + r * m2(N - 1, N - 2 if N >= 2 else 0)
    assert hennemann_alpha_2d(bs, one(X), smooth=False)[0, 0] == pytest.approx(0.5, abs=1e-9)
    if N >= 3:
        X = m2(0, 0) + 0.5 * m2(N - 2, N - 2)
        assert hennemann_alpha_2d(bs, one(X), smooth=False)[0, 0] == 0.0
