"""Pins of the oracle's 2D subcell blending limiter (the tensor-product
extension of Sec. 4; readings in oracle.limiter.Blending2D):

- alpha = 0 is the plain 2D cRK-FR step, bit for bit;
- alpha = 1 is first-order finite volumes on the 2D subcell grid (cells
  w_p dx x w_q dy, written out independently here);
- on y-invariant smooth data the 2D limited step equals the 1D limited step
  on every row (h, hu; hv stays zero for alpha 0 or 1 and conserved
  otherwise);
- a circular dam break onto a thin layer stays positive and conserves mass;
- the 2D indicator vanishes on smooth data and on polynomials of degree
  N - 2 in each variable, and is near 1 at a jump;
- the well-balanced form with the limiter keeps a lake at rest (GLL).
"""
import numpy as np
import pytest

from oracle import fourier
from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.limiter import Blending1D, Blending2D, hennemann_alpha_2d
from oracle.systems import ShallowWater1D, ShallowWater2D, ShallowWater2DWB

G = 9.81


def grid(N, Ex, Ey, family="gl"):
    bs = Basis(N, family)
    dx, dy = 1.0 / Ex, 1.0 / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    return bs, x, y, dx, dy


def flow(x, y):
    b = 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u = np.stack([1.2 - b + 0.05 * np.sin(2 * np.pi * (x + y)), 0.2 * np.cos(2 * np.pi * y),
                  0.1 * np.sin(2 * np.pi * x)])
    return u, b


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll"), (3, "gl")])
def test_alpha_zero_is_the_plain_2d_step(N, family):
    bs, x, y, dx, dy = grid(N, 5, 4, family)
    u, b = flow(x, y)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family)
    dt = sch.compute_dt(u, b, fourier.cfl_number(N, family, halvings=30), 0.5)
    assert np.array_equal(Blending2D(sch, alpha=0.0).step(u, b, dt), sch.step(u, b, dt))


def subcell_fv_2d(sy, u, c, w, dx, dy, dt):
    """First-order FV on the global grid of subcells, written out with the
    fluxes of Eq. combined.num.flux in each direction."""
    M, Ey, Ex, n, _ = u.shape
    U = u.transpose(0, 1, 3, 2, 4).reshape(M, Ey * n, Ex * n)     # [var, global row, global col]
    C = c.transpose(0, 2, 1, 3).reshape(Ey * n, Ex * n)
    Wx = np.tile(w, Ex) * dx
    Wy = np.tile(w, Ey) * dy
    out = U.copy()
    R, K = U.shape[1], U.shape[2]
    for r in range(R):
        for k in range(K):
            for d, (r2, k2), width in ((0, (r, (k + 1) % K), Wx), (1, ((r + 1) % R, k), Wy)):
                uL, uR, cL, cR = U[:, r, k], U[:, r2, k2], C[r, k], C[r2, k2]
                flux = sy.flux_x if d == 0 else sy.flux_y
                nc = sy.ncprod_x if d == 0 else sy.ncprod_y
                speed = sy.speed_x if d == 0 else sy.speed_y
                lam = max(speed(uL, cL), speed(uR, cR))
                f = 0.5 * (flux(uL, cL) + flux(uR, cR)) - 0.5 * lam * (uR - uL)
                un, cn = 0.5 * (uL + uR), 0.5 * (cL + cR)
                iL = k if d == 0 else r
                iR = k2 if d == 0 else r2
                out[:, r, k] -= dt / width[iL] * (f + nc(uL, cL, un, cn))
                out[:, r2, k2] += dt / width[iR] * (f + nc(uR, cR, un, cn))
    return out.reshape(M, Ey, n, Ex, n).transpose(0, 1, 3, 2, 4)


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll")])
def test_alpha_one_is_2d_subcell_finite_volumes(N, family):
    bs, x, y, dx, dy = grid(N, 3, 2, family)
    u, b = flow(x, y)
    sy = ShallowWater2D(G)
    sch = Scheme2D(sy, N, dx, dy, family=family)
    dt = 0.05 * min(dx, dy) * np.min(bs.w) / 4.0
    got = Blending2D(sch, alpha=1.0).step(u, b, dt)
    want = subcell_fv_2d(sy, u, b, bs.w, dx, dy, dt)
    assert np.max(np.abs(got - want)) < 1e-14


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
def test_y_invariant_data_matches_1d_limiter(alpha):
    N, Ex, Ey = 3, 8, 3
    bs, x, y, dx, dy = grid(N, Ex, Ey)
    b = 0.1 * np.sin(2 * np.pi * x) ** 2
    h = 1.0 + 0.1 * np.cos(2 * np.pi * x) - b
    u = np.stack([h, 0.3 * np.sin(2 * np.pi * x), np.zeros_like(h)])
    sch2 = Scheme2D(ShallowWater2D(G), N, dx, dy)
    dt = 0.5 * fourier.cfl_number(N, halvings=30) * dx / (0.5 + np.sqrt(G * 1.2))
    got = Blending2D(sch2, alpha=alpha).step(u, b, dt)
    sch1 = Scheme1D(ShallowWater1D(G), N, dx)
    want = Blending1D(sch1, alpha=alpha).step(u[:2, 0, :, 0, :], b[0, :, 0, :], dt)
    for v in range(2):
        assert np.max(np.abs(got[v] - want[v][None, :, None, :])) < 1e-13
    if alpha in (0.0, 1.0):
        assert np.max(np.abs(got[2])) < 1e-13
    else:
        # the blended y-face flux of hv mixes the time-averaged pressure (high
        # order) with the pressure at t^n (first order), so hv moves by O(dt)
        # inside each element, with zero total (conservation)
        W = dx * dy * bs.w[:, None] * bs.w[None, :]
        assert np.max(np.abs(got[2])) < 1e-3
        assert abs(np.sum(W * got[2])) < 1e-15


def test_circular_dam_break_positive_and_conservative():
    N, E = 3, 12
    bs, x, y, dx, dy = grid(N, E, E, "gll")
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    h = np.where(r2 < 0.2 ** 2, 1.0, 1e-3)
    u = np.stack([h, np.zeros_like(h), np.zeros_like(h)])
    b = np.zeros_like(h)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    cfl = fourier.cfl_number(N, "gll", halvings=30)
    W = dx * dy * bs.w[:, None] * bs.w[None, :]
    m0 = np.sum(W * u[0])
    v = u.copy()
    for _ in range(15):
        v = lim.step(v, b, sch.compute_dt(v, b, cfl, 0.1))
        assert np.min(v[0]) > 0.0
    assert abs(np.sum(W * v[0]) - m0) < 1e-13
    assert np.max(lim.last_alpha) > 0.5


@pytest.mark.parametrize("N", [3, 4])
def test_indicator_2d(N):
    bs, x, y, dx, dy = grid(N, 10, 8)
    assert np.all(hennemann_alpha_2d(bs, 1.0 + 0.2 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)) == 0.0)
    assert np.all(hennemann_alpha_2d(bs, 1.0 + 0.5 * x ** (N - 2) * y ** (N - 2)) == 0.0)
    a = hennemann_alpha_2d(bs, np.where(x < 0.515, 1.0, 0.0), smooth=False)
    assert np.all(a[:, 5] > 0.9) and np.all(a[:, :4] == 0.0) and np.all(a[:, 7:] == 0.0)


@pytest.mark.parametrize("alpha,Cf", [(None, 0.0), (0.4, 0.0), (None, 2.0)])
def test_well_balanced_lake_at_rest_with_2d_limiter(alpha, Cf):
    from oracle.sources import ChezyFriction
    N = 3
    bs, x, y, dx, dy = grid(N, 6, 5, "gll")
    b = 0.3 * np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2) / (2 * 0.08 ** 2)) + np.where(x > 0.7, 0.2, 0.0)
    u0 = np.stack([1.0 - b, np.zeros_like(b), np.zeros_like(b)])
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy, family="gll",
                   source=ChezyFriction(Cf) if Cf else None)
    lim = Blending2D(sch, alpha=alpha)
    u = u0.copy()
    for _ in range(8):
        u = lim.step(u, b, 1e-3)
    assert np.max(np.abs(u - u0)) < 1e-13


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll")])
def test_alpha_one_with_friction_is_fv_then_backward_euler(N, family):
    """With Chezy friction and alpha = 1 the limited step is the first-order
    subcell FV update followed by a backward-Euler friction step per node,
    here in closed form (m parallel to the FV momentum r, |m| the positive
    root of |m| + dt C_f |m|^2 / h^2 = |r|) instead of the oracle's Newton
    iteration."""
    from oracle.sources import ChezyFriction
    bs, x, y, dx, dy = grid(N, 3, 2, family)
    u, b = flow(x, y)
    sy = ShallowWater2D(G)
    Cf = 2.0
    sch = Scheme2D(sy, N, dx, dy, family=family, source=ChezyFriction(Cf))
    dt = 0.05 * min(dx, dy) * np.min(bs.w) / 4.0
    got = Blending2D(sch, alpha=1.0).step(u, b, dt)
    fv = subcell_fv_2d(sy, u, b, bs.w, dx, dy, dt)
    h, rx, ry = fv
    nr = np.sqrt(rx * rx + ry * ry)
    k = dt * Cf / (h * h)
    f = 2.0 / (1.0 + np.sqrt(1.0 + 4.0 * k * nr))   # |m| / |r|, without cancellation
    want = np.stack([h, rx * f, ry * f])
    assert np.max(np.abs(got - want)) < 1e-13
