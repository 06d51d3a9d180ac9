"""Physical systems u_t + f(u)_x [+ g(u)_y] + B(w) grad w = 0 with a static
coefficient field c (test infrastructure only).

Sec. 3, Eq. flux.and.non.cons; Sec. 5.1.3 (variable-coefficient advection cast
with B depending on the coefficient, "B(u, x)"); Sec. 5, Eq. time.step.2d for
the 2D form.  The state is w = (u, c) where u holds the M evolved variables
and c the static coefficient (a(x) for advection, the bathymetry b(x) for
shallow water).  ``ncprod(u, c, du, dc)`` returns the M evolved rows of the
matrix-vector product B(w) (du, dc); the row of c is zero because c is static.

Array convention: the variable index is the leading axis of ``u``/``du``;
``c``/``dc`` have no variable axis.
"""
import numpy as np  # noqa: F401  (constants)

from .xp import xp_of


class VarCoeffAdvection:
    """v_t + a(x) v_x = 0 (Sec. 5.1.3, Eq. var.coeff.adv): u = (v), c = a,
    f = 0, B(w)(du, dc) = a du, spectral radius of f' + B is |a|."""
    M = 1
    name = "varadv"

    def flux(self, u, c):
        return xp_of(u).zeros_like(u)

    def ncprod(self, u, c, du, dc):
        return c[None] * du

    def speed(self, u, c):
        xp = xp_of(u, c)
        return xp.abs(c) * xp.ones_like(u[0])


class ShallowWater1D:
    """Shallow water with bathymetry as a non-conservative product:
    h_t + m_x = 0,  m_t + (m^2/h + g h^2/2)_x + g h b_x = 0.
    u = (h, m), c = b, f = (m, m^2/h + g h^2/2), B(w)(du, db) = (0, g h db).
    Eigenvalues of f' + B on (h, m, b): v - sqrt(g h), 0, v + sqrt(g h)
    with v = m / h, so the spectral radius is |v| + sqrt(g h)."""
    M = 2
    name = "swe1d"
    # admissibility constraints P(u) > 0 (Sec. 2, Eq. uad.form): h > 0
    admissibility = [lambda u: u[0]]

    def __init__(self, g=9.81):
        self.g = g

    def flux(self, u, c):
        h, m = u[0], u[1]
        return xp_of(u).stack([m, m * m / h + 0.5 * self.g * h * h])

    def ncprod(self, u, c, du, dc):
        xp = xp_of(u, dc)
        h = u[0]
        return xp.stack([xp.zeros_like(h * dc), self.g * h * dc])

    def speed(self, u, c):
        xp = xp_of(u)
        h, m = u[0], u[1]
        return xp.abs(m / h) + xp.sqrt(self.g * h)


class ShallowWater2D:
    """2D shallow water with bathymetry: u = (h, hu, hv), c = b,
    f = (hu, (hu)^2/h + g h^2/2, (hu)(hv)/h),
    g = (hv, (hu)(hv)/h, (hv)^2/h + g h^2/2),
    B1(w)(du, db) = (0, g h db, 0), B2(w)(du, db) = (0, 0, g h db).
    Spectral radii: |u| + sqrt(g h) in x, |v| + sqrt(g h) in y."""
    M = 3
    name = "swe2d"
    admissibility = [lambda u: u[0]]

    def __init__(self, g=9.81):
        self.g = g

    def flux_x(self, u, c):
        h, mx, my = u[0], u[1], u[2]
        p = 0.5 * self.g * h * h
        return xp_of(u).stack([mx, mx * mx / h + p, mx * my / h])

    def flux_y(self, u, c):
        h, mx, my = u[0], u[1], u[2]
        p = 0.5 * self.g * h * h
        return xp_of(u).stack([my, mx * my / h, my * my / h + p])

    def ncprod_x(self, u, c, du, dc):
        xp = xp_of(u, dc)
        h = u[0]
        z = xp.zeros_like(h * dc)
        return xp.stack([z, self.g * h * dc, z])

    def ncprod_y(self, u, c, du, dc):
        xp = xp_of(u, dc)
        h = u[0]
        z = xp.zeros_like(h * dc)
        return xp.stack([z, z, self.g * h * dc])

    def speed_x(self, u, c):
        xp = xp_of(u)
        h, mx = u[0], u[1]
        return xp.abs(mx / h) + xp.sqrt(self.g * h)

    def speed_y(self, u, c):
        xp = xp_of(u)
        h, my = u[0], u[2]
        return xp.abs(my / h) + xp.sqrt(self.g * h)


class ShallowWater1DWB(ShallowWater1D):
    """Well-balanced form of 1D shallow water (the variant the paper lists as
    open, Sec. 6): the hydrostatic pressure moves into the non-conservative
    product,
        h_t + m_x = 0,  m_t + (m^2/h)_x + g h (h + b)_x = 0,
    u = (h, m), c = b, f = (m, m^2/h), B(w)(du, db) = (0, g h (du_h + db)).
    f' + B has the same eigenvalues as before (v -+ sqrt(g h)), and the
    Rusanov dissipation of the h equation acts on the free surface
    eta = h + b (``dissipated``), so that a lake at rest (m = 0, eta
    constant) has no local, flux, dissipation or fluctuation term."""
    name = "swe1d_wb"

    def flux(self, u, c):
        h, m = u[0], u[1]
        return xp_of(u).stack([m, m * m / h])

    def ncprod(self, u, c, du, dc):
        xp = xp_of(u, du)
        h = u[0]
        return xp.stack([xp.zeros_like(h * dc), self.g * h * (du[0] + dc)])

    def dissipated(self, U, c):
        return xp_of(U).stack([U[0] + c, U[1]])


class ShallowWater2DWB(ShallowWater2D):
    """Well-balanced form of 2D shallow water: pressure in the products,
    B1(w)(du, db) = (0, g h (du_h + db), 0), B2(w)(du, db) = (0, 0,
    g h (du_h + db)), f = (hu, (hu)^2/h, (hu)(hv)/h), g = (hv, (hu)(hv)/h,
    (hv)^2/h); dissipation of the h equation on eta = h + b."""
    name = "swe2d_wb"

    def flux_x(self, u, c):
        h, mx, my = u[0], u[1], u[2]
        return xp_of(u).stack([mx, mx * mx / h, mx * my / h])

    def flux_y(self, u, c):
        h, mx, my = u[0], u[1], u[2]
        return xp_of(u).stack([my, mx * my / h, my * my / h])

    def ncprod_x(self, u, c, du, dc):
        xp = xp_of(u, du)
        h = u[0]
        z = xp.zeros_like(h * dc)
        return xp.stack([z, self.g * h * (du[0] + dc), z])

    def ncprod_y(self, u, c, du, dc):
        xp = xp_of(u, du)
        h = u[0]
        z = xp.zeros_like(h * dc)
        return xp.stack([z, z, self.g * h * (du[0] + dc)])

    def dissipated(self, U, c):
        return xp_of(U).stack([U[0] + c, U[1], U[2]])
