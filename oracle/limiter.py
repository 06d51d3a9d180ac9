"""Subcell blending limiter with admissibility preservation, 1D and its
tensor-product 2D extension (test infrastructure only).

Sec. 4 of the paper, in its order:

  u^{n+1}_e = (1 - alpha_e) u^{H,n+1}_e + alpha_e u^{L,n+1}_e
                                               (Eq. blended.scheme)
  u^L: first-order finite volumes on the N+1 subcells of element e, subcell p
       of width w_p dx (Eq. subcell.defn), with the non-conservative Rusanov
       fluxes f^{num,+-}(u_{e,p}, u_{e,p+1}) of Eq. combined.num.flux at the
       inner subfaces (Eq. numflux.args) and the source implicitly
       (Eq. low.order.update);
  at element faces both schemes use
       F^{+-} = (1 - alpha_{e+1/2}) F^{HO,+-} + alpha_{e+1/2} f^{num,+-}(u_{e,N}, u_{e+1,0}),
       alpha_{e+1/2} = (alpha_e + alpha_{e+1}) / 2          (Eq. Fblend),
  limited by Algorithm 1 so that the two low-order updates next to the face
  stay admissible, and finally Algorithm 2 limits alpha_e per element so that
  every node is admissible.

F^{HO,+-} is the cRK-FR time-averaged numerical flux F^num + B(w^{n,+-}) W^num
(Eqs. numflux.cons, good.numflux.non.cons).  With alpha = 0 everywhere and
no admissibility violation the step is the plain cRK-FR step.

The admissibility constraints of a system are ``admissibility`` (a list of
functions P(u), admissible if P > 0); shallow water: h.  theta follows
Eq. theta.formula for these linear (concave) constraints, applied when the
candidate state has P below epsilon; epsilon is a tenth of P at the
low-order state (the factor the paper takes).

The smoothness indicator alpha_e is the one of Hennemann et al. (2021) that
the paper refers to, restated here: the modal energy in the highest (and
second highest) orthonormal Legendre mode of an indicator variable, mapped
through a logistic function around the threshold a 10^(-c (N+1)^(1/4)),
a = 0.5, c = 1.8, sharpness s = ln((1 - 1e-4) / 1e-4), values below
alpha_min = 1e-3 set to 0 and above 1 - alpha_min to 1, capped at
alpha_max, then raised to half the neighbours' values.
"""
import numpy as np

from .crkfr import face_fluxes
from .sources import point_implicit_solve


# ----------------------------------------------------------------------------
# smoothness indicator
# ----------------------------------------------------------------------------
def legendre_orthonormal(j, x):
    """sqrt((2j+1)/2) P_j(x) on [-1, 1] (three-term recurrence)."""
    p0, p1 = np.ones_like(x), x
    if j == 0:
        return np.sqrt(0.5) * p0
    for k in range(1, j):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    return np.sqrt((2 * j + 1) / 2.0) * p1


def modal_coefficients(basis, X):
    """Coefficients of the nodal values X[..., p] in the orthonormal Legendre
    basis of [0, 1] mapped to [-1, 1] (inverse Vandermonde)."""
    n = len(basis.xi)
    V = np.stack([legendre_orthonormal(j, 2.0 * basis.xi - 1.0) for j in range(n)], axis=1)
    return np.einsum("jp,...p->...j", np.linalg.inv(V), X)


def hennemann_alpha(basis, X, a=0.5, c=1.8, alpha_min=1e-3, alpha_max=1.0, smooth=True):
    """alpha_e from the nodal indicator variable X[e, p] (periodic mesh)."""
    N = len(basis.xi) - 1
    m = modal_coefficients(basis, X)
    tot = np.sum(m * m, axis=-1)
    e1 = np.where(tot > 0.0, m[..., N] ** 2 / np.where(tot > 0.0, tot, 1.0), 0.0)
    if N >= 2:
        tot2 = np.sum(m[..., :N] ** 2, axis=-1)
        e2 = np.where(tot2 > 0.0, m[..., N - 1] ** 2 / np.where(tot2 > 0.0, tot2, 1.0), 0.0)
        energy = np.maximum(e1, e2)
    else:
        energy = e1
    T = a * 10.0 ** (-c * (N + 1) ** 0.25)
    s = np.log((1.0 - 1e-4) / 1e-4)
    alpha = 1.0 / (1.0 + np.exp(-s / T * (energy - T)))
    alpha = np.where(alpha < alpha_min, 0.0, alpha)
    alpha = np.where(alpha > 1.0 - alpha_min, 1.0, alpha)
    alpha = np.minimum(alpha, alpha_max)
    if smooth:
        alpha = np.maximum(alpha, 0.5 * np.maximum(np.roll(alpha, 1), np.roll(alpha, -1)))
    return alpha


# ----------------------------------------------------------------------------
# first-order fluxes (Eq. combined.num.flux)
# ----------------------------------------------------------------------------
def low_order_fluxes(sy, uL, uR, cL, cR):
    """f^{num,-}, f^{num,+} between states uL (left) and uR (right):
    (f(uL) + f(uR))/2 - lam/2 (uR - uL) + B(w_-+) (wL + wR)/2, lam the larger
    spectral radius; the dissipated jump is the system's ``dissipated`` state
    if it has one."""
    lam = np.maximum(sy.speed(uL, cL), sy.speed(uR, cR))
    diss = getattr(sy, "dissipated", None)
    jump = (uR - uL) if diss is None else diss(uR, cR) - diss(uL, cL)
    f = 0.5 * (sy.flux(uL, cL) + sy.flux(uR, cR)) - 0.5 * lam * jump
    u_num, c_num = 0.5 * (uL + uR), 0.5 * (cL + cR)
    return f + sy.ncprod(uL, cL, u_num, c_num), f + sy.ncprod(uR, cR, u_num, c_num)


def theta_linear(P, eps, ua, ub):
    """Weight of the candidate ub in theta ub + (1 - theta) ua so that the
    linear constraint P reaches eps (Eq. theta.formula); 1 where P(ub) >= eps."""
    Pa, Pb = P(ua), P(ub)
    den = np.where(Pb - Pa != 0.0, Pb - Pa, 1.0)
    th = np.minimum(1.0, np.abs((eps - Pa) / den))
    return np.where(Pb < eps, th, 1.0)


# ----------------------------------------------------------------------------
# blended step
# ----------------------------------------------------------------------------
class Blending1D:
    """Blended cRK-FR / subcell FV step of a Scheme1D (frozen face reading).

    ``alpha``: None (the indicator on ``indicator_var``), a number or an
    array (E,) to force the blending coefficients (for the pins)."""

    def __init__(self, scheme, alpha=None, indicator_var=0, admissible=True):
        self.sch = scheme
        self.alpha = alpha
        self.var = indicator_var
        self.admissible = admissible

    def coefficients(self, u, c):
        E = u.shape[-2]
        if self.alpha is None:
            return hennemann_alpha(self.sch.basis, u[self.var])
        return np.broadcast_to(np.asarray(self.alpha, dtype=float), (E,)).copy()

    def step(self, u, c, dt):
        sch, bs = self.sch, self.sch.basis
        sy = sch.sys
        N = len(bs.xi) - 1
        dx = sch.dx
        alpha = self.coefficients(u, c)
        constraints = getattr(sy, "admissibility", []) if self.admissible else []

        # high-order element-local part and face fluxes (face k: elements k-1 | k)
        loc = sch.local(u, c, dt)
        r = lambda X: np.roll(X, 1, axis=-1)
        Fho_m, Fho_p, Ft_m, Ft_p, _ = face_fluxes(
            r(loc["F_r"]), loc["F_l"], r(loc["U_r"]), loc["U_l"], r(loc["un_r"]), loc["un_l"],
            r(loc["c_r"]), loc["c_l"], sy.speed, sy.ncprod, dissipated=getattr(sy, "dissipated", None))

        # first-order fluxes: element faces (node N of k-1 | node 0 of k) and
        # the inner subfaces of every element (node p | node p+1)
        fo_m, fo_p = low_order_fluxes(sy, r(u[..., N]), u[..., 0], r(c[..., N]), c[..., 0])
        fi_m, fi_p = low_order_fluxes(sy, u[..., :-1], u[..., 1:], c[..., :-1], c[..., 1:])

        # Eq. Fblend
        af = 0.5 * (r(alpha) + alpha)
        F_m = (1.0 - af) * Fho_m + af * fo_m
        F_p = (1.0 - af) * Fho_p + af * fo_p

        w = bs.w
        # Algorithm 1 at every face k
        if constraints:
            u0, uN = u[..., 0], r(u[..., N])
            f0_inner = fi_m[..., 0]            # right flux of node 0 of element k
            fN_inner = r(fi_p[..., N - 1])     # left flux of node N of element k-1
            c0 = dt / (w[0] * dx)
            cN = dt / (w[N] * dx)
            low0 = u0 - c0 * (f0_inner - fo_p)
            lowN = uN - cN * (fo_m - fN_inner)
            for P in constraints:
                t0 = u0 - c0 * (f0_inner - F_p)
                tN = uN - cN * (F_m - fN_inner)
                th = np.minimum(theta_linear(P, 0.1 * P(low0), low0, t0),
                                theta_linear(P, 0.1 * P(lowN), lowN, tN))
                F_m = th * F_m + (1.0 - th) * fo_m
                F_p = th * F_p + (1.0 - th) * fo_p

        # high-order update with the face fluxes F (Eq. crkfr.non.cons.final)
        T_right = np.roll(F_m - Ft_m, -1, axis=-1)
        T_left = F_p - Ft_p
        RH = loc["vol"] + (T_right[..., None] * bs.gRp + T_left[..., None] * bs.gLp) / dx
        uH = u - dt * RH

        # low-order update (Eq. low.order.update)
        right = np.concatenate([fi_m, np.roll(F_m, -1, axis=-1)[..., None]], axis=-1)
        left = np.concatenate([F_p[..., None], fi_p], axis=-1)
        uL = u - dt / (w * dx) * (right - left)
        if sch.source is not None:
            uL = point_implicit_solve(sch.source, uL, c, dt)

        # Eq. blended.scheme, then Algorithm 2 per element
        out = (1.0 - alpha)[:, None] * uH + alpha[:, None] * uL
        for P in constraints:
            eps = 0.1 * np.min(P(uL), axis=-1, keepdims=True)
            th = np.min(theta_linear(P, eps, uL, out), axis=-1)
            out = th[:, None] * out + (1.0 - th)[:, None] * uL
        self.last_alpha = alpha
        return out


# ----------------------------------------------------------------------------
# 2D (tensor-product subcells)
# ----------------------------------------------------------------------------
def hennemann_alpha_2d(basis, X, a=0.5, c=1.8, alpha_min=1e-3, alpha_max=1.0, smooth=True):
    """alpha per element from the nodal indicator variable X[ey, ex, q, p]
    (periodic mesh): the tensor-product modal coefficients m_ij; the energy
    share of the modes with i = N or j = N, and (N >= 2) of those with
    max(i, j) = N - 1 among the modes below N; the same logistic map as in
    1D; smoothing with half the largest of the four face neighbours."""
    N = len(basis.xi) - 1
    n = N + 1
    V = np.stack([legendre_orthonormal(j, 2.0 * basis.xi - 1.0) for j in range(n)], axis=1)
    Vi = np.linalg.inv(V)
    m = np.einsum("iq,jp,...qp->...ij", Vi, Vi, X)
    m2 = m * m
    tot = np.sum(m2, axis=(-2, -1))
    clip1 = np.sum(m2[..., :N, :N], axis=(-2, -1))
    e1 = np.where(tot > 0.0, (tot - clip1) / np.where(tot > 0.0, tot, 1.0), 0.0)
    if N >= 2:
        clip2 = np.sum(m2[..., :N - 1, :N - 1], axis=(-2, -1))
        e2 = np.where(clip1 > 0.0, (clip1 - clip2) / np.where(clip1 > 0.0, clip1, 1.0), 0.0)
        energy = np.maximum(e1, e2)
    else:
        energy = e1
    T = a * 10.0 ** (-c * (N + 1) ** 0.25)
    s = np.log((1.0 - 1e-4) / 1e-4)
    alpha = 1.0 / (1.0 + np.exp(-s / T * (energy - T)))
    alpha = np.where(alpha < alpha_min, 0.0, alpha)
    alpha = np.where(alpha > 1.0 - alpha_min, 1.0, alpha)
    alpha = np.minimum(alpha, alpha_max)
    if smooth:
        nb = np.maximum(np.maximum(np.roll(alpha, 1, 0), np.roll(alpha, -1, 0)),
                        np.maximum(np.roll(alpha, 1, 1), np.roll(alpha, -1, 1)))
        alpha = np.maximum(alpha, 0.5 * nb)
    return alpha


class _Dir:
    """The x or y direction of a 2D system, seen as a 1D system for the
    first-order fluxes."""

    def __init__(self, sy, d):
        self.flux = sy.flux_x if d == 0 else sy.flux_y
        self.ncprod = sy.ncprod_x if d == 0 else sy.ncprod_y
        self.speed = sy.speed_x if d == 0 else sy.speed_y
        if hasattr(sy, "dissipated"):
            self.dissipated = sy.dissipated


class Blending2D:
    """Blended cRK-FR / subcell FV step of a Scheme2D, the tensor-product
    extension of Sec. 4 (reading): subcells of w_p dx x w_q dy, first-order
    fluxes of Eq. combined.num.flux across every x- and y-subface, Eq. Fblend
    per face node.  The first-order update splits as
        u^L = 1/2 (u - 2 dt/(w_p dx) dx-differences) + 1/2 (u - 2 dt/(w_q dy) dy-differences),
    so Algorithm 1 limits each face's flux so that the doubled-dt
    one-direction updates of its two adjacent nodes stay admissible (their
    average then is); Algorithm 2 acts per element on all n^2 nodes."""

    def __init__(self, scheme, alpha=None, indicator_var=0, admissible=True):
        self.sch = scheme
        self.alpha = alpha
        self.var = indicator_var
        self.admissible = admissible

    def coefficients(self, u, c):
        if self.alpha is None:
            return hennemann_alpha_2d(self.sch.basis, u[self.var])
        return np.broadcast_to(np.asarray(self.alpha, dtype=float), u.shape[1:3]).copy()

    def step(self, u, c, dt):
        sch, bs = self.sch, self.sch.basis
        sy = sch.sys
        N = len(bs.xi) - 1
        w = bs.w
        alpha = self.coefficients(u, c)
        constraints = getattr(sy, "admissibility", []) if self.admissible else []
        diss = getattr(sy, "dissipated", None)
        loc = sch.local(u, c, dt)
        rx = lambda X: np.roll(X, 1, axis=-2)   # element (ey, ex-1) of trace arrays (.., ey, ex, n)
        ry = lambda X: np.roll(X, 1, axis=-3)   # element (ey-1, ex)
        dirs = (_Dir(sy, 0), _Dir(sy, 1))

        # high-order face fluxes: x-face (ey, k) between (ey, k-1) | (ey, k),
        # y-face (k, ex) between (k-1, ex) | (k, ex); one value per face node
        Hx = face_fluxes(rx(loc["F_r"]), loc["F_l"], rx(loc["U_r"]), loc["U_l"], rx(loc["un_r"]),
                         loc["un_l"], rx(loc["c_r"]), loc["c_l"], sy.speed_x, sy.ncprod_x,
                         dissipated=diss)
        Hy = face_fluxes(ry(loc["G_t"]), loc["G_b"], ry(loc["U_t"]), loc["U_b"], ry(loc["un_t"]),
                         loc["un_b"], ry(loc["c_t"]), loc["c_b"], sy.speed_y, sy.ncprod_y,
                         dissipated=diss)
        # first-order fluxes at element faces (nodal values next to the face)
        # and across the inner subfaces
        ex_ = lambda X, p: X[..., :, p]            # column p of every element: (.., ey, ex, q)
        ey_ = lambda X, q: X[..., q, :]            # row q: (.., ey, ex, p)
        fxo = low_order_fluxes(dirs[0], rx(ex_(u, N)), ex_(u, 0), rx(ex_(c, N)), ex_(c, 0))
        fyo = low_order_fluxes(dirs[1], ry(ey_(u, N)), ey_(u, 0), ry(ey_(c, N)), ey_(c, 0))
        fxi = low_order_fluxes(dirs[0], u[..., :, :-1], u[..., :, 1:], c[..., :, :-1], c[..., :, 1:])
        fyi = low_order_fluxes(dirs[1], u[..., :-1, :], u[..., 1:, :], c[..., :-1, :], c[..., 1:, :])

        # Eq. Fblend
        ax = (0.5 * (np.roll(alpha, 1, axis=1) + alpha))[..., None]
        ay = (0.5 * (np.roll(alpha, 1, axis=0) + alpha))[..., None]
        Fx = [(1.0 - ax) * Hx[k] + ax * fxo[k] for k in (0, 1)]
        Fy = [(1.0 - ay) * Hy[k] + ay * fyo[k] for k in (0, 1)]

        # Algorithm 1 with doubled-dt one-direction updates
        for P in constraints:
            for F, fo, fi, width, d in ((Fx, fxo, fxi, sch.dx, 0), (Fy, fyo, fyi, sch.dy, 1)):
                if d == 0:
                    u0, uN = ex_(u, 0), rx(ex_(u, N))
                    f0_in = fi[0][..., :, 0]                 # right flux of node p = 0
                    fN_in = rx(fi[1][..., :, N - 1])         # left flux of node p = N of (ey, ex-1)
                else:
                    u0, uN = ey_(u, 0), ry(ey_(u, N))
                    f0_in = fi[0][..., 0, :]
                    fN_in = ry(fi[1][..., N - 1, :])
                c0 = 2.0 * dt / (w[0] * width)
                cN = 2.0 * dt / (w[N] * width)
                low0 = u0 - c0 * (f0_in - fo[1])
                lowN = uN - cN * (fo[0] - fN_in)
                t0 = u0 - c0 * (f0_in - F[1])
                tN = uN - cN * (F[0] - fN_in)
                th = np.minimum(theta_linear(P, 0.1 * P(low0), low0, t0),
                                theta_linear(P, 0.1 * P(lowN), lowN, tN))
                F[0] = th * F[0] + (1.0 - th) * fo[0]
                F[1] = th * F[1] + (1.0 - th) * fo[1]

        # high-order update with the face fluxes (corrections of Scheme2D)
        Tx_m, Tx_p = Fx[0] - Hx[2], Fx[1] - Hx[3]
        Ty_m, Ty_p = Fy[0] - Hy[2], Fy[1] - Hy[3]
        Tr = np.roll(Tx_m, -1, axis=-2)
        Tt = np.roll(Ty_m, -1, axis=-3)
        uH = u - dt * (loc["vol"] + sch._corrections(Tr, Tx_p, Tt, Ty_p))

        # first-order update
        right = np.concatenate([fxi[0], np.roll(Fx[0], -1, axis=-2)[..., :, None]], axis=-1)
        left = np.concatenate([Fx[1][..., :, None], fxi[1]], axis=-1)
        top = np.concatenate([fyi[0], np.roll(Fy[0], -1, axis=-3)[..., None, :]], axis=-2)
        bottom = np.concatenate([Fy[1][..., None, :], fyi[1]], axis=-2)
        uL = (u - dt / (w[None, :] * sch.dx) * (right - left)
              - dt / (w[:, None] * sch.dy) * (top - bottom))
        if sch.source is not None:
            uL = point_implicit_solve(sch.source, uL, c, dt)

        # Eq. blended.scheme and Algorithm 2 per element
        a4 = alpha[..., None, None]
        out = (1.0 - a4) * uH + a4 * uL
        for P in constraints:
            eps = 0.1 * np.min(P(uL), axis=(-2, -1), keepdims=True)
            th = np.min(theta_linear(P, eps, uL, out), axis=(-2, -1))[..., None, None]
            out = th * out + (1.0 - th) * uL
        self.last_alpha = alpha
        return out
