"""cRK-FR step for non-conservative systems, 1D and 2D (test infrastructure only).

Follows Sec. 3 in the paper's order:

  inner stages  u^(i) = u^n - dt sum_{j<i} a_ij (dloc f(u^(j)) + B(w^(j)) dloc w^(j))
                (Eq. crkfr.non.cons.final, first line; dloc from Eq. dlocx.defn)
  time averages F = sum_j b_j f(u^(j))           (Eq. disc.avg.flux)
                U = sum_j b_j u^(j)              (Eq. time.avg.soln)
                Bloc = sum_j b_j B(w^(j)) dloc w^(j)   (Eq. local.time.avg.non.cons)
  face fluxes   F^num = (F^- + F^+)/2 - lam/2 (U^+ - U^-)   (Eq. numflux.cons)
                lam = max over the two sides of sigma(f' + B)  (Eq. combined.wave.speed)
                F^num,nc,+- = B(w^{n,+-}) W^num              (Eq. good.numflux.non.cons)
                F^tot,+- = F^+- + F^nc,+-                    (Eq. total.F.non.cons)
  final update  u^{n+1} = u^n - dt [dloc F + Bloc
                  + (F^num,- - F^tot,-)_{e+1/2} dx g_R + (F^num,+ - F^tot,+)_{e-1/2} dx g_L]
                (Eq. crkfr.non.cons.final)

With a source term s(u) (Sec. 2, Eqs. crkfr.inner, crkfr, avg.source) the
inner stages add dt sum_{j<=i} a_ij s(u^(j)) with the implicit tableau of a
double Butcher tableau, the stage equation being solved point by point
(oracle.sources), and the final update adds dt S, S = sum_i b_i s(u^(i)).

The readings of the oracle package docstring apply (``nc_face``, ``lam_state``,
``coef_dissipation``).  Meshes are uniform and periodic.

Layouts: 1D u[var, elem, node], c[elem, node];
2D u[var, ey, ex, qy, px], c[ey, ex, qy, px] (qy is the y-node index,
px the x-node index).
"""
import numpy as np

from .basis import Basis
from .sources import point_implicit_solve
from .tableau import ImexTableau, default_tableau, imex_tableau
from .xp import xp_of

FROZEN, LITERAL, STAGEWISE = "frozen", "literal", "stagewise"


# ----------------------------------------------------------------------------
# element-local derivatives (Eq. dlocx.defn with d/dx = (1/dx) d/dxi)
# ----------------------------------------------------------------------------
def dloc_1d(D, X):
    return xp_of(X).einsum("pj,...j->...p", D, X)


def dlocx_2d(D, X):
    return xp_of(X).einsum("pj,...qj->...qp", D, X)


def dlocy_2d(D, X):
    return xp_of(X).einsum("qj,...jp->...qp", D, X)


def trace_1d(l, X):
    return xp_of(X).einsum("p,...p->...", l, X)


def tracex_2d(l, X):
    """Extrapolation along x to a vertical face, one value per y-node."""
    return xp_of(X).einsum("p,...qp->...q", l, X)


def tracey_2d(l, X):
    """Extrapolation along y to a horizontal face, one value per x-node."""
    return xp_of(X).einsum("q,...qp->...p", l, X)


# ----------------------------------------------------------------------------
# face terms (one Riemann problem per face node)
# ----------------------------------------------------------------------------
def face_terms(flux_m, flux_p, U_m, U_p, un_m, un_p, c_m, c_p,
               speed, ncprod, nc_face=FROZEN, lam_state="n",
               stage_m=None, stage_p=None, b=None, dissipated=None):
    """Face term on each side, T^+- = F^num,+- - F^tot,+- (Eq. total.F.non.cons).

    ``*_m`` is the left (minus) side of the face, ``*_p`` the right (plus) side.
    ``stage_m/stage_p`` (lists of stage traces) are needed only for the
    'literal' and 'stagewise' readings.  ``dissipated(U, c)``, if given, is
    the state whose jump the Rusanov term dissipates (default U itself).
    Returns (T_minus, T_plus, lam).
    """
    Fn_m, Fn_p, Ft_m, Ft_p, lam = face_fluxes(flux_m, flux_p, U_m, U_p, un_m, un_p, c_m, c_p,
                                             speed, ncprod, nc_face, lam_state, stage_m,
                                             stage_p, b, dissipated)
    return Fn_m - Ft_m, Fn_p - Ft_p, lam


def face_fluxes(flux_m, flux_p, U_m, U_p, un_m, un_p, c_m, c_p,
                speed, ncprod, nc_face=FROZEN, lam_state="n",
                stage_m=None, stage_p=None, b=None, dissipated=None):
    """The two parts of the face terms: the time-averaged numerical fluxes
    F^num,+- = F^num + F^num,nc,+- and the extrapolated total fluxes
    F^tot,+- = F^+- + F^nc,+- (Eq. total.F.non.cons), and lam.
    Returns (F^num,-, F^num,+, F^tot,-, F^tot,+, lam)."""
    xp = xp_of(U_m, un_m, flux_m)
    if lam_state == "n":
        lam = xp.maximum(speed(un_m, c_m), speed(un_p, c_p))
    else:
        lam = xp.maximum(speed(U_m, c_m), speed(U_p, c_p))
    if dissipated is None:
        Fnum = 0.5 * (flux_m + flux_p) - 0.5 * lam * (U_p - U_m)
    else:
        Fnum = 0.5 * (flux_m + flux_p) - 0.5 * lam * (dissipated(U_p, c_p) - dissipated(U_m, c_m))
    U_num = 0.5 * (U_m + U_p)
    c_num = 0.5 * (c_m + c_p)
    if nc_face == FROZEN:
        num_nc_m = ncprod(un_m, c_m, U_num, c_num)
        num_nc_p = ncprod(un_p, c_p, U_num, c_num)
        ext_nc_m = ncprod(un_m, c_m, U_m, c_m)
        ext_nc_p = ncprod(un_p, c_p, U_p, c_p)
    else:
        ext_nc_m = sum(bj * ncprod(sm, c_m, sm, c_m) for bj, sm in zip(b, stage_m))
        ext_nc_p = sum(bj * ncprod(sp, c_p, sp, c_p) for bj, sp in zip(b, stage_p))
        if nc_face == LITERAL:
            num_nc_m = ncprod(un_m, c_m, U_num, c_num)
            num_nc_p = ncprod(un_p, c_p, U_num, c_num)
        elif nc_face == STAGEWISE:
            num_nc_m = sum(bj * ncprod(sm, c_m, 0.5 * (sm + sp), c_num)
                           for bj, sm, sp in zip(b, stage_m, stage_p))
            num_nc_p = sum(bj * ncprod(sp, c_p, 0.5 * (sm + sp), c_num)
                           for bj, sm, sp in zip(b, stage_m, stage_p))
        else:
            raise ValueError(nc_face)
    return Fnum + num_nc_m, Fnum + num_nc_p, flux_m + ext_nc_m, flux_p + ext_nc_p, lam


def _set_tableau(obj, N, tableau, source):
    """Explicit (A, b) for the flux terms and, with a source, the implicit
    (Ai, bi); the default is default_tableau(N), or imex_tableau(N) when a
    source is given."""
    if tableau is None:
        tableau = imex_tableau(N) if source is not None else default_tableau(N)
    if isinstance(tableau, ImexTableau):
        obj.A, obj.b = tableau.Ae, tableau.be
        obj.Ai, obj.bi = tableau.Ai, tableau.bi
    else:
        if source is not None:
            raise ValueError("a source term needs a double (IMEX) tableau")
        obj.A, obj.b = tableau
        obj.Ai = obj.bi = None
    obj.source = source


def inner_stages(obj, u, c, dt, Lfun):
    """Stages u^(i) of Eq. crkfr.non.cons.final (with a source: Eq.
    crkfr.inner), the local operators L_i = Lfun(u^(i)) and, with a source,
    the time-averaged source S = sum_i b_i s(u^(i)) (else None)."""
    stages, L, Src = [], [], []
    for i in range(len(obj.b)):
        acc = 0.0
        for j in range(i):
            if obj.A[i, j] != 0.0:
                acc = acc + obj.A[i, j] * L[j]
        ui = u - dt * acc
        if obj.source is not None:
            for j in range(i):
                if obj.Ai[i, j] != 0.0:
                    ui = ui + (dt * obj.Ai[i, j]) * Src[j]
            ui = point_implicit_solve(obj.source, ui, c, dt * obj.Ai[i, i])
            Src.append(obj.source.source(ui, c))
        stages.append(ui)
        L.append(Lfun(ui))
    S = None
    if obj.source is not None:
        S = sum(bj * sj for bj, sj in zip(obj.bi, Src))
    return stages, L, S


# ----------------------------------------------------------------------------
# 1D
# ----------------------------------------------------------------------------
class Scheme1D:
    """cRK-FR on a uniform periodic 1D mesh of E elements of width dx."""

    def __init__(self, system, N, dx, family="gl", tableau=None,
                 nc_face=FROZEN, lam_state="n", coef_dissipation=False, source=None):
        self.sys = system
        self.basis = Basis(N, family)
        _set_tableau(self, N, tableau, source)
        self.dx = dx
        self.nc_face = nc_face
        self.lam_state = lam_state
        self.coef_dissipation = coef_dissipation

    # -- element-local part -------------------------------------------------
    def local(self, u, c, dt):
        """Inner stages and time averages on a batch of elements.

        u: (M, ..., n), c: (..., n).  Returns a dict with the volume term
        dloc F + Bloc and the face traces (right = xi 1, left = xi 0)."""
        sy, bs = self.sys, self.basis
        D = bs.D / self.dx
        dc = dloc_1d(D, c)
        stages, L, S = inner_stages(
            self, u, c, dt,
            lambda ui: dloc_1d(D, sy.flux(ui, c)) + sy.ncprod(ui, c, dloc_1d(D, ui), dc))
        F = sum(bj * sy.flux(uj, c) for bj, uj in zip(self.b, stages))
        U = sum(bj * uj for bj, uj in zip(self.b, stages))
        Bloc = sum(bj * sy.ncprod(uj, c, dloc_1d(D, uj), dc)
                   for bj, uj in zip(self.b, stages))
        out = dict(vol=dloc_1d(D, F) + Bloc if S is None else dloc_1d(D, F) + Bloc - S,
                   F_r=trace_1d(bs.l1, F), F_l=trace_1d(bs.l0, F),
                   U_r=trace_1d(bs.l1, U), U_l=trace_1d(bs.l0, U),
                   un_r=trace_1d(bs.l1, u), un_l=trace_1d(bs.l0, u),
                   c_r=trace_1d(bs.l1, c), c_l=trace_1d(bs.l0, c))
        if self.nc_face != FROZEN:
            out["st_r"] = [trace_1d(bs.l1, uj) for uj in stages]
            out["st_l"] = [trace_1d(bs.l0, uj) for uj in stages]
        return out

    def _faces(self, lm, lp, elem_axis_len=None):
        """Face terms for faces whose minus side data is ``lm`` (traces at
        xi = 1 of the left element) and plus side ``lp`` (xi = 0 of the right
        element)."""
        sy = self.sys
        return face_terms(lm["F_r"], lp["F_l"], lm["U_r"], lp["U_l"],
                          lm["un_r"], lp["un_l"], lm["c_r"], lp["c_l"],
                          sy.speed, sy.ncprod, self.nc_face, self.lam_state,
                          lm.get("st_r"), lp.get("st_l"), self.b, getattr(sy, "dissipated", None))

    # -- full periodic step --------------------------------------------------
    def residual(self, u, c, dt, bloch=None):
        """R such that u^{n+1} = u^n - dt R (Eq. crkfr.non.cons.final).

        ``bloch`` (a phase theta) treats the mesh as one period of a Bloch
        wave: values wrapped across the periodic boundary are multiplied by
        exp(-+ i theta).  Used only by the von Neumann analysis."""
        bs = self.basis
        xp = xp_of(u)
        loc = self.local(u, c, dt)
        ph = 1.0 if bloch is None else np.exp(-1j * bloch)

        def left_neighbour(X, scale=True):
            # element e-1 for each e (periodic); face k has minus side = elem k-1
            Y = xp.roll(X, 1, axis=-1)
            if bloch is not None and scale:
                Y = Y.astype(complex)
                Y[..., 0] = Y[..., 0] * ph
            return Y

        lm = {}
        for k in ("F_r", "U_r", "un_r"):
            lm[k] = left_neighbour(loc[k])
        lm["c_r"] = left_neighbour(loc["c_r"], scale=False)
        if "st_r" in loc:
            lm["st_r"] = [left_neighbour(x) for x in loc["st_r"]]
        lp = {k: loc[k] for k in ("F_l", "U_l", "un_l", "c_l")}
        if "st_l" in loc:
            lp["st_l"] = loc["st_l"]
        T_m, T_p, lam = self._faces(lm, lp)
        # element e: right face is face e+1 (minus side), left face is face e
        T_right = xp.roll(T_m, -1, axis=-1)
        if bloch is not None:
            T_right = T_right.astype(complex)
            T_right[..., -1] = T_right[..., -1] / ph
        gR, gL = xp.asarray(bs.gRp), xp.asarray(bs.gLp)
        R = loc["vol"] + (T_right[..., None] * gR + T_p[..., None] * gL) / self.dx
        self._last_lam = lam
        return R

    def step(self, u, c, dt):
        R = self.residual(u, c, dt)
        return u - dt * R

    def step_coef(self, u, c, dt):
        """Step with the literal augmented form (reading 2 switched off): the
        coefficient is an evolved variable with zero flux, so its only update
        is the Rusanov dissipation of the face flux."""
        R = self.residual(u, c, dt)
        bs = self.basis
        lam = self._last_lam
        c_r, c_l = trace_1d(bs.l1, c), trace_1d(bs.l0, c)
        c_m = np.roll(c_r, 1, axis=-1)
        Fnum_c = -0.5 * lam * (c_l - c_m)
        Rc = (np.roll(Fnum_c, -1, axis=-1)[..., None] * bs.gRp
              + Fnum_c[..., None] * bs.gLp) / self.dx
        return u - dt * R, c - dt * Rc

    # -- sampled step: u^{n+1} on selected elements only --------------------
    def step_elements(self, u, c, dt, elems):
        """u^{n+1} of the elements ``elems`` only, computed from the
        3-element stencil (e-1, e, e+1) of each; returns (M, len(elems), n)."""
        elems = np.asarray(elems)
        E = u.shape[-2]
        idx = np.stack([(elems - 1) % E, elems, (elems + 1) % E], axis=-1)  # (S,3)
        loc = self.local(u[:, idx, :], c[idx, :], dt)
        bs = self.basis
        pick = lambda d, k, j: d[k][..., j]
        left = {k: pick(loc, k, 0) for k in ("F_r", "U_r", "un_r", "c_r")}
        mid_l = {k: pick(loc, k, 1) for k in ("F_l", "U_l", "un_l", "c_l")}
        mid_r = {k: pick(loc, k, 1) for k in ("F_r", "U_r", "un_r", "c_r")}
        right = {k: pick(loc, k, 2) for k in ("F_l", "U_l", "un_l", "c_l")}
        if self.nc_face != FROZEN:
            left["st_r"] = [x[..., 0] for x in loc["st_r"]]
            mid_l["st_l"] = [x[..., 1] for x in loc["st_l"]]
            mid_r["st_r"] = [x[..., 1] for x in loc["st_r"]]
            right["st_l"] = [x[..., 2] for x in loc["st_l"]]
        _, T_p_left, _ = self._faces(left, mid_l)
        T_m_right, _, _ = self._faces(mid_r, right)
        R = loc["vol"][..., 1, :] + (T_m_right[..., None] * bs.gRp
                                     + T_p_left[..., None] * bs.gLp) / self.dx
        return u[:, elems, :] - dt * R

    # -- time step (Sec. 5, Eq. time.step.2d with g = 0, B_2 = 0) -------------
    def element_means(self, u, c):
        w = self.basis.w
        return np.einsum("p,...p->...", w, u), np.einsum("p,...p->...", w, c)

    def max_rate(self, u, c):
        ub, cb = self.element_means(u, c)
        return np.max(self.sys.speed(ub, cb) / self.dx)

    def compute_dt(self, u, c, cfl, cs):
        return cs * cfl / self.max_rate(u, c)


# ----------------------------------------------------------------------------
# 2D (tensor product, line by line)
# ----------------------------------------------------------------------------
class Scheme2D:
    """cRK-FR on a uniform periodic Ey x Ex mesh of dx x dy quads."""

    def __init__(self, system, N, dx, dy, family="gl", tableau=None,
                 nc_face=FROZEN, lam_state="n", source=None):
        self.sys = system
        self.basis = Basis(N, family)
        _set_tableau(self, N, tableau, source)
        self.dx, self.dy = dx, dy
        self.nc_face = nc_face
        self.lam_state = lam_state

    def _L(self, ui, c, Dx, Dy, dcx, dcy):
        sy = self.sys
        return (dlocx_2d(Dx, sy.flux_x(ui, c)) + dlocy_2d(Dy, sy.flux_y(ui, c))
                + sy.ncprod_x(ui, c, dlocx_2d(Dx, ui), dcx)
                + sy.ncprod_y(ui, c, dlocy_2d(Dy, ui), dcy))

    def local(self, u, c, dt):
        """Inner stages, time averages, volume term and face traces on a
        batch of elements.  u: (M, ..., n, n), c: (..., n, n)."""
        sy, bs = self.sys, self.basis
        Dx, Dy = bs.D / self.dx, bs.D / self.dy
        dcx, dcy = dlocx_2d(Dx, c), dlocy_2d(Dy, c)
        stages, L, S = inner_stages(self, u, c, dt,
                                    lambda ui: self._L(ui, c, Dx, Dy, dcx, dcy))
        F = sum(bj * sy.flux_x(uj, c) for bj, uj in zip(self.b, stages))
        G = sum(bj * sy.flux_y(uj, c) for bj, uj in zip(self.b, stages))
        U = sum(bj * uj for bj, uj in zip(self.b, stages))
        Bloc = sum(bj * (sy.ncprod_x(uj, c, dlocx_2d(Dx, uj), dcx)
                         + sy.ncprod_y(uj, c, dlocy_2d(Dy, uj), dcy))
                   for bj, uj in zip(self.b, stages))
        l0, l1 = bs.l0, bs.l1
        vol = dlocx_2d(Dx, F) + dlocy_2d(Dy, G) + Bloc
        out = dict(vol=vol if S is None else vol - S)
        for name, X in (("F", F), ("U", U), ("un", u), ("c", c)):
            out[name + "_r"] = tracex_2d(l1, X)
            out[name + "_l"] = tracex_2d(l0, X)
        for name, X in (("G", G), ("U", U), ("un", u), ("c", c)):
            out[name + "_t"] = tracey_2d(l1, X)
            out[name + "_b"] = tracey_2d(l0, X)
        if self.nc_face != FROZEN:
            out["st_r"] = [tracex_2d(l1, x) for x in stages]
            out["st_l"] = [tracex_2d(l0, x) for x in stages]
            out["st_t"] = [tracey_2d(l1, x) for x in stages]
            out["st_b"] = [tracey_2d(l0, x) for x in stages]
        return out

    def _xface(self, m, p):
        """x-face between a left element (traces ``m``, side r) and a right
        element (traces ``p``, side l)."""
        sy = self.sys
        return face_terms(m["F_r"], p["F_l"], m["U_r"], p["U_l"], m["un_r"], p["un_l"],
                          m["c_r"], p["c_l"], sy.speed_x, sy.ncprod_x, self.nc_face,
                          self.lam_state, m.get("st_r"), p.get("st_l"), self.b,
                          getattr(sy, "dissipated", None))

    def _yface(self, m, p):
        """y-face between a lower element (``m``, side t) and an upper element
        (``p``, side b)."""
        sy = self.sys
        return face_terms(m["G_t"], p["G_b"], m["U_t"], p["U_b"], m["un_t"], p["un_b"],
                          m["c_t"], p["c_b"], sy.speed_y, sy.ncprod_y, self.nc_face,
                          self.lam_state, m.get("st_t"), p.get("st_b"), self.b,
                          getattr(sy, "dissipated", None))

    def _corrections(self, Tr, Tl, Tt, Tb):
        """Correction terms (Eq. crkfr.non.cons.final) from the face terms at
        the right (Tr), left (Tl), top (Tt) and bottom (Tb) faces."""
        bs = self.basis
        xp = xp_of(Tr)
        gR, gL = xp.asarray(bs.gRp), xp.asarray(bs.gLp)
        cx = (Tr[..., :, None] * gR + Tl[..., :, None] * gL) / self.dx
        cy = (Tt[..., None, :] * gR[:, None] + Tb[..., None, :] * gL[:, None]) / self.dy
        return cx + cy

    def residual(self, u, c, dt):
        ns = xp_of(u)
        loc = self.local(u, c, dt)
        ax_y, ax_x = -3, -2   # element axes of the trace arrays (..., ey, ex, node)

        def sel(d, keys, shift, axis):
            out = {}
            for k in keys:
                v = d.get(k)
                if v is None:
                    continue
                if isinstance(v, list):
                    out[k] = [ns.roll(x, shift, axis=axis) for x in v]
                else:
                    out[k] = ns.roll(v, shift, axis=axis)
            return out

        xm = sel(loc, ("F_r", "U_r", "un_r", "c_r", "st_r"), 1, ax_x)
        xp = sel(loc, ("F_l", "U_l", "un_l", "c_l", "st_l"), 0, ax_x)
        Txm, Txp, _ = self._xface(xm, xp)           # face (ey, kx): elem kx-1 | elem kx
        ym = sel(loc, ("G_t", "U_t", "un_t", "c_t", "st_t"), 1, ax_y)
        yp = sel(loc, ("G_b", "U_b", "un_b", "c_b", "st_b"), 0, ax_y)
        Tym, Typ, _ = self._yface(ym, yp)           # face (ky, ex): elem ky-1 below | ky above
        Tr = ns.roll(Txm, -1, axis=ax_x)
        Tt = ns.roll(Tym, -1, axis=ax_y)
        return loc["vol"] + self._corrections(Tr, Txp, Tt, Typ)

    def step(self, u, c, dt):
        return u - dt * self.residual(u, c, dt)

    def step_elements(self, u, c, dt, ey, ex):
        """u^{n+1} of the elements (ey[k], ex[k]) only, from their 5-element
        stencils; returns (M, S, n, n)."""
        ey, ex = np.asarray(ey), np.asarray(ex)
        Ey, Ex = u.shape[1], u.shape[2]
        sy_ = np.stack([ey, ey, ey, (ey - 1) % Ey, (ey + 1) % Ey], axis=-1)
        sx_ = np.stack([ex, (ex - 1) % Ex, (ex + 1) % Ex, ex, ex], axis=-1)
        loc = self.local(u[:, sy_, sx_], c[sy_, sx_], dt)
        # stencil slots: 0 centre, 1 left, 2 right, 3 below, 4 above
        pick = lambda k, j: ([x[..., j, :] for x in loc[k]] if isinstance(loc[k], list)
                             else loc[k][..., j, :])
        keys = lambda suf: [k for k in loc if k.endswith(suf)]
        slot = lambda suf, j: {k: pick(k, j) for k in keys(suf)}
        _, Tl, _ = self._xface(slot("_r", 1), slot("_l", 0))
        Tr, _, _ = self._xface(slot("_r", 0), slot("_l", 2))
        _, Tb, _ = self._yface(slot("_t", 3), slot("_b", 0))
        Tt, _, _ = self._yface(slot("_t", 0), slot("_b", 4))
        R = loc["vol"][..., 0, :, :] + self._corrections(Tr, Tl, Tt, Tb)
        return u[:, ey, ex] - dt * R

    # -- time step (Sec. 5, Eq. time.step.2d) --------------------------------
    def element_means(self, u, c):
        w = self.basis.w
        return (np.einsum("q,p,...qp->...", w, w, u), np.einsum("q,p,...qp->...", w, w, c))

    def max_rate(self, u, c):
        ub, cb = self.element_means(u, c)
        sy = self.sys
        return np.max(sy.speed_x(ub, cb) / self.dx + sy.speed_y(ub, cb) / self.dy)

    def compute_dt(self, u, c, cfl, cs):
        return cs * cfl / self.max_rate(u, c)
