"""Semi-discrete FR scheme for non-conservative systems in 1D
(test infrastructure only).

Sec. 3, Eq. general.non.conservative.fr.one with the numerical fluxes of
Eqs. combined.num.flux.fr, non.cons.num.flux.basic, combined.num.flux and
the extrapolations of Eq. total.flux.non.cons:

  du/dt = -[ dloc f(u) + B(w) dloc w
             + (f^num,- - f^tot,-)_{e+1/2} dx g_R + (f^num,+ - f^tot,+)_{e-1/2} dx g_L ]

  f^num,+- = f^num + B(w^+-) w^num,  w^num = (w^- + w^+)/2
  f^num    = (f(u^-) + f(u^+))/2 - lam/2 (u^+ - u^-),  lam = max sigma(f' + B)
  f^tot,+- = B(w^+-) w^+- + f^+-   (f^+- extrapolated from the discontinuous flux)

Used as the dt -> 0 limit of the cRK-FR residual.  Written separately from
``crkfr.face_terms`` on purpose.
"""
import numpy as np

from .basis import Basis


def rhs_1d(system, N, dx, u, c, family="gl"):
    bs = Basis(N, family)
    D = bs.D / dx
    f = system.flux(u, c)
    du = np.einsum("pj,...j->...p", D, u)
    dc = np.einsum("pj,...j->...p", D, c)
    vol = np.einsum("pj,...j->...p", D, f) + system.ncprod(u, c, du, dc)

    ext = lambda l, X: np.einsum("p,...p->...", l, X)
    # element traces at xi = 1 (right) and xi = 0 (left)
    uR, uL = ext(bs.l1, u), ext(bs.l0, u)
    fR, fL = ext(bs.l1, f), ext(bs.l0, f)
    cR, cL = ext(bs.l1, c), ext(bs.l0, c)
    # face k: minus side = element k-1 (periodic), plus side = element k
    um, fm, cm = np.roll(uR, 1, -1), np.roll(fR, 1, -1), np.roll(cR, 1, -1)
    up, fp, cp = uL, fL, cL
    lam = np.maximum(system.speed(um, cm), system.speed(up, cp))
    fnum = 0.5 * (fm + fp) - 0.5 * lam * (up - um)
    unum, cnum = 0.5 * (um + up), 0.5 * (cm + cp)
    fnum_m = fnum + system.ncprod(um, cm, unum, cnum)
    fnum_p = fnum + system.ncprod(up, cp, unum, cnum)
    ftot_m = system.ncprod(um, cm, um, cm) + fm
    ftot_p = system.ncprod(up, cp, up, cp) + fp
    jump_right = np.roll(fnum_m - ftot_m, -1, -1)   # face e+1/2 seen from element e
    jump_left = fnum_p - ftot_p                     # face e-1/2 seen from element e
    corr = (jump_right[..., None] * bs.gRp + jump_left[..., None] * bs.gLp) / dx
    return -(vol + corr)
