"""Reference oracle for the compact Runge-Kutta flux reconstruction (cRK-FR)
scheme for non-conservative hyperbolic systems (Babbar & Ranocha, 2025).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
CPU restatement of the scheme in numpy FP64.  It exists to check the CUDA
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference arm may import it; the product library never does,
and the two share no code (only the seeded input generators in
``paper_2512_08611_gb300.workloads`` serve both, and those hold none of the
method's arithmetic).

Modules
-------
basis      reference element: nodes, weights, Lagrange basis, D, l(0), l(1),
           correction-function derivatives (Sec. 2; App. B, Eq. correction.identities)
tableau    Butcher tableaux: explicit ones, and the double (IMEX) tableaux
           HT(1,1,2) and SSP3-IMEX(4,3,3) of App. C
sources    source terms (linear damping, Chezy friction) and the
           point-implicit stage solve (Sec. 2, Eqs. crkfr.inner, avg.source)
systems    physical systems: variable-coefficient advection, shallow water
           with bathymetry as a non-conservative product (Sec. 3, Sec. 5.1.3)
crkfr      the cRK-FR step, residual and time step in 1D and 2D
           (Sec. 3, Eqs. crkfr.non.cons.final, total.F.non.cons,
           local.time.avg.non.cons, good.numflux.non.cons; Sec. 5 Eq. time.step.2d)
semidisc   semi-discrete FR right-hand side (Eq. general.non.conservative.fr.one)
fourier    von Neumann analysis giving CFL(N) (Sec. 5, remark under Eq. time.step.2d)
exact      characteristics solution of the variable-coefficient test, L2 error

Readings where the paper is silent or ambiguous (each is a switch where it
matters; the default is listed first):

1. Face non-conservative terms: ``nc_face='frozen'`` uses B(w^{n,+-}) for
   both the numerical non-conservative flux (Eq. good.numflux.non.cons) and
   the extrapolation term F^{nc,+-} = B(w^{n,+-}) W^{+-}; ``'literal'`` takes
   F^{nc,+-} = sum_j b_j B(w^{(j)+-}) w^{(j)+-} as printed under
   Eq. total.F.non.cons; ``'stagewise'`` uses Eq. bad.numflux.non.cons with
   the literal extrapolation.
2. The coefficient field c (a(x) or the bathymetry b) is static: it is not
   evolved and receives no dissipation (``coef_dissipation=False``).
3. The Rusanov speed at a face is the max over the two u^n traces
   (``lam_state='n'``); ``'avg'`` uses the time-averaged traces.
4. Tableaux (order N+1): N=0 forward Euler, N=1 HT(1,1,2) explicit part,
   N=2 the explicit part of SSP3-IMEX(4,3,3), N=3 classical RK4, N=4
   Butcher's six-stage fifth-order method.
5. CFL(N) is the largest nu with spectral radius <= 1 + tau over the
   wavenumber grid kappa_k = pi k / 256, k = 0..256 (bisection, 60 halvings),
   tau = 1e-12 for N <= 3 and 1e-4 for N = 4 (see ``fourier``).
6. 2D is the tensor-product, line-by-line extension; face quantities are
   evaluated at every face node.
7. The implicit tableau of SSP3-IMEX(4,3,3) as printed in App. C (Eq.
   ssp33.butcher) disagrees with its own node column (rows 2 and 3 sum to
   alpha and 2/3 + alpha, the printed c_2, c_3 are 0 and 1) and, so read, is
   only first order and not L-stable, against the paper's statements.  The
   oracle takes rows 2 and 3 as (-alpha, alpha, 0, 0) and
   (0, 1 - alpha, alpha, 0): the rows that sum to the printed c_2 = 0 and
   c_3 = 1 and that make the pair third order and L-stable (the cited source
   of the scheme, Pareschi & Russo 2005, has these rows).  Row 4 is used as
   printed (its sum is 1/2; the printed c_4 = 1 plays no role for an
   autonomous source).
8. With a source, the tableau is SSP3-IMEX(4,3,3) at every degree (the
   paper's stiff tests use it at N = 3; HT(1,1,2) makes the N = 1 step grow
   under a stiff source), and CFL(N) is that of its explicit part.
"""
