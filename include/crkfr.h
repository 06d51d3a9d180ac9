/*
 * crkfr.h - C ABI of the GB300 (sm_103a) compact Runge-Kutta flux
 * reconstruction library for non-conservative hyperbolic systems
 * (Babbar & Ranocha, "Admissibility preserving compact Runge-Kutta flux
 * reconstruction for non-conservative hyperbolic equations with stiff
 * source terms", arXiv 2512.08611).
 *
 * One time step of the method (Sec. 3, Eqs. crkfr.non.cons.final,
 * total.F.non.cons, local.time.avg.non.cons, good.numflux.non.cons) for
 *
 *     u_t + f(u)_x [+ g(u)_y] + B(w) grad w = 0,   w = (u, c),
 *
 * where c is a static coefficient field (a(x) for variable-coefficient
 * advection, Sec. 5.1.3; the bathymetry b for shallow water).  The inner
 * Runge-Kutta stages use only the element-local derivative; only the final
 * stage couples neighbours through one time-averaged numerical flux per face,
 * the non-conservative fluctuation B(w^{n,+-}) (W^num - W^{+-}) and the FR
 * correction-function derivatives (App. B, Eq. correction.identities).
 *
 * Conventions
 * -----------
 * - Arithmetic is IEEE FP64 throughout.
 * - Meshes are uniform and periodic: dim 1 with E elements on [lo, hi], or
 *   dim 2 with Ex x Ey quads on [lo0, hi0] x [lo1, hi1].
 * - Nodal layout (row-major, contiguous, FP64):
 *     1D: u[var][elem][p]            c[elem][p]
 *     2D: u[var][ey][ex][q][p]       c[ey][ex][q][p]
 *   p is the x node index, q the y node index, 0..N, at the solution points
 *   returned by crkfr_get_nodes (position of node p of element e:
 *   lo + (e + xi_p) * dx).
 * - Variables: advection (v); 1D shallow water (h, hu); 2D shallow water
 *   (h, hu, hv) (the same for the well-balanced forms).  Degree N is 0..4
 *   (1D) or 1..4 (2D).
 * - Pointers named *_dev are device pointers on the current CUDA device;
 *   *_host are host pointers.  The caller owns every pointer it passes; the
 *   library never frees them and keeps none of them past the call.
 *   Buffers the method needs between kernels (face traces, a second state,
 *   the static coefficient terms, a device status word) are owned by the
 *   context and sized at crkfr_set_mesh.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *   asynchronous on that stream unless they return a host value, in which
 *   case they synchronise that stream only.
 * - Errors: every entry point returns a crkfr_status; nothing traps or
 *   throws across the ABI.  crkfr_last_error gives the context's last error
 *   text; crkfr_last_error(NULL) gives the calling host thread's last error
 *   of a call that has no context to hold it (crkfr_create,
 *   crkfr_batch_create, crkfr_step_1d_noalloc).  A context is not
 *   thread-safe; use one context per host thread.
 */
#ifndef CRKFR_H
#define CRKFR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crkfr_ctx crkfr_ctx;

typedef enum {
  CRKFR_OK = 0,
  CRKFR_ERR_ARG = -1,          /* invalid argument or size                     */
  CRKFR_ERR_UNSUPPORTED = -2,  /* system / degree / node family not built      */
  CRKFR_ERR_CUDA = -3,         /* a CUDA runtime call failed                    */
  CRKFR_ERR_NONPHYSICAL = -4,  /* h <= 0 or a non-finite value was produced    */
  CRKFR_ERR_STATE = -6,        /* call out of order (e.g. no mesh set yet)      */
  CRKFR_ERR_ALLOC = -7         /* device or host allocation failed             */
} crkfr_status;

/* The well-balanced forms move the hydrostatic pressure into the
 * non-conservative product, g h (h + b)_x, and dissipate the free surface
 * eta = h + b in the Rusanov flux of the h equation, so that a lake at rest
 * (hu = 0, eta constant) is kept to round-off; the paper lists well-balanced
 * cRK methods as open (Sec. 6).  Same variables and layouts as the standard
 * forms. */
typedef enum {
  CRKFR_SYS_VARADV_1D = 0,     /* v_t + a(x) v_x = 0, c = a (Sec. 5.1.3)        */
  CRKFR_SYS_SWE_1D = 1,        /* shallow water, c = b, B(w)(du,db) = (0, g h db) */
  CRKFR_SYS_SWE_2D = 2,        /* 2D shallow water, B1 = (0,g h db,0), B2 = (0,0,g h db) */
  CRKFR_SYS_SWE_1D_WB = 3,     /* well-balanced 1D: f = (hu, (hu)^2/h),
                                  B(w)(du,db) = (0, g h (du_h + db))               */
  CRKFR_SYS_SWE_2D_WB = 4      /* well-balanced 2D: pressure-free fluxes,
                                  B1 = (0, g h (du_h+db), 0), B2 = (0, 0, g h (du_h+db)) */
} crkfr_system;

typedef enum {
  CRKFR_NODES_GL = 0,          /* Gauss-Legendre points, Radau correction (Sec. 2) */
  CRKFR_NODES_GLL = 1          /* Gauss-Lobatto-Legendre points, g_2 correction   */
} crkfr_nodes;

/* Source term s(u) of u_t + ... = s(u) (Sec. 2, Eq. con.law.source), treated
 * implicitly in the inner stages (Eq. crkfr.inner) with the double tableau
 * SSP3-IMEX(4,3,3) of App. C (Eq. ssp33.butcher; its implicit rows 2 and 3
 * are read as the rows that sum to the printed nodes c_2 = 0, c_3 = 1, which
 * make the pair third order and L-stable as the paper states).  The final
 * update adds dt sum_i b_i s(u^(i)) (Eqs. crkfr, avg.source).  Each stage's
 * implicit equation is solved point by point in closed form. */
typedef enum {
  CRKFR_SRC_NONE = 0,          /* no source: the explicit tableau of degree N      */
  CRKFR_SRC_LINEAR_DAMPING = 1,/* s = -K v, advection only (model problem, App. A) */
  CRKFR_SRC_CHEZY = 2          /* s = (0, -C_f |v| v) on the momentum, shallow water
                                  only (the friction term of Sec. 5.5), v = hu/h   */
} crkfr_source;

typedef struct {
  int32_t system;      /* crkfr_system                                               */
  int32_t degree;      /* polynomial degree N                                        */
  int32_t nodes;       /* crkfr_nodes                                                */
  int32_t source;      /* crkfr_source; a source that does not belong to the system
                          gives CRKFR_ERR_UNSUPPORTED                                */
  double gravity;      /* g for shallow water; ignored for advection                */
  double cfl_safety;   /* C_s of Sec. 5, Eq. time.step.2d; 0 < C_s <= 1             */
  double cfl_number;   /* CFL(N) of Eq. time.step.2d; <= 0 selects the library's own
                          von Neumann value (crkfr_get_cfl), which with a source is
                          that of the explicit part of SSP3-IMEX(4,3,3)              */
  double source_coef;  /* K or C_f, finite and >= 0; ignored without a source       */
  /* Readings of the paper that are switches of the method (a zero-filled
   * config selects the built default of each; any other value returns
   * CRKFR_ERR_UNSUPPORTED, with the reason in crkfr_last_error(NULL)): */
  int32_t rk;          /* order of the Runge-Kutta tableau of Eq. crkfr.non.cons.final:
                          0 or the default order, N+1 without a source (forward Euler,
                          HT(1,1,2) and SSP3-IMEX(4,3,3) explicit parts, classical RK4,
                          Butcher's six-stage fifth-order method for N = 0..4) and 3
                          with one (SSP3-IMEX(4,3,3), App. C)                       */
  int32_t nc_face_mode; /* crkfr_nc_face: the face non-conservative terms (Sec. 3):
                          only CRKFR_NC_FROZEN is built                               */
  int32_t coef_dissipation; /* 0: the coefficient c (a or b) is static, no dissipation
                          acts on it (built); 1: the literal augmented form w = (u, c)
                          whose Rusanov term would let c drift (not built)            */
  int32_t reserved;    /* must be 0                                                   */
} crkfr_config;

/* Face non-conservative terms of Sec. 3 when B depends on the evolving
 * variables.  FROZEN: F^{nc,+-} = B(w^{n,+-}) W^{+-}, the B of Eq.
 * good.numflux.non.cons frozen at t^n for both the numerical and the
 * extrapolated term (the reading this library builds); LITERAL: the
 * extrapolation under Eq. total.F.non.cons with stage values as printed;
 * STAGEWISE: Eq. bad.numflux.non.cons stage by stage.  The last two keep
 * every stage's traces; they exist in the CPU oracle, not here. */
typedef enum {
  CRKFR_NC_FROZEN = 0,
  CRKFR_NC_LITERAL = 1,
  CRKFR_NC_STAGEWISE = 2
} crkfr_nc_face;

/* Create a context for one system / degree / node family / source.  Runs
 * the library's von Neumann analysis of the scheme for linear advection when
 * cfg->cfl_number <= 0 (Sec. 5, under Eq. time.step.2d).  *out is set to NULL
 * on failure, and crkfr_last_error(NULL) gives the reason. */
crkfr_status crkfr_create(crkfr_ctx** out, const crkfr_config* cfg);

/* Free the context and every device buffer it owns (synchronises the device).
 * Resource management only: the paper has no counterpart. */
void crkfr_destroy(crkfr_ctx* ctx);

/* Uniform mesh (Sec. 2, Eqs. reference.element, ref.map).
 * dim must match the system (1 or 2); n_elem[dim] > 0 (Ex first, then Ey);
 * lo[dim] < hi[dim]; periodic_mask: bit d set = periodic in direction d.
 * Only periodic meshes are built (periodic_mask = 1 in 1D, 3 in 2D;
 * otherwise CRKFR_ERR_UNSUPPORTED).  Allocates the context's device buffers
 * (about 6x the state size in 1D, 5x in 2D).  Invalidates the coefficients. */
crkfr_status crkfr_set_mesh(crkfr_ctx* ctx, int32_t dim, const int64_t* n_elem,
                            const double* lo, const double* hi, int32_t periodic_mask);

/* Number of FP64 values of the state u (vars x nodes: (N+1)^dim nodal
 * values of the solution polynomial per element, Sec. 2, Eq. soln.poly) and
 * of the coefficient field c, for the mesh that is set. */
crkfr_status crkfr_sizes(const crkfr_ctx* ctx, int64_t* n_state, int64_t* n_coef);

/* Solution points xi_p in [0, 1] and quadrature weights w_p (N+1 values each,
 * host arrays) of the context's node family (Sec. 2, Eq. soln.points). */
crkfr_status crkfr_get_nodes(const crkfr_ctx* ctx, double* xi_host, double* w_host);

/* CFL(N) of Sec. 5, Eq. time.step.2d, that the context uses (given or
 * computed). */
crkfr_status crkfr_get_cfl(const crkfr_ctx* ctx, double* cfl_host);

/* Static coefficient field c at the solution points (device, layout above):
 * a(x) for advection, the bathymetry b for shallow water, the static part of
 * w = (u, c) in the non-conservative product B(w) dw/dx (Sec. 3, Eq.
 * crkfr.non.cons.final; c as a field of x rather than an evolved variable,
 * Sec. 5.1.3).  The library derives and stores what the scheme needs from it
 * (the local non-conservative factor B(c) dloc c per node and the face
 * traces of c). */
crkfr_status crkfr_set_coefficients(crkfr_ctx* ctx, const double* c_dev, void* stream);

/* Time step of Sec. 5, Eq. time.step.2d for the state u_dev:
 * C_s CFL(N) / max_e (sigma(f' + B_1)(ubar_e)/dx + sigma(g' + B_2)(ubar_e)/dy)
 * with element means ubar_e = sum_p w_p u_ep.  Synchronises the stream. */
crkfr_status crkfr_compute_dt(crkfr_ctx* ctx, const double* u_dev, double* dt_host,
                              void* stream);

/* Time-averaged residual of one cRK-FR step of size dt > 0:
 * r = (u^{n+1} - u^n) / dt, evaluated directly (not by differencing) as
 * -(dloc F + Bloc + face corrections) of Eq. crkfr.non.cons.final.
 * u_dev and r_dev must not overlap. */
crkfr_status crkfr_residual(crkfr_ctx* ctx, const double* u_dev, double dt, double* r_dev,
                            void* stream);

/* Advance u_dev in place by nsteps >= 0 cRK-FR steps.  dt > 0: that fixed
 * step; dt <= 0 (or -inf): the step of Eq. time.step.2d recomputed on the
 * device from the current state before every step (no host
 * synchronisation); a NaN or +inf dt returns CRKFR_ERR_ARG.  The context
 * accumulates simulated time on the device; the size of the last step
 * taken, which in the CFL mode exists only on the device, is returned by
 * crkfr_get_time (which synchronises), so that crkfr_step itself stays
 * asynchronous. */
crkfr_status crkfr_step(crkfr_ctx* ctx, double* u_dev, double dt, int64_t nsteps,
                        void* stream);

/* Advance with the step of Eq. time.step.2d until time t_end, shortening the
 * last step to land on t_end exactly (steps after that are no-ops).  Runs
 * chunks of device steps and reads the time back between chunks.  At most
 * max_steps steps; *steps_taken (may be NULL) receives the number of steps
 * that advanced the state.  Returns CRKFR_ERR_ARG if t_end is not reached
 * within max_steps. */
crkfr_status crkfr_advance(crkfr_ctx* ctx, double* u_dev, double t_end, int64_t max_steps,
                           int64_t* steps_taken, void* stream);

/* The step of crkfr_step (Sec. 3, Eq. crkfr.non.cons.final) on host memory;
 * the host transfers have no counterpart in the paper.  Copies u_in_host to a context-owned
 * device state, steps, and copies the result to u_out_host (the two may be
 * the same buffer).  In 2D the last step's kernels run in up to 5 parts of
 * element rows, of decreasing size, and each part's rows are copied back on a context-owned
 * stream while the later parts compute (u_out_host should be pinned for the
 * copies to overlap).  Synchronises the stream. */
crkfr_status crkfr_step_host(crkfr_ctx* ctx, const double* u_in_host, double* u_out_host,
                             double dt, int64_t nsteps, void* stream);

/* Domain decomposition of the 2D step into horizontal slabs (one per rank
 * or per GPU), and of the 1D step into element ranges (below).  The only coupling of a cRK-FR step across the slab boundary
 * is the face Riemann problem after the element-local stages (Sec. 3), so a
 * step of a slab is: crkfr_step_local; exchange of one block of face traces
 * with each neighbour; crkfr_step_faces.
 *
 * crkfr_set_subdomain(ctx, 1), after crkfr_set_mesh and before
 * crkfr_set_coefficients, makes the context's mesh (Ex x Ey_local, periodic
 * in x) one slab of a mesh that continues above and below.  In this mode
 * crkfr_set_coefficients expects c with two extra rows,
 * c[Ey_local + 2][Ex][n][n]: row 0 is the element row below the slab and row
 * Ey_local + 1 the row above (periodic neighbours at the ends of the whole
 * mesh).  crkfr_step, crkfr_advance, crkfr_step_host and crkfr_residual
 * return CRKFR_ERR_STATE; crkfr_compute_dt gives the slab's own step (the
 * step of the whole mesh is the minimum over slabs).
 *
 * crkfr_halo_buffers returns device pointers into the context's trace
 * buffer, each to `count` contiguous doubles: send_bottom (traces of the
 * bottom element row, bottom side: the rank below stores them as its
 * recv_top), send_top (top row, top side: becomes the rank above's
 * recv_bottom), recv_bottom and recv_top.  The pointers stay valid until the
 * next crkfr_set_mesh.
 *
 * crkfr_step_local runs the element-local kernel with the step dt > 0 and
 * writes the send blocks; crkfr_step_faces (after recv_bottom and recv_top
 * have been filled) solves the face problems, applies the corrections and
 * writes u_dev in place.
 *
 * 1D: the same entry points make a context one contiguous range of elements
 * of a periodic 1D mesh.  The fused 1D step recomputes the stages of each
 * element's neighbours itself, so what crosses a range boundary is the
 * state of the element beyond it: crkfr_set_coefficients expects
 * c[E_local + 2][n] (element 0 the left neighbour element, E_local + 1 the
 * right one); crkfr_halo_buffers gives send_bottom (the state [var][n] of
 * this range's first element, then the raw limiter indicator of its first
 * and second elements: the rank on the left stores it as its recv_top),
 * send_top (its last element's state, then the raw indicator of its last
 * and second-to-last elements: becomes the right rank's recv_bottom),
 * recv_bottom (the left neighbour's) and recv_top (the right one's),
 * `count` = vars (N+1) + 2 doubles each, in a context-owned buffer
 * allocated by crkfr_set_subdomain; crkfr_step_local (dt > 0) computes the
 * raw indicator of the range's elements when the limiter uses it and writes
 * the send blocks (without an indicator its two slots are zero);
 * crkfr_step_faces runs the step of the range with those neighbour states
 * and writes u_dev (through the context's work buffer).  The limiter needs
 * a range of at least two elements (else CRKFR_ERR_UNSUPPORTED): alpha_e of
 * the element next to the range, which the face between two ranges blends
 * with, takes the raw indicator of the element beyond it into account.
 *
 * The subcell blending limiter on 2D slabs (crkfr_set_limiter on a slab of
 * at least two element rows, else CRKFR_ERR_UNSUPPORTED) adds two exchanges
 * to a step.  Its coefficient alpha_e (Sec. 4) takes the largest neighbour's
 * raw indicator into account, and the face between two slabs blends with
 * both elements' alpha, so a limited slab step is: crkfr_step_indicator (the
 * raw indicator of the slab's own rows; nothing in CRKFR_LIMITER_FIXED
 * mode); exchange of the indicator rows (crkfr_limiter_halo_buffers kind 0:
 * send_bottom its rows 0 and 1, send_top its rows Ey_local - 2 and
 * Ey_local - 1, recv_bottom the two rows below the slab, recv_top the two
 * above, count = 2 Ex doubles, pointers into the context's indicator
 * buffers); crkfr_step_local (smoothing of alpha over the slab and the rows
 * next to it, then the local kernel); exchange of the face traces
 * (crkfr_halo_buffers) and of the limiter's face data (kind 1: the nodal
 * states, coefficients and first-order inner fluxes next to the slab's
 * boundary faces, laid out as the trace blocks, count = 8 Ex (N+1)
 * doubles); crkfr_step_faces.  The pointers stay valid until the next
 * crkfr_set_mesh.  A limited slab step equals the single-domain limited
 * step bit for bit.  crkfr_step_indicator and crkfr_limiter_halo_buffers
 * return CRKFR_ERR_STATE on a context that is not a limited 2D slab. */
crkfr_status crkfr_set_subdomain(crkfr_ctx* ctx, int32_t enable);
crkfr_status crkfr_halo_buffers(crkfr_ctx* ctx, double** send_bottom, double** send_top,
                                double** recv_bottom, double** recv_top, int64_t* count);
crkfr_status crkfr_step_local(crkfr_ctx* ctx, const double* u_dev, double dt, void* stream);
crkfr_status crkfr_step_faces(crkfr_ctx* ctx, double* u_dev, void* stream);
crkfr_status crkfr_step_indicator(crkfr_ctx* ctx, const double* u_dev, void* stream);
crkfr_status crkfr_limiter_halo_buffers(crkfr_ctx* ctx, int32_t kind, double** send_bottom,
                                        double** send_top, double** recv_bottom,
                                        double** recv_top, int64_t* count);

/* Adjoint of the step of Sec. 3, Eq. crkfr.non.cons.final (the paper has
 * no adjoint; it is this library's differentiation path).
 * Adjoint of one 2D shallow-water step with fixed dt > 0 (standard form,
 * GL nodes, no source term, context not in subdomain mode (slabs: the phased form below); otherwise
 * CRKFR_ERR_UNSUPPORTED or CRKFR_ERR_STATE).  With u^{n+1} = S(u^n; b) the step of crkfr_step
 * and a scalar J: given ubar1 = dJ/du^{n+1} (device, state layout), writes
 * ubar0 = (dS/du^n)^T ubar1 and adds (dS/db)^T ubar1 to bbar (device,
 * coefficient layout [Ey][Ex][n][n]), b being the field passed to
 * crkfr_set_coefficients.  The exact discrete adjoint of the kernels'
 * arithmetic; at the non-smooth points |m/h| uses sign(0) = 0 and the
 * maximum of two wave speeds follows the side the forward step selected.
 * u_dev is u^n and is not modified; ubar1 and ubar0 must not overlap.  The
 * simulated time is not changed.  Allocates the adjoint trace buffers on the
 * first call. */
crkfr_status crkfr_step_adjoint(crkfr_ctx* ctx, const double* u_dev, const double* ubar1_dev,
                                double* ubar0_dev, double* bbar_dev, double dt, void* stream);

/* The same adjoint step on a 2D slab (crkfr_set_subdomain; the contexts
 * crkfr_step_adjoint takes otherwise), in phases.  The slab computes the face
 * adjoints of both its boundary faces itself, so a step is:
 * crkfr_adjoint_local (the forward traces of u^n, as crkfr_step_local writes
 * them, and the y-correction sums of ubar1 the neighbouring slabs need);
 * exchange of the traces (crkfr_halo_buffers) and of the sums
 * (crkfr_adjoint_halo_buffers: send_bottom the sums of the slab's bottom
 * row's columns with g_L', which the slab below stores as its recv_top;
 * send_top those of its top row with g_R', the slab above's recv_bottom;
 * count = 3 Ex (N+1) doubles each, context-owned, valid until the next
 * crkfr_set_mesh, available after the first crkfr_adjoint_local);
 * crkfr_adjoint_faces (writes ubar0 of the slab's elements and adds the
 * gradient of their bathymetry to bbar, [Ey_local][Ex][n][n]: the halo rows
 * of the coefficient field get none here, their own slab adds it).  Equal
 * bit for bit to crkfr_step_adjoint on the whole mesh, row for row.  Both
 * phases return CRKFR_ERR_STATE on a context that is not a 2D slab. */
crkfr_status crkfr_adjoint_local(crkfr_ctx* ctx, const double* u_dev, const double* ubar1_dev,
                                 double dt, void* stream);
crkfr_status crkfr_adjoint_halo_buffers(crkfr_ctx* ctx, double** send_bottom, double** send_top,
                                        double** recv_bottom, double** recv_top,
                                        int64_t* count);
crkfr_status crkfr_adjoint_faces(crkfr_ctx* ctx, const double* u_dev, const double* ubar1_dev,
                                 double* ubar0_dev, double* bbar_dev, double dt, void* stream);

/* Recorded steps of a 2D slab (the slab form of crkfr_step_record and
 * crkfr_step_adjoint_recorded; records of crkfr_record_size doubles).
 * crkfr_step_local_record: the local phase of the step from u_dev with dt,
 * writing the face traces and the inner stage values into the record
 * (advance 1: a step, whose crkfr_step_faces_record follows; advance 0:
 * the record of the state only, u_dev and the time unchanged); then the
 * record's boundary blocks of y traces are exchanged with the neighbouring
 * slabs (crkfr_record_halo_buffers: pointers into `record`, laid out and
 * paired as those of crkfr_halo_buffers); crkfr_step_faces_record: the
 * face phase reading the traces from the record, writing u_dev.  The
 * adjoint of a recorded step: crkfr_adjoint_sums (the y-correction sums of
 * ubar1, exchanged as after crkfr_adjoint_local), then
 * crkfr_adjoint_faces_recorded, which reads the traces and stage values
 * from the record.  Equal bit for bit to the unrecorded slab step and
 * adjoint.  CRKFR_ERR_STATE on a context that is not a 2D slab. */
crkfr_status crkfr_step_local_record(crkfr_ctx* ctx, const double* u_dev, double dt,
                                     double* record, int32_t advance, void* stream);
crkfr_status crkfr_record_halo_buffers(crkfr_ctx* ctx, double* record, double** send_bottom,
                                       double** send_top, double** recv_bottom, double** recv_top,
                                       int64_t* count);
crkfr_status crkfr_step_faces_record(crkfr_ctx* ctx, double* u_dev, const double* record,
                                     void* stream);
crkfr_status crkfr_adjoint_sums(crkfr_ctx* ctx, const double* ubar1_dev, void* stream);
crkfr_status crkfr_adjoint_faces_recorded(crkfr_ctx* ctx, const double* u_dev,
                                          const double* record, const double* ubar1_dev,
                                          double* ubar0_dev, double* bbar_dev, double dt,
                                          void* stream);

/* Recorded steps for the adjoint of Sec. 3, Eq. crkfr.non.cons.final (the
 * paper has no adjoint; this is this library's differentiation path).  A
 * reverse pass that recomputes a segment of forward steps from a checkpoint
 * can keep, for each step, what the adjoint step would otherwise recompute:
 * the face traces of u^n (the Riemann problems' inputs, Eqs. numflux.cons,
 * good.numflux.non.cons) and the inner stage values 1..S-1 of Eq.
 * crkfr.non.cons.final.  Same contexts as crkfr_step_adjoint (2D slabs:
 * crkfr_step_local_record and its siblings, below; crkfr_record_size serves
 * both).
 *
 * crkfr_record_size: *count = doubles of one step record (x- and y-face
 * traces and stage values: 14 n (2 Ex Ey + 2 Ex) + 3 (S-1) Ex Ey n^2 with
 * n = N+1 and S the stages of the degree's tableau); CRKFR_ERR_STATE before
 * crkfr_set_mesh of a 2D mesh.
 *
 * crkfr_step_record: with advance = 1, one step of u_dev in place with the
 * fixed dt > 0 (as crkfr_step with nsteps = 1, advancing the simulated
 * time), whose element-local kernel writes the record of the step from the
 * input state into record_dev; with advance = 0, only the record of the
 * step from u_dev is written (u_dev and the time are unchanged).  record_dev:
 * device, caller-owned, crkfr_record_size doubles, not overlapping u_dev; its
 * layout is the library's and may change between versions.
 *
 * crkfr_step_adjoint_recorded: crkfr_step_adjoint of the step from u_dev with
 * step dt, reading the face traces and stage values from record_dev (written
 * by crkfr_step_record for the same u_dev, dt and coefficients) instead of
 * recomputing them: the forward element-local kernel is not launched and the
 * reverse local kernel does not recompute the stages.  Arguments and errors
 * otherwise as crkfr_step_adjoint. */
crkfr_status crkfr_record_size(const crkfr_ctx* ctx, int64_t* count);
crkfr_status crkfr_step_record(crkfr_ctx* ctx, double* u_dev, double dt, double* record_dev,
                               int32_t advance, void* stream);
crkfr_status crkfr_step_adjoint_recorded(crkfr_ctx* ctx, const double* u_dev,
                                         const double* record_dev, const double* ubar1_dev,
                                         double* ubar0_dev, double* bbar_dev, double dt,
                                         void* stream);

/* Subcell blending limiter of the step (Sec. 4; in 2D its tensor-product
 * extension).  Each element blends the cRK-FR update with a first-order
 * finite-volume update on its subcells of widths w_p dx (x w_q dy in 2D)
 * (Eqs. subcell.defn, low.order.update; non-conservative Rusanov fluxes of
 * Eq. combined.num.flux across every subface; a source, if any, by backward
 * Euler), u = (1 - alpha_e) u^H + alpha_e u^L (Eq. blended.scheme).  Both
 * schemes use the face flux (1 - alpha_f) F^HO + alpha_f f^LO with alpha_f
 * the mean of the two elements' alpha (Eq. Fblend).  For shallow water the
 * face flux is limited so that the two low-order node updates next to the
 * face keep h above a tenth of their first-order values (Algorithm 1; in 2D
 * on the one-direction updates with 2 dt, whose mean is the first-order
 * update), and each element's blend is limited towards its first-order
 * update so that h stays above a tenth of the smallest first-order depth
 * (Algorithm 2); h > 0 then holds when the first-order scheme on the
 * smallest subcell is positive, lam dt <= w_min dx / 2 in 1D, and in 2D the
 * same for each one-direction update with 2 dt (choose C_s accordingly).
 *
 * mode CRKFR_LIMITER_BLEND: alpha_e from the smoothness indicator of
 * Hennemann et al. (2021), on v (advection) or h (shallow water; in 2D on
 * the tensor-product modes), raised to half the largest neighbour value;
 * CRKFR_LIMITER_FIXED: alpha_e = alpha for every element (for checks);
 * CRKFR_LIMITER_NONE switches it off.  Contexts with N >= 1 only; 1D meshes
 * whole and periodic; 2D meshes whole and periodic or slabs of at least two
 * element rows (crkfr_set_subdomain, whose limited step is described there)
 * (else CRKFR_ERR_UNSUPPORTED); call after crkfr_set_mesh, which switches the
 * limiter off.  Applies to crkfr_step, crkfr_advance and crkfr_step_host, and
 * to the phased step of a 2D slab; crkfr_residual stays that of the
 * unlimited step; crkfr_step_local and crkfr_step_faces refuse limited whole
 * meshes, crkfr_step_adjoint every limited context.  A 2D context allocates the
 * limiter's buffers (one more state and 32 (Ey + 1) Ex (N+1) doubles of face
 * data) on the first call that switches it on.  crkfr_limiter_alpha copies
 * the alpha_e of the last limited step into alpha_dev (n_elem doubles,
 * element (ey, ex) at ey Ex + ex, device). */
typedef enum {
  CRKFR_LIMITER_NONE = 0,
  CRKFR_LIMITER_BLEND = 1,
  CRKFR_LIMITER_FIXED = 2
} crkfr_limiter;
crkfr_status crkfr_set_limiter(crkfr_ctx* ctx, int32_t mode, double alpha);

/* Threads per block of the fused 1D step kernel, which gives each element one
 * thread and each block threads - 2 elements between two recomputed
 * neighbours.  0 (the default): chosen per mesh among 64, 96 and 128 so that
 * the busiest SM gets the fewest threads; 64, 96 or 128: that size for every
 * step.  Only the schedule changes, not a bit of the results.  Applies to the
 * unlimited step of 1D contexts (crkfr_step, crkfr_advance, crkfr_step_host,
 * crkfr_step_local); the limited step and crkfr_residual run 128-thread
 * blocks.  CRKFR_ERR_UNSUPPORTED on a 2D context, CRKFR_ERR_ARG for other
 * values; kept across crkfr_set_mesh. */
crkfr_status crkfr_set_tile_1d(crkfr_ctx* ctx, int32_t threads);
crkfr_status crkfr_limiter_alpha(crkfr_ctx* ctx, double* alpha_dev, void* stream);

/* Simulated time and the size of the last step taken (synchronises). */
crkfr_status crkfr_get_time(crkfr_ctx* ctx, double* t_host, double* last_dt_host, void* stream);

/* Reset the simulated time to t (asynchronous).  Bookkeeping only: the
 * paper has no counterpart. */
crkfr_status crkfr_set_time(crkfr_ctx* ctx, double t, void* stream);

/* Read and clear the device status word: CRKFR_OK, or CRKFR_ERR_NONPHYSICAL
 * if any step since the last call produced h <= 0 or a non-finite value
 * (shallow water: the admissible set of Sec. 2, h > 0) or a non-finite value
 * (advection).  Synchronises. */
crkfr_status crkfr_get_status(crkfr_ctx* ctx, void* stream);

/* Number of kernel launches the context has issued (for accounting; the
 * paper has no counterpart). */
int64_t crkfr_launch_count(const crkfr_ctx* ctx);

/* Kernel timing.  While enabled, the context records a CUDA event pair on
 * the launch stream around every kernel it launches; crkfr_profile_read
 * synchronises on the recorded events and returns, for one kernel kind, the
 * launches and summed device time (ms) since profiling was enabled.
 * Enabling (again) clears the accumulated values.  Measurement aid: the
 * paper has no counterpart. */
typedef enum {
  CRKFR_KERNEL_STEP_1D = 0,    /* fused 1D step                              */
  CRKFR_KERNEL_LOCAL_2D = 1,   /* 2D element-local stages and face traces    */
  CRKFR_KERNEL_FACE_2D = 2,    /* 2D face Riemann problems, corrections, update */
  CRKFR_KERNEL_RATE = 3,       /* wave-speed rate of a state (time step)     */
  CRKFR_KERNEL_COEF = 4,       /* static coefficient terms                   */
  CRKFR_KERNEL_ADJOINT_2D = 5, /* 2D adjoint step (face and local kernels)   */
  CRKFR_KERNEL_INDICATOR = 6,  /* smoothness indicator of the limiter (1D, 2D) */
  CRKFR_KERNEL_KINDS = 7
} crkfr_kernel_kind;
crkfr_status crkfr_profile_enable(crkfr_ctx* ctx, int32_t enable);
crkfr_status crkfr_profile_read(crkfr_ctx* ctx, int32_t kind, int64_t* launches, double* total_ms);

/* (Testing aid; the paper has no counterpart.)
 * Self-check of the FP64 elementary operations the kernels implement
 * themselves instead of the IEEE division and square root: out[i] = 1/x[i]
 * (op 0), sqrt(x[i]) (op 1) or 1/sqrt(x[i]) (op 2) for n values, device
 * arrays, computed by the same device functions the step uses (FP32 seed
 * built from the bit pattern, one third-order refinement).  Lets a test
 * bound their error. */
crkfr_status crkfr_math_check(const double* x_dev, double* out_dev, int64_t n, int32_t op,
                              void* stream);

/* (Measurement aid; the paper has no counterpart.)
 * FP64 throughput probe: the peak rates the step kernels' rooflines are
 * measured against.  One launch of `blocks` blocks of CRKFR_PROBE_BLOCK
 * threads; every thread runs `iters` loop iterations of independent FP64
 * dependency chains (issue-bound, not latency-bound):
 *   mode 0: 8 FMA chains per thread on the FP64 pipe of the CUDA cores;
 *   mode 1: 4 chains of the FP64 tensor-core instruction mma.sync m8n8k4
 *           (8 x 8 x 4 FMAs per warp instruction) per warp;
 *   mode 2: both in every loop iteration (shows whether they share a unit).
 * sink_dev: device array of blocks * CRKFR_PROBE_BLOCK doubles, written
 * (keeps the work live).  *flops: the FP64 flops the launch performs (an
 * FMA counts 2).  Asynchronous on `stream`; the caller times it with events.
 * Limits: 1 <= blocks <= CRKFR_PROBE_MAX_BLOCKS, 1 <= iters <=
 * CRKFR_PROBE_MAX_ITERS (at most about 2 s of work); otherwise
 * CRKFR_ERR_ARG without a launch. */
#define CRKFR_PROBE_BLOCK 256
#define CRKFR_PROBE_MAX_BLOCKS 9728
#define CRKFR_PROBE_MAX_ITERS 65536
crkfr_status crkfr_fp64_probe(int32_t mode, int32_t blocks, int32_t iters, double* sink_dev,
                              double* flops, void* stream);

/* crkfr_step_1d_noalloc: crkfr_step for a 1D system without any device
 * memory allocation.  The paper has no counterpart to this entry point; it
 * concerns memory handling only.
 *
 * Some callers cannot let a library call cudaMalloc: applications that hand
 * out all device memory from their own pool and forbid allocations behind
 * their back, and stepping loops that may not pay the device-wide
 * synchronisation an allocation or a free can cause.  crkfr_step needs a
 * context whose crkfr_set_mesh allocates buffers.  This entry point instead
 * keeps everything it needs besides the caller's input and output (the
 * static coefficient terms, the second state buffer, the stepping state) in
 * one static device array of 2^21 doubles (16 MiB), which every GPU that
 * loads the library holds until the process exits.  It calls no cudaMalloc,
 * no cudaFree and no allocating library routine, and launches the same
 * kernels as crkfr_step.
 *
 * cfg: as for crkfr_create (a 1D system);
 * a uniform periodic mesh of n_elem elements on [lo, hi]; c_dev: the
 * coefficient field [elem][p]; u_in_dev, u_out_dev: the state
 * [var][elem][p], the same buffer or not overlapping at all; dt > 0: fixed
 * step, dt <= 0 (or -inf): the CFL step that crkfr_step uses, recomputed
 * before every step; a NaN or +inf dt returns CRKFR_ERR_ARG; nsteps >= 0
 * (0 copies u_in to u_out).
 * Limit: n_elem * (N+1) * (vars + 1) + 2 n_elem (plus alignment) must fit
 * the array, e.g. about 123,000 elements for shallow water at N = 4;
 * larger meshes return CRKFR_ERR_ARG without touching the GPU.
 * This entry point cannot report a non-physical state: the kernels' flag
 * (h <= 0 or a non-finite value) stays in the shared array and the next call
 * clears it, and in the CFL mode such a state gives a zero step, so later
 * steps leave it unchanged and the call still returns CRKFR_OK.  Callers
 * that need the check use crkfr_step and crkfr_get_status, or test the
 * output themselves.
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and the array
 * keeps the last call's contents (each call clears what must start at zero),
 * so calls that overlap on the GPU (other streams, other host threads) race.
 * Asynchronous on `stream`. */
crkfr_status crkfr_step_1d_noalloc(const crkfr_config* cfg, int64_t n_elem, double lo, double hi,
                                   const double* c_dev, const double* u_in_dev, double* u_out_dev,
                                   double dt, int64_t nsteps, void* stream);

/* Ragged ensembles of independent 1D meshes (one system, node family and
 * C_s for all; per instance its own degree, element count, interval,
 * coefficient field and, with the CFL step, its own time step).  A step of
 * the whole ensemble is one kernel launch per degree class over a work list
 * of (instance, 126-element tile) pairs running the same fused step as
 * crkfr_step (Sec. 3, Eq. crkfr.non.cons.final; Sec. 5, Eq. time.step.2d per
 * instance), so instances of any size share the GPU.  The batching itself
 * has no counterpart in the paper.
 *
 * crkfr_batch_create: cfg->system a 1D system (cfg->degree ignored); n instances with degrees[i], n_elem[i] elements on
 * [lo[i], hi[i]] (host arrays).  Allocates the batch's device buffers.
 * crkfr_batch_layout: offsets (n+1 values each, host) of every instance in
 * the packed state (instance i's u[var][elem][p] starts at state_offsets[i])
 * and in the packed coefficient field ([elem][p] at coef_offsets[i]).
 * crkfr_batch_set_coefficients: packed c (device).
 * crkfr_batch_step: nsteps steps of the packed state u in place; dt > 0: the
 * same fixed step for all, dt <= 0: each instance's own step of Sec. 5,
 * Eq. time.step.2d.  use_graph != 0 captures the whole call once into a
 * CUDA graph (re-captured when u, nsteps or dt change) and replays it on
 * `stream`.  crkfr_batch_get_times / get_status read the instances'
 * simulated times (host array of n) and the status word (synchronise). */
typedef struct crkfr_batch crkfr_batch;
crkfr_status crkfr_batch_create(crkfr_batch** out, const crkfr_config* cfg, int32_t n,
                                const int32_t* degrees, const int64_t* n_elem, const double* lo,
                                const double* hi);
void crkfr_batch_destroy(crkfr_batch* batch);
crkfr_status crkfr_batch_layout(const crkfr_batch* batch, int64_t* state_offsets,
                                int64_t* coef_offsets);
crkfr_status crkfr_batch_set_coefficients(crkfr_batch* batch, const double* c_dev, void* stream);
crkfr_status crkfr_batch_step(crkfr_batch* batch, double* u_dev, double dt, int64_t nsteps,
                              int32_t use_graph, void* stream);
crkfr_status crkfr_batch_get_times(crkfr_batch* batch, double* t_host, void* stream);

/* Launch shape of a batch step (no counterpart in the paper; it changes only
 * how the work is scheduled, never the result, which stays bitwise the same):
 * tiles_per_block (1..1024) tiles of the work list run in turn by each block
 * of a step launch; order 0 keeps the work lists in instance order, 1 puts
 * the tiles of the largest instances first; parallel 1 runs the degree
 * classes, which share no data, as concurrent branches (one stream each,
 * forked and joined around the whole call) instead of one serial chain.
 * crkfr_batch_autotune times every combination of tiles_per_block in
 * {1, 2, 4, 8}, both orders and both modes as a captured graph of `steps`
 * CFL steps of the state u_dev, on a scratch copy (u_dev and the instances'
 * times are left unchanged), keeps the fastest, and reports its time per
 * step through crkfr_batch_get_tuning.  Synchronises the stream; allocates a
 * state-sized scratch buffer for the duration of the call. */
crkfr_status crkfr_batch_set_tuning(crkfr_batch* batch, int32_t tiles_per_block, int32_t order,
                                    int32_t parallel);
crkfr_status crkfr_batch_get_tuning(const crkfr_batch* batch, int32_t* tiles_per_block,
                                    int32_t* order, int32_t* parallel, double* ms_per_step);
crkfr_status crkfr_batch_autotune(crkfr_batch* batch, const double* u_dev, int32_t steps,
                                  void* stream);
crkfr_status crkfr_batch_get_status(crkfr_batch* batch, void* stream);
int64_t crkfr_batch_launch_count(const crkfr_batch* batch);
/* Kernel timing of an ensemble (measurement aid; the paper has no
 * counterpart).  While enabled, every step kernel launched by
 * crkfr_batch_step without a graph is bracketed by a CUDA event pair on its
 * stream; crkfr_batch_profile_read synchronises on them and returns the
 * number of timed launches and their summed device time (ms) since
 * profiling was enabled.  Enabling (again) clears the sums.  Calls with a
 * graph are not timed: compare their wall time with this sum to see the
 * time between kernels. */
crkfr_status crkfr_batch_profile_enable(crkfr_batch* batch, int32_t enable);
crkfr_status crkfr_batch_profile_read(crkfr_batch* batch, int64_t* launches, double* total_ms);
const char* crkfr_batch_last_error(const crkfr_batch* batch);

/* Static strings (the paper has no counterpart).  crkfr_last_error(NULL):
 * the calling thread's last error of a call without a context. */
const char* crkfr_error_string(crkfr_status status);
const char* crkfr_last_error(const crkfr_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CRKFR_H */
