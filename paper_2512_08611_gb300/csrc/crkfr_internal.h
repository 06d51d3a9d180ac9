// Internal declarations shared by the host API and the kernels of libcrkfr.
#pragma once

#include <cstdint>
#include <string>

#include "crkfr.h"

namespace crkfr {

constexpr int kMaxN = 4;
constexpr int kMaxNodes = kMaxN + 1;

// properties of a crkfr_system value (valid values only)
inline bool sys_is_swe(int s) {
  return s == CRKFR_SYS_SWE_1D || s == CRKFR_SYS_SWE_2D || s == CRKFR_SYS_SWE_1D_WB ||
         s == CRKFR_SYS_SWE_2D_WB;
}
inline bool sys_is_wb(int s) { return s == CRKFR_SYS_SWE_1D_WB || s == CRKFR_SYS_SWE_2D_WB; }
inline bool sys_is_2d(int s) { return s == CRKFR_SYS_SWE_2D || s == CRKFR_SYS_SWE_2D_WB; }
inline int sys_vars(int s) { return s == CRKFR_SYS_VARADV_1D ? 1 : sys_is_2d(s) ? 3 : 2; }
inline bool sys_valid(int s) { return s >= CRKFR_SYS_VARADV_1D && s <= CRKFR_SYS_SWE_2D_WB; }

// Reference-element and mesh tables passed to every kernel by value, so they
// live in the kernel parameter bank (read through the constant cache) and
// several contexts with different degrees or meshes can coexist.
struct Tables {
  double Dx[kMaxNodes][kMaxNodes];  // D / dx   (Eq. diff.matrix, d/dx = (1/dx) d/dxi)
  double Dy[kMaxNodes][kMaxNodes];  // D / dy
  double l0[kMaxNodes];             // l_p(0)
  double l1[kMaxNodes];             // l_p(1)
  double gRx[kMaxNodes];            // 0.5 g_R'(xi_p) / dx, g_R'(xi_p) = l_p(1)/w_p
  double gLx[kMaxNodes];            // 0.5 g_L'(xi_p) / dx, g_L'(xi_p) = -l_p(0)/w_p
  double gRy[kMaxNodes];            // 0.5 g_R'(xi_p) / dy
  double gLy[kMaxNodes];            // 0.5 g_L'(xi_p) / dy
  double w[kMaxNodes];              // quadrature weights
  double inv_w[kMaxNodes];          // 1 / w_p
  double inv_dx, inv_dy;
  double gravity, half_gravity;
  // The kernels accumulate time averages with the weights b_i / b_ref, b_ref
  // the first non-zero weight of the tableau (so that stage is a copy);
  // b_ref multiplies dt instead, and the fluctuation term, which is not a
  // time average, uses g / b_ref.
  double b0;       // b_ref
  double face_g;   // g / b_ref
  double inv_b0;   // 1 / b_ref
  double inv_gravity;  // 1 / g (0 without gravity)
  double sqrt_gravity; // sqrt(g) (0 without gravity)
  double w2[kMaxNodes][kMaxNodes];  // w_q w_p (element means of 2D nodal fields)
  double src_coef; // source coefficient: K (linear damping) or C_f (Chezy)
  // smoothness indicator of the subcell limiter: nodal values -> coefficients
  // in the orthonormal Legendre basis, threshold T(N) and s / T
  double Vinv[kMaxNodes][kMaxNodes];
  double ind_T, ind_sharp;
};

// Subcell blending limiter of a 1D step (kernels_limit.cu).
struct LimitArgs {
  int mode;                 // CRKFR_LIMITER_*: 0 none, 1 indicator, 2 fixed alpha
  double alpha_fixed;       // alpha of mode 2
  const double* alpha_raw;  // [E] indicator before smoothing (mode 1)
  const double* cnode;      // [E][n] nodal coefficient field c
  double* alpha_out;        // [E] blending coefficient each owner used
};

// Device-resident stepping state of a context.
struct DevState {
  unsigned long long rate[3];  // max_e of the wave-speed rate, IEEE bits of a
                               // non-negative double (bit order = value order)
  double time[2];              // simulated time, double buffered
  double dt_cur;               // step size of the step in flight
  double dt_last;              // step size of the last completed step
  unsigned long long nadv;     // number of steps with dt > 0
  unsigned int status;         // bit 0: non-physical state seen
  unsigned int pad;
};

// Per-launch stepping parameters.
struct StepCtl {
  double dt_fixed;   // > 0: fixed step; otherwise CFL step from rate[slot_read]
  double cs_cfl;     // C_s * CFL(N)
  double t_end;      // CFL mode: clip the step to land on t_end (inf: none)
  int slot_read;     // rate slot of the current state
  int slot_write;    // rate slot for the new state
  int slot_reset;    // rate slot zeroed by this step
  int tslot;         // time slot read by this step
  int want_rate;     // compute the rate of the new state
  int residual;      // 1: write r = (u^{n+1}-u^n)/dt instead of u^{n+1}
  int skip_bookkeeping;  // 2D local kernel launched in row parts: 1 on all
                         // parts but the first (the step's time bookkeeping
                         // runs once)
};

struct HostBasis {
  int N = 0, n = 1;
  bool gll = false;
  double xi[kMaxNodes] = {}, w[kMaxNodes] = {};
  double D[kMaxNodes][kMaxNodes] = {};
  double l0[kMaxNodes] = {}, l1[kMaxNodes] = {};
  double gL[kMaxNodes] = {}, gR[kMaxNodes] = {};
};

// api.cu: validity of cfg->source / cfg->source_coef for cfg->system
// (CRKFR_OK, CRKFR_ERR_ARG or CRKFR_ERR_UNSUPPORTED), and the coefficient the
// kernels take (0 without a source)
crkfr_status check_source(const crkfr_config* cfg);
// api.cu: the scheme switches of cfg (rk, nc_face_mode, coef_dissipation,
// reserved) for degree N: CRKFR_OK for the built defaults, otherwise
// CRKFR_ERR_UNSUPPORTED (or CRKFR_ERR_ARG) with the reason recorded for
// crkfr_last_error(NULL)
crkfr_status check_options(const crkfr_config* cfg, int N);
// api.cu: records the reason of a failed call without a context (thread-local)
crkfr_status fail_global(crkfr_status s, const char* msg);
void clear_global_error();
double source_coef(const crkfr_config& cfg);

// basis.cpp
bool build_basis(int N, bool gll, HostBasis* out);
// CFL(N) of the explicit tableau the step uses (imex: SSP3-IMEX(4,3,3)).
double von_neumann_cfl(const HostBasis& b, bool imex);
// Kernel tables for a uniform mesh (dy ignored in 1D, pass 0); imex selects
// the weights of SSP3-IMEX(4,3,3), src_coef the source coefficient.
void fill_tables(const HostBasis& b, double dx, double dy, double gravity, bool imex,
                 double src_coef, Tables* T);

// Launchers (kernels_1d.cu / kernels_2d.cu).  Return cudaError_t as int.
struct Launch1D {
  int system;  // crkfr_system
  int N;
  bool gll;
  bool imex;   // source term with SSP3-IMEX(4,3,3)
  int64_t E;
  const double* u_in;
  double* u_out;
  const double* snode;   // [E][n]
  const double* sface;   // [E][2]
  DevState* st;
  Tables tab;            // reference element (dx = 1)
  double xs;             // 1 / dx
  StepCtl ctl;
  LimitArgs lim;         // mode 0: no limiter
  // subdomain of a larger 1D mesh: the element left of element 0 and the
  // element right of element E-1 come from here instead of the periodic
  // wrap; per side ghost_stride_1d(M, n) doubles: u [M][n] and the raw
  // limiter indicator of that element and of the one beyond it [2] (both
  // exchanged every step: ghost_dyn_1d(M, n) doubles), then the static node
  // terms [n], the face traces of c [2] and the nodal c [n] (null: periodic)
  const double* ghost;
  // threads per block of the unlimited step: 0 = chosen per mesh, else 64,
  // 96 or 128
  int tile_threads;
};
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int ghost_dyn_1d(int M, int n) { return M * n + 2; }
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int ghost_stride_1d(int M, int n) { return M * n + 2 * n + 4; }
int launch_step_1d(const Launch1D& L, void* stream);
int launch_step_1d_limit(const Launch1D& L, void* stream);   // kernels_limit.cu
int launch_alpha_1d(const Launch1D& L, double* alpha_raw, void* stream);
int launch_step_1d_imex(const Launch1D& L, void* stream);   // kernels_imex.cu
int launch_rate_1d(const Launch1D& L, int slot, void* stream);
int launch_coef_1d(int system, int N, int64_t E, const double* c, double* snode, double* sface,
                   const Tables& tab, void* stream);

// Ragged ensemble of independent 1D meshes advanced together: every block
// takes one (instance, tile) pair from a work list of one degree class.
struct BatchInstance {
  int64_t E;          // elements
  int64_t u_off;      // offset of the instance's state in the packed state
  int64_t sn_off;     // offset in the packed static node terms ([E][n])
  int64_t sf_off;     // offset in the packed face traces of c ([E][2])
  double xs;          // 1 / dx
  DevState* st;       // the instance's stepping state
};
struct WorkItem {
  int32_t inst;
  int32_t tile;
};
struct LaunchBatch1D {
  int system;
  int N;
  bool gll;
  bool imex;
  const BatchInstance* inst;
  const WorkItem* work;
  int64_t nwork;
  int64_t grid;       // blocks of the step launch (<= 0 or >= nwork: one per item)
  const double* u_in;
  double* u_out;
  const double* snode;
  const double* sface;
  Tables tab;         // reference element of degree N
  StepCtl ctl;
};
int launch_step_1d_batch(const LaunchBatch1D& B, void* stream);
int launch_step_1d_batch_imex(const LaunchBatch1D& B, void* stream);   // kernels_imex.cu
int launch_rate_1d_batch(const LaunchBatch1D& B, int slot, void* stream);
constexpr int kTile1D = 126;   // elements a 1D block owns (128 threads, 2 halo)

// Subcell blending limiter of a 2D step (kernels_limit2d.cu).
struct LimitArgs2D {
  int mode;                 // CRKFR_LIMITER_*: 0 none, 1 indicator, 2 fixed alpha
  double alpha_fixed;       // alpha of mode 2
  const double* alpha;      // [Ey][Ex] blending coefficient of the step (smoothed)
  const double* cnode;      // [Ey][Ex][n][n] nodal coefficient field c
  double* ulo;              // [3][Ey][Ex][n][n] first-order update without the
                            // element-face terms (local kernel -> face kernel)
  double* lx;               // x-face data [8][2][Ey][Ex][n]: side 0 the element's
                            // node p = 0, side 1 node p = N
  double* ly;               // y-face data [Ey+2][2][8][Ex][n], rows as the y traces
  // slab of a larger mesh (null: periodic in y): the smoothed coefficient of
  // the element rows below and above the slab, [2][Ex] (row -1, row Ey)
  const double* alpha_halo;
};

struct Launch2D {
  int N;
  bool gll;
  bool imex;             // Chezy friction with SSP3-IMEX(4,3,3)
  bool wb;               // well-balanced form
  int64_t Ex, Ey;
  const double* u_in;
  double* u_out;         // step: may equal u_in
  double* w;             // [3][Ey][Ex][n][n] scratch
  double* trx;           // x-face traces [7][2][Ey][Ex][n]
  double* try_;          // y-face traces [Ey+2][2][7][Ex][n]: element row r in buffer
                         // row r+1, halo rows 0 (row below) and Ey+1 (row above)
  const double* snode;   // [2][Ey][Ex][n][n]: g dx b, g dy b
  const double* sface;   // (g/b_0)(b+ - b-): [Ey][Ex][n] at the left x-face of each
                         // element, then [Ey+1][Ex][n] at the y-face below row k
  int periodic_y;        // 1: the local kernel fills the halo rows from its own mesh
  DevState* st;
  Tables tab;
  StepCtl ctl;
  LimitArgs2D lim;       // mode 0: no limiter
  // element rows [row_begin, row_end) the local and face kernels process
  // (for the face kernel row_begin a multiple of 8, row_end a multiple of 8
  // or Ey): the whole mesh by default
  int64_t row_begin, row_end;
  // recorded steps (crkfr_step_record): the local kernel also stores the
  // inner stage values 1..S-1, [S-1][3][Ey][Ex][n][n]
  double* stages;
  // local operator of the first stage computed ahead (the host-buffer step
  // overlaps it with the upload of the state): 1 = compute L(u^n) only and
  // store it in w; 2 = the step, reading L(u^n) from w (standard form only)
  int pre;
};
// Adjoint of one 2D step (kernels_adj2d.cu); the forward local kernel must
// have written the traces of u^n first.
struct Launch2DAdj {
  int N;
  int64_t Ex, Ey;
  double dt;
  const double* u;       // u^n
  const double* ubar1;   // adjoint of u^{n+1}
  double* ubar0;         // adjoint of u^n (written)
  double* bbar;          // adjoint of the nodal bathymetry [Ey][Ex][n][n] (accumulated)
  const double* snode;
  const double* sface;
  const double* trx;     // forward traces of u^n
  const double* try_;
  double* atrx;          // adjoint traces [7][2][Ey][Ex][n]
  double* atry;          // adjoint traces [Ey][2][7][Ex][n]
  double* gbar;          // adjoint of the face jumps: [Ey][Ex][n] x faces, [Ey][Ex][n] y faces
  // stage values 1..S-1 of the step from u^n, [S-1][3][Ey][Ex][n][n], as the
  // forward local kernel stored them (crkfr_step_record); null: recompute
  const double* stages;
  // slab of a larger mesh (null: periodic in y): the y-correction sums of
  // ubar1 of the element rows next to the slab, [3][Ex][n] each: below, the
  // sums of its top row's columns with g_R'; above, of its bottom row's
  // columns with g_L' (the face adjoint then covers the slab's Ey + 1 rows of
  // y faces, its top face included, and gbar holds Ey + 1 rows of y faces)
  const double* sums_below;
  const double* sums_above;
  Tables tab;
};
// The sums the neighbouring slabs need, [2][3][Ex][n]: the slab's bottom row
// with g_L' (for the slab below), its top row with g_R' (for the slab above).
int launch_adjoint_sums_2d(int N, int64_t Ex, int64_t Ey, const double* ubar1, const Tables& T,
                           double* send, void* stream);
// the forward local kernel (standard form, GL or GLL, no source) that also
// stores the inner stage values into L.stages (kernels_adj2d.cu)
int launch_local_2d_stages(const Launch2D& L, void* stream);
int launch_adjoint_2d(const Launch2DAdj& A, void* stream);   // A.stages null or not

int launch_local_2d(const Launch2D& L, void* stream);   // L.pre 0 or 2
int launch_local_2d_first(const Launch2D& L, void* stream);   // L_0 only (pre = 1)
int launch_local_2d_imex(const Launch2D& L, void* stream);   // kernels_imex.cu
int launch_face_2d(const Launch2D& L, void* stream);
// well-balanced instantiations (kernels_wb.cu)
int launch_step_1d_wb(const Launch1D& L, void* stream);
int launch_step_1d_batch_wb(const LaunchBatch1D& B, void* stream);
int launch_local_2d_wb(const Launch2D& L, void* stream);
int launch_face_2d_wb(const Launch2D& L, void* stream);
int launch_rate_2d(const Launch2D& L, int slot, void* stream);
// limited instantiations (kernels_limit2d.cu, kernels_limit2d_wb.cu) and the
// blending coefficients of a 2D step: indicator into alpha_raw (mode 1), then
// the smoothed (mode 1) or fixed (mode 2) coefficients into alpha
int launch_local_2d_limit(const Launch2D& L, void* stream);
int launch_face_2d_limit(const Launch2D& L, void* stream);
int launch_local_2d_limit_wb(const Launch2D& L, void* stream);
int launch_face_2d_limit_wb(const Launch2D& L, void* stream);
int launch_alpha_2d(const Launch2D& L, double* alpha_raw, double* alpha, void* stream);
// The indicator of the slab's own rows only (a slab of a larger mesh, before
// the exchange of its boundary rows) and the smoothing with the neighbours'
// raw rows: raw_below [2][Ex] (rows -2, -1), raw_above [2][Ex] (rows Ey,
// Ey + 1); writes alpha [Ey][Ex] and alpha_halo [2][Ex] (rows -1, Ey).
int launch_indicator_2d(const Launch2D& L, double* alpha_raw, void* stream);
int launch_smooth_2d_halo(const Launch2D& L, const double* alpha_raw, const double* raw_below,
                          const double* raw_above, double* alpha, double* alpha_halo,
                          void* stream);
// c: [Ey][Ex][n][n] (periodic in y) or, with halo_rows, [Ey+2][Ex][n][n]
// holding the row below and the row above the mesh as rows 0 and Ey+1
int launch_coef_2d(int N, bool gll, int64_t Ex, int64_t Ey, const double* c, bool halo_rows,
                   double* snode, double* sface, const Tables& tab, void* stream);

}  // namespace crkfr
