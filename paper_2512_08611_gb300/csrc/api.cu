// C ABI of libcrkfr (declared in include/crkfr.h): context, mesh, static
// coefficient terms, time-step control and the stepping entry points.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "crkfr.h"
#include "crkfr_internal.h"
#include "device_common.cuh"

using namespace crkfr;

// row chunks of the last face kernel of crkfr_step_host (2D), each read back
// to the host as soon as it is final
constexpr int kHostChunks = 8;

struct crkfr_ctx {
  crkfr_config cfg{};
  HostBasis basis;
  Tables tab{};
  double cfl = 0.0;
  double xs = 1.0;   // 1 / dx
  int M = 1;
  int dim = 0;
  int64_t Ex = 0, Ey = 1;
  double lo[2] = {0, 0}, hi[2] = {1, 1};
  int64_t n_state = 0, n_coef = 0;
  double* d_snode = nullptr;
  double* d_sface = nullptr;
  double* d_work = nullptr;
  double* d_trx = nullptr;
  double* d_try = nullptr;
  double* d_stage = nullptr;  // device copy of host state for crkfr_step_host
  double* d_atrx = nullptr;   // adjoint traces and face-jump adjoints (crkfr_step_adjoint)
  double* d_atry = nullptr;
  double* d_gbar = nullptr;
  double* d_cnode = nullptr;      // nodal coefficient field (subcell limiter)
  double* d_alpha_raw = nullptr;  // indicator per element before smoothing
  double* d_alpha = nullptr;      // blending coefficient of the last limited step
  double* d_ulo = nullptr;        // 2D limiter: first-order update without face terms
  double* d_lx = nullptr;         // 2D limiter: x- and y-face data
  double* d_ly = nullptr;
  double* d_ghost = nullptr;      // 1D subdomain: the two neighbour elements (Launch1D::ghost)
  double* d_send = nullptr;       // 1D subdomain: this slab's two end elements' u
  double* d_araw_halo = nullptr;  // 2D slab with the limiter: the neighbours' raw indicator,
                                  // rows -2, -1 (below) and Ey, Ey + 1 (above), [4][Ex]
  double* d_alpha_halo = nullptr; // 2D slab with the limiter: smoothed rows -1, Ey, [2][Ex]
  double* d_adj_send = nullptr;   // 2D slab adjoint: y-correction sums of ubar1 for the
  double* d_adj_recv = nullptr;   // neighbours / from them, [2][3][Ex][n] each
  double sub_dt = 0.0;            // 1D subdomain: dt of the step between local and faces
  int limit_mode = CRKFR_LIMITER_NONE;
  int tile_1d = 0;                // crkfr_set_tile_1d
  double alpha_fixed = 0.0;
  // crkfr_step_host: a copy stream and events to read finished rows of the
  // last step back while the face kernel updates the next rows
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rows[kHostChunks] = {};
  cudaEvent_t ev_in[kHostChunks] = {};   // upload parts arrived (upload_ahead)
  cudaEvent_t ev_copied = nullptr;
  DevState* d_state = nullptr;
  bool coef_set = false;
  bool subdomain = false;   // 2D slab of a larger mesh: halo rows come from outside
  int64_t nstep = 0;
  int64_t launches = 0;
  int device = -1;
  std::string err;
  // kernel timing (crkfr_profile_*)
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  int64_t prof_n[CRKFR_KERNEL_KINDS] = {};
  double prof_ms[CRKFR_KERNEL_KINDS] = {};
};

namespace {

crkfr_status fail(crkfr_ctx* c, crkfr_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

crkfr_status cuda_fail(crkfr_ctx* c, int e, const char* where) {
  return fail(c, CRKFR_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString((cudaError_t)e));
}

#define CK(ctx, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

void free_buffers(crkfr_ctx* c) {
  cudaFree(c->d_snode);
  cudaFree(c->d_sface);
  cudaFree(c->d_work);
  cudaFree(c->d_trx);
  cudaFree(c->d_try);
  cudaFree(c->d_stage);
  cudaFree(c->d_state);
  cudaFree(c->d_atrx);
  cudaFree(c->d_atry);
  cudaFree(c->d_gbar);
  cudaFree(c->d_cnode);
  cudaFree(c->d_alpha_raw);
  cudaFree(c->d_alpha);
  cudaFree(c->d_ulo);
  cudaFree(c->d_lx);
  cudaFree(c->d_ly);
  cudaFree(c->d_ghost);
  cudaFree(c->d_send);
  cudaFree(c->d_araw_halo);
  cudaFree(c->d_alpha_halo);
  cudaFree(c->d_adj_send);
  cudaFree(c->d_adj_recv);
  c->d_ghost = c->d_send = c->d_araw_halo = c->d_alpha_halo = nullptr;
  c->d_adj_send = c->d_adj_recv = nullptr;
  c->d_cnode = c->d_alpha_raw = c->d_alpha = c->d_ulo = c->d_lx = c->d_ly = nullptr;
  c->d_atrx = c->d_atry = c->d_gbar = nullptr;
  c->d_snode = c->d_sface = c->d_work = c->d_trx = c->d_try = c->d_stage = nullptr;
  c->d_state = nullptr;
}

crkfr_status check_device(crkfr_ctx* c) {
  int d = -1;
  CK(c, cudaGetDevice(&d));
  if (d != c->device) return fail(c, CRKFR_ERR_STATE, "current device differs from the mesh's device");
  return CRKFR_OK;
}

cudaEvent_t take_event(crkfr_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Runs `launch` (returns a cudaError_t as int); with profiling on, brackets
// it with an event pair on the launch stream.
template <class F>
int timed(crkfr_ctx* c, int kind, cudaStream_t s, F launch) {
  // an NVTX range per launch, named by kernel kind (visible to ncu --nvtx;
  // a no-op without a tool attached)
  static const char* const names[CRKFR_KERNEL_KINDS] = {
      "crkfr step 1d", "crkfr local 2d", "crkfr face 2d", "crkfr rate",
      "crkfr coef",    "crkfr adjoint 2d", "crkfr indicator"};
  struct Range {
    explicit Range(const char* n) { nvtxRangePushA(n); }
    ~Range() { nvtxRangePop(); }
  } range(names[kind]);
  if (!c->prof) return launch();
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (!a || !b) return launch();
  cudaEventRecord(a, s);
  const int e = launch();
  cudaEventRecord(b, s);
  c->pending.push_back({kind, a, b});
  return e;
}

// Synchronises on the pending event pairs and accumulates their durations.
crkfr_status drain_profile(crkfr_ctx* c, bool keep) {
  crkfr_status st = CRKFR_OK;
  for (auto& r : c->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      st = cuda_fail(c, e, "profile events");
    } else if (keep) {
      c->prof_n[r.kind] += 1;
      c->prof_ms[r.kind] += ms;
    }
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
  return st;
}

__global__ void k_math_check(const double* __restrict__ x, double* __restrict__ out, int64_t n,
                             int op) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = op == 0 ? drcp(x[i]) : op == 1 ? dsqrt_pos(x[i]) : drsqrt_pos(x[i]);
}

// the two end elements' states of a 1D subdomain: send[side][v][p]
// The two end elements of a 1D range for its neighbours, per side
// ghost_dyn_1d(M, n) doubles: u [M][n] of the end element, then the raw
// limiter indicator of the end element and of the next one inwards (raw
// null, no indicator: zeros; raw needs E >= 2).
__global__ void k_pack_ends_1d(const double* __restrict__ u, const double* __restrict__ raw,
                               double* __restrict__ send, int64_t E, int M, int n) {
  const int per = ghost_dyn_1d(M, n);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * per) return;
  const int side = i / per, j = i - side * per;
  if (j < M * n) {
    const int v = j / n, p = j - v * n;
    send[i] = u[((int64_t)v * E + (side ? E - 1 : 0)) * n + p];
  } else {
    const int k = j - M * n;   // 0: the end element, 1: the next one inwards
    send[i] = raw ? raw[side ? E - 1 - k : k] : 0.0;
  }
}

__global__ void k_set_time(DevState* st, int slot, double t) {
  st->time[slot] = t;
  st->time[slot ^ 1] = t;
}

Launch1D make1d(crkfr_ctx* c) {
  Launch1D L{};
  L.system = c->cfg.system;
  L.N = c->cfg.degree;
  L.gll = c->cfg.nodes == CRKFR_NODES_GLL;
  L.imex = c->cfg.source != CRKFR_SRC_NONE;
  L.E = c->Ex;
  L.snode = c->d_snode;
  L.sface = c->d_sface;
  L.st = c->d_state;
  L.tab = c->tab;
  L.xs = c->xs;
  L.lim.mode = c->limit_mode;
  L.lim.alpha_fixed = c->alpha_fixed;
  L.lim.alpha_raw = c->d_alpha_raw;
  L.lim.cnode = c->d_cnode;
  L.lim.alpha_out = c->d_alpha;
  L.ghost = c->subdomain ? c->d_ghost : nullptr;
  L.tile_threads = c->tile_1d;
  return L;
}

Launch2D make2d(crkfr_ctx* c) {
  Launch2D L{};
  L.N = c->cfg.degree;
  L.gll = c->cfg.nodes == CRKFR_NODES_GLL;
  L.imex = c->cfg.source != CRKFR_SRC_NONE;
  L.wb = sys_is_wb(c->cfg.system);
  L.Ex = c->Ex;
  L.Ey = c->Ey;
  L.w = c->d_work;
  L.trx = c->d_trx;
  L.try_ = c->d_try;
  L.snode = c->d_snode;
  L.sface = c->d_sface;
  L.st = c->d_state;
  L.tab = c->tab;
  L.periodic_y = c->subdomain ? 0 : 1;
  L.row_begin = 0;
  L.row_end = c->Ey;
  return L;
}

crkfr_status ready(crkfr_ctx* c) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  if (!c->coef_set) return fail(c, CRKFR_ERR_STATE, "no coefficients set");
  return check_device(c);
}

// The limiter's arguments of a 2D launch (mode none: left empty).  On a slab
// of a larger mesh the face kernel takes the smoothed coefficient of the
// rows next to the slab from alpha_halo.
void fill_limit_2d(crkfr_ctx* c, Launch2D& L) {
  if (c->limit_mode == CRKFR_LIMITER_NONE) return;
  L.lim.mode = c->limit_mode;
  L.lim.alpha_fixed = c->alpha_fixed;
  L.lim.alpha = c->d_alpha;
  L.lim.cnode = c->d_cnode;
  L.lim.ulo = c->d_ulo;
  L.lim.lx = c->d_lx;
  L.lim.ly = c->d_ly;
  L.lim.alpha_halo = c->subdomain ? c->d_alpha_halo : nullptr;
}

// A subdomain with the limiter: a 1D range of at least two elements, a 2D
// slab of at least two element rows (the two elements / rows of raw
// indicator each neighbour needs) with the halo rows' buffers.
crkfr_status check_limited_slab(crkfr_ctx* c) {
  if (c->dim == 1) {
    // a range sends the raw indicator of its two end elements per side
    if (c->Ex < 2) return fail(c, CRKFR_ERR_UNSUPPORTED, "a limited range needs two elements");
    return CRKFR_OK;
  }
  if (c->Ey < 2) return fail(c, CRKFR_ERR_UNSUPPORTED, "a limited slab needs two element rows");
  if (c->d_araw_halo) return CRKFR_OK;
  if (cudaMalloc(&c->d_araw_halo, sizeof(double) * 4 * c->Ex) != cudaSuccess ||
      cudaMalloc(&c->d_alpha_halo, sizeof(double) * 2 * c->Ex) != cudaSuccess) {
    cudaFree(c->d_araw_halo);
    cudaFree(c->d_alpha_halo);
    c->d_araw_halo = c->d_alpha_halo = nullptr;
    cudaGetLastError();
    return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
  }
  CK(c, cudaMemset(c->d_araw_halo, 0, sizeof(double) * 4 * c->Ex));
  CK(c, cudaMemset(c->d_alpha_halo, 0, sizeof(double) * 2 * c->Ex));
  return CRKFR_OK;
}

// rate of state u (max over elements of the wave-speed rate) into `slot`
crkfr_status launch_rate(crkfr_ctx* c, const double* u, int slot, cudaStream_t s) {
  CK(c, cudaMemsetAsync(&c->d_state->rate[slot], 0, sizeof(unsigned long long), s));
  int e;
  if (c->dim == 1) {
    Launch1D L = make1d(c);
    L.u_in = u;
    e = timed(c, CRKFR_KERNEL_RATE, s, [&] { return launch_rate_1d(L, slot, s); });
  } else {
    Launch2D L = make2d(c);
    L.u_in = u;
    e = timed(c, CRKFR_KERNEL_RATE, s, [&] { return launch_rate_2d(L, slot, s); });
  }
  if (e) return cuda_fail(c, e, "rate kernel");
  c->launches += 1;
  return CRKFR_OK;
}

// The local and face kernels of a 2D step in up to 5 parts of element rows,
// each part's rows of u (contiguous per variable) copied to
// host_out on the copy stream as soon as its face kernel has finished, while
// the later parts compute; the stream s then waits for the last copy.  The
// face kernel of part k needs the local kernel of the rows next to it, so the
// order is: local of the last part (the periodic neighbour of row 0), local
// of part 0, then local of part k+1 before the face kernel of part k.  The
// local kernels read only their own rows of u, which no earlier face kernel
// of this step writes.  The first local launch does the step's bookkeeping.
crkfr_status ensure_copy_stream(crkfr_ctx* c) {
  if (!c->copy_stream) {
    CK(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    for (auto& ev : c->ev_rows) CK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (auto& ev : c->ev_in) CK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(c, cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
  }
  return CRKFR_OK;
}

crkfr_status step_with_readback(crkfr_ctx* c, Launch2D L, const double* u, double* host_out,
                                cudaStream_t s) {
  crkfr_status sc = ensure_copy_stream(c);
  if (sc != CRKFR_OK) return sc;
  const int64_t Ey = c->Ey, Ne = c->Ex * c->Ey;
  const int64_t nn = (int64_t)c->basis.n * c->basis.n;
  // parts of decreasing size, 6:4:3:2:1 of the rows in multiples of 8 rows:
  // each part's read-back overlaps the compute of the later ones, and only
  // the last, smallest part's read-back ends the step (fewer launches than
  // equal parts with as short a tail)
  static constexpr int kCum[5] = {6, 10, 13, 15, 16};
  int64_t ends[5];
  int parts = 0;
  for (int i = 0; i < 5; ++i) {
    const int64_t e = i == 4 ? Ey : (Ey * kCum[i] / 16) / 8 * 8;
    if (e > (parts ? ends[parts - 1] : 0)) ends[parts++] = e;
  }
  auto r_begin = [&](int k) { return k == 0 ? (int64_t)0 : ends[k - 1]; };
  auto r_end = [&](int k) { return ends[k]; };
  bool first = true;
  auto local_part = [&](int k) -> crkfr_status {
    Launch2D P = L;
    P.row_begin = r_begin(k);
    P.row_end = r_end(k);
    P.ctl.skip_bookkeeping = first ? 0 : 1;
    first = false;
    int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(P, s); });
    if (e) return cuda_fail(c, e, "2D local kernel");
    c->launches += 1;
    return CRKFR_OK;
  };
  auto face_part = [&](int k) -> crkfr_status {
    Launch2D P = L;
    P.row_begin = r_begin(k);
    P.row_end = r_end(k);
    int e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(P, s); });
    if (e) return cuda_fail(c, e, "2D face kernel");
    c->launches += 1;
    CK(c, cudaEventRecord(c->ev_rows[k], s));
    CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_rows[k], 0));
    const size_t off = (size_t)(P.row_begin * c->Ex) * nn;
    const size_t bytes = sizeof(double) * (size_t)((P.row_end - P.row_begin) * c->Ex) * nn;
    for (int v = 0; v < 3; ++v)
      CK(c, cudaMemcpyAsync(host_out + v * Ne * nn + off, u + v * Ne * nn + off, bytes,
                            cudaMemcpyDeviceToHost, c->copy_stream));
    return CRKFR_OK;
  };
  crkfr_status st;
  if (parts > 1 && (st = local_part(parts - 1)) != CRKFR_OK) return st;
  if ((st = local_part(0)) != CRKFR_OK) return st;
  for (int k = 0; k < parts; ++k) {
    if (k + 1 <= parts - 2 && (st = local_part(k + 1)) != CRKFR_OK) return st;
    if ((st = face_part(k)) != CRKFR_OK) return st;
  }
  CK(c, cudaEventRecord(c->ev_copied, c->copy_stream));
  CK(c, cudaStreamWaitEvent(s, c->ev_copied, 0));
  return CRKFR_OK;
}

// The upload of a host state for crkfr_step_host (2D standard form): the
// rows are copied in parts on the copy stream, and as soon as a part has
// arrived the compute stream computes its wave-speed rate (CFL mode) and the
// first stage's local operator L(u^n), which needs no time step, into the
// work buffer; the step then starts from those (run_steps, first_ahead).  So
// that work, about an eighth of the step, overlaps the upload, which the CFL
// step cannot otherwise overlap: its time step needs the rate of every
// element.
crkfr_status upload_ahead(crkfr_ctx* c, const double* host_in, double* u, bool cfl_mode,
                          cudaStream_t s) {
  crkfr_status st = ensure_copy_stream(c);
  if (st != CRKFR_OK) return st;
  const int64_t Ey = c->Ey, Ne = c->Ex * c->Ey;
  const int64_t nn = (int64_t)c->basis.n * c->basis.n;
  int64_t rows = (Ey + kHostChunks - 1) / kHostChunks;
  rows = (rows + 7) / 8 * 8;
  const int parts = (int)((Ey + rows - 1) / rows);
  const int slot = (int)(c->nstep % 3);
  if (cfl_mode) CK(c, cudaMemsetAsync(c->d_state->rate, 0, sizeof(c->d_state->rate), s));
  // the copies into u follow everything queued on s before this call
  CK(c, cudaEventRecord(c->ev_copied, s));
  CK(c, cudaStreamWaitEvent(c->copy_stream, c->ev_copied, 0));
  for (int k = 0; k < parts; ++k) {
    const int64_t rb = (int64_t)k * rows, re = rb + rows < Ey ? rb + rows : Ey;
    const size_t off = (size_t)(rb * c->Ex) * nn;
    const size_t bytes = sizeof(double) * (size_t)((re - rb) * c->Ex) * nn;
    for (int v = 0; v < c->M; ++v)
      CK(c, cudaMemcpyAsync(u + v * Ne * nn + off, host_in + v * Ne * nn + off, bytes,
                            cudaMemcpyHostToDevice, c->copy_stream));
    CK(c, cudaEventRecord(c->ev_in[k], c->copy_stream));
    CK(c, cudaStreamWaitEvent(s, c->ev_in[k], 0));
    Launch2D L = make2d(c);
    L.u_in = u;
    L.row_begin = rb;
    L.row_end = re;
    if (cfl_mode) {
      int e = timed(c, CRKFR_KERNEL_RATE, s, [&] { return launch_rate_2d(L, slot, s); });
      if (e) return cuda_fail(c, e, "rate kernel");
      c->launches += 1;
    }
    int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d_first(L, s); });
    if (e) return cuda_fail(c, e, "2D local kernel (first stage)");
    c->launches += 1;
  }
  return CRKFR_OK;
}

// nsteps steps of u in place.  dt > 0 fixed, otherwise CFL (clipped to t_end).
// host_out (2D, optional): the last step runs in row parts and each part's
// rows are copied to host_out on the context's copy stream as soon as they
// are final (step_with_readback); the caller's stream waits for the copies.
// *copied tells whether that happened.
crkfr_status run_steps(crkfr_ctx* c, double* u, double dt, int64_t nsteps, double t_end,
                       cudaStream_t s, double* host_out = nullptr, bool* copied = nullptr,
                       bool first_ahead = false) {
  if (copied) *copied = false;
  if (nsteps <= 0) return CRKFR_OK;
  const bool cfl_mode = !(dt > 0.0);
  // first_ahead (2D standard form): the caller has already computed the
  // first stage's local operator of u into the work buffer and, in the CFL
  // mode, the rate of u into slot nstep % 3 (upload_ahead)
  if (cfl_mode && !first_ahead) {
    CK(c, cudaMemsetAsync(c->d_state->rate, 0, sizeof(c->d_state->rate), s));
    crkfr_status st = launch_rate(c, u, (int)(c->nstep % 3), s);
    if (st != CRKFR_OK) return st;
  }
  StepCtl ctl{};
  ctl.dt_fixed = cfl_mode ? 0.0 : dt;
  ctl.cs_cfl = c->cfg.cfl_safety * c->cfl;
  ctl.t_end = t_end;
  ctl.want_rate = cfl_mode ? 1 : 0;
  ctl.residual = 0;
  if (c->dim == 1) {
    // ping-pong between u and the work buffer, ending in u
    double* bufs[2] = {u, c->d_work};
    int cur = 0;
    if (nsteps % 2 == 1) {
      CK(c, cudaMemcpyAsync(c->d_work, u, sizeof(double) * c->n_state, cudaMemcpyDeviceToDevice, s));
      cur = 1;
    }
    Launch1D L = make1d(c);
    for (int64_t k = 0; k < nsteps; ++k) {
      ctl.slot_read = (int)(c->nstep % 3);
      ctl.slot_write = (int)((c->nstep + 1) % 3);
      ctl.slot_reset = (int)((c->nstep + 2) % 3);
      ctl.tslot = (int)(c->nstep % 2);
      // (the last step's rate would go unread: every call starts from the
      // rate of its input)
      ctl.want_rate = cfl_mode && k + 1 < nsteps ? 1 : 0;
      L.ctl = ctl;
      L.u_in = bufs[cur];
      L.u_out = bufs[cur ^ 1];
      if (c->limit_mode == CRKFR_LIMITER_BLEND) {
        int ea = timed(c, CRKFR_KERNEL_INDICATOR, s,
                       [&] { return launch_alpha_1d(L, c->d_alpha_raw, s); });
        if (ea) return cuda_fail(c, ea, "indicator kernel");
        c->launches += 1;
      }
      int e = timed(c, CRKFR_KERNEL_STEP_1D, s, [&] { return launch_step_1d(L, s); });
      if (e) return cuda_fail(c, e, "1D step kernel");
      c->launches += 1;
      c->nstep += 1;
      cur ^= 1;
    }
  } else {
    Launch2D L = make2d(c);
    fill_limit_2d(c, L);
    for (int64_t k = 0; k < nsteps; ++k) {
      ctl.slot_read = (int)(c->nstep % 3);
      ctl.slot_write = (int)((c->nstep + 1) % 3);
      ctl.slot_reset = (int)((c->nstep + 2) % 3);
      ctl.tslot = (int)(c->nstep % 2);
      ctl.want_rate = cfl_mode && k + 1 < nsteps ? 1 : 0;
      L.ctl = ctl;
      L.u_in = u;
      L.u_out = u;
      L.pre = (first_ahead && k == 0) ? 2 : 0;
      if (c->limit_mode != CRKFR_LIMITER_NONE) {
        int ea = timed(c, CRKFR_KERNEL_INDICATOR, s,
                       [&] { return launch_alpha_2d(L, c->d_alpha_raw, c->d_alpha, s); });
        if (ea) return cuda_fail(c, ea, "indicator kernels");
        c->launches += c->limit_mode == CRKFR_LIMITER_BLEND ? 2 : 1;
      }
      if (host_out && k == nsteps - 1) {
        crkfr_status st = step_with_readback(c, L, u, host_out, s);
        if (st != CRKFR_OK) return st;
        if (copied) *copied = true;
      } else {
        int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(L, s); });
        if (e) return cuda_fail(c, e, "2D local kernel");
        e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(L, s); });
        if (e) return cuda_fail(c, e, "2D face kernel");
        c->launches += 2;
      }
      c->nstep += 1;
    }
  }
  return CRKFR_OK;
}

}  // namespace

namespace crkfr {

crkfr_status check_source(const crkfr_config* cfg) {
  if (cfg->source == CRKFR_SRC_NONE) return CRKFR_OK;
  if (cfg->source != CRKFR_SRC_LINEAR_DAMPING && cfg->source != CRKFR_SRC_CHEZY)
    return CRKFR_ERR_ARG;
  if (!(cfg->source_coef >= 0.0) || !std::isfinite(cfg->source_coef)) return CRKFR_ERR_ARG;
  const bool swe = sys_is_swe(cfg->system);
  if (cfg->source == CRKFR_SRC_LINEAR_DAMPING && cfg->system != CRKFR_SYS_VARADV_1D)
    return CRKFR_ERR_UNSUPPORTED;
  if (cfg->source == CRKFR_SRC_CHEZY && !swe) return CRKFR_ERR_UNSUPPORTED;
  return CRKFR_OK;
}

double source_coef(const crkfr_config& cfg) {
  return cfg.source == CRKFR_SRC_NONE ? 0.0 : cfg.source_coef;
}

thread_local std::string g_last_error;

crkfr_status fail_global(crkfr_status s, const char* msg) {
  g_last_error = msg;
  return s;
}

void clear_global_error() { g_last_error.clear(); }

crkfr_status check_options(const crkfr_config* cfg, int N) {
  if (cfg->reserved != 0) return fail_global(CRKFR_ERR_ARG, "crkfr_config.reserved must be 0");
  const int order = cfg->source != CRKFR_SRC_NONE ? 3 : N + 1;
  if (cfg->rk != 0 && cfg->rk != order)
    return fail_global(CRKFR_ERR_UNSUPPORTED,
                       "rk: only the default tableau is built (order N+1 without a source, "
                       "3 with one)");
  if (cfg->nc_face_mode == CRKFR_NC_LITERAL || cfg->nc_face_mode == CRKFR_NC_STAGEWISE)
    return fail_global(CRKFR_ERR_UNSUPPORTED,
                       "nc_face_mode: only the frozen face terms are built (the literal and "
                       "stagewise readings exist in the CPU oracle)");
  if (cfg->nc_face_mode != CRKFR_NC_FROZEN)
    return fail_global(CRKFR_ERR_ARG, "nc_face_mode: not a crkfr_nc_face value");
  if (cfg->coef_dissipation == 1)
    return fail_global(CRKFR_ERR_UNSUPPORTED,
                       "coef_dissipation: only the static coefficient is built");
  if (cfg->coef_dissipation != 0) return fail_global(CRKFR_ERR_ARG, "coef_dissipation: 0 or 1");
  return CRKFR_OK;
}

}  // namespace crkfr

extern "C" {

const char* crkfr_error_string(crkfr_status s) {
  switch (s) {
    case CRKFR_OK: return "ok";
    case CRKFR_ERR_ARG: return "invalid argument";
    case CRKFR_ERR_UNSUPPORTED: return "unsupported system, degree or node family";
    case CRKFR_ERR_CUDA: return "CUDA runtime error";
    case CRKFR_ERR_NONPHYSICAL: return "non-physical state (h <= 0 or non-finite value)";
    case CRKFR_ERR_STATE: return "call out of order";
    case CRKFR_ERR_ALLOC: return "allocation failed";
  }
  return "unknown status";
}

const char* crkfr_last_error(const crkfr_ctx* c) {
  return c ? c->err.c_str() : g_last_error.c_str();
}

int64_t crkfr_launch_count(const crkfr_ctx* c) { return c ? c->launches : 0; }


crkfr_status crkfr_create(crkfr_ctx** out, const crkfr_config* cfg) {
  clear_global_error();
  if (!out) return fail_global(CRKFR_ERR_ARG, "null argument");
  *out = nullptr;
  if (!cfg) return fail_global(CRKFR_ERR_ARG, "null argument");
  if (!sys_valid(cfg->system)) return fail_global(CRKFR_ERR_UNSUPPORTED, "unknown system");
  if (crkfr_status st = check_source(cfg); st != CRKFR_OK)
    return fail_global(st, "source term invalid or not built for this system");
  if (cfg->nodes != CRKFR_NODES_GL && cfg->nodes != CRKFR_NODES_GLL)
    return fail_global(CRKFR_ERR_UNSUPPORTED, "unknown node family");
  const int minN = (sys_is_2d(cfg->system) || cfg->nodes == CRKFR_NODES_GLL) ? 1 : 0;
  if (cfg->degree < minN || cfg->degree > kMaxN)
    return fail_global(CRKFR_ERR_UNSUPPORTED, "degree not built for this system and node family");
  if (!(cfg->cfl_safety > 0.0) || cfg->cfl_safety > 1.0)
    return fail_global(CRKFR_ERR_ARG, "cfl_safety must lie in (0, 1]");
  if (cfg->system != CRKFR_SYS_VARADV_1D && !(cfg->gravity > 0.0))
    return fail_global(CRKFR_ERR_ARG, "gravity must be positive");
  if (crkfr_status st = check_options(cfg, cfg->degree); st != CRKFR_OK) return st;
  crkfr_ctx* c = new (std::nothrow) crkfr_ctx();
  if (!c) return fail_global(CRKFR_ERR_ALLOC, "host allocation failed");
  c->cfg = *cfg;
  c->M = sys_vars(cfg->system);
  if (!build_basis(cfg->degree, cfg->nodes == CRKFR_NODES_GLL, &c->basis)) {
    delete c;
    return CRKFR_ERR_UNSUPPORTED;
  }
  c->cfl = cfg->cfl_number > 0.0 ? cfg->cfl_number
                                 : von_neumann_cfl(c->basis, cfg->source != CRKFR_SRC_NONE);
  *out = c;
  return CRKFR_OK;
}

void crkfr_destroy(crkfr_ctx* c) {
  if (!c) return;
  if (c->dim != 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_buffers(c);
    for (auto& r : c->pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->copy_stream) {
      cudaStreamDestroy(c->copy_stream);
      for (auto ev : c->ev_rows) cudaEventDestroy(ev);
      for (auto ev : c->ev_in) cudaEventDestroy(ev);
      cudaEventDestroy(c->ev_copied);
    }
    if (prev != c->device && prev >= 0) cudaSetDevice(prev);
  }
  delete c;
}

crkfr_status crkfr_set_mesh(crkfr_ctx* c, int32_t dim, const int64_t* n_elem, const double* lo,
                            const double* hi, int32_t periodic_mask) {
  if (!c || !n_elem || !lo || !hi) return fail(c, CRKFR_ERR_ARG, "null argument");
  const int want = sys_is_2d(c->cfg.system) ? 2 : 1;
  if (dim != want) return fail(c, CRKFR_ERR_ARG, "dimension does not match the system");
  if (periodic_mask < 0 || periodic_mask >= (1 << dim))
    return fail(c, CRKFR_ERR_ARG, "periodic_mask has bits beyond the mesh's dimension");
  if (periodic_mask != (1 << dim) - 1)
    return fail(c, CRKFR_ERR_UNSUPPORTED, "only periodic meshes are built");
  for (int d = 0; d < dim; ++d) {
    if (n_elem[d] <= 0) return fail(c, CRKFR_ERR_ARG, "element count must be positive");
    if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
      return fail(c, CRKFR_ERR_ARG, "need lo < hi, finite");
  }
  const int n = c->basis.n;
  const int64_t Ex = n_elem[0], Ey = dim == 2 ? n_elem[1] : 1;
  const int64_t Ne = Ex * Ey;
  if (Ne > (int64_t)1 << 31 || Ne * n * n * c->M > ((int64_t)1 << 40))
    return fail(c, CRKFR_ERR_ARG, "mesh too large");
  if (c->dim != 0) {
    cudaDeviceSynchronize();
    free_buffers(c);
  }
  c->dim = 0;
  c->coef_set = false;
  CK(c, cudaGetDevice(&c->device));
  const int64_t nodes = dim == 2 ? Ne * n * n : Ne * n;
  c->Ex = Ex;
  c->Ey = Ey;
  c->n_state = nodes * c->M;
  c->n_coef = nodes;
  for (int d = 0; d < 2; ++d) {
    c->lo[d] = d < dim ? lo[d] : 0.0;
    c->hi[d] = d < dim ? hi[d] : 1.0;
  }
  const double dx = (c->hi[0] - c->lo[0]) / (double)Ex;
  const double dy = (c->hi[1] - c->lo[1]) / (double)Ey;
  // 1D kernels take reference-element tables and 1/dx as a scalar
  fill_tables(c->basis, dim == 2 ? dx : 1.0, dim == 2 ? dy : 0.0,
              c->cfg.system == CRKFR_SYS_VARADV_1D ? 0.0 : c->cfg.gravity,
              c->cfg.source != CRKFR_SRC_NONE, source_coef(c->cfg), &c->tab);
  c->xs = (double)Ex / (c->hi[0] - c->lo[0]);   // 1/dx, as the batch path computes it

  size_t sn, sf;
  if (dim == 1) {
    sn = (size_t)Ne * n;
    sf = (size_t)Ne * 2;
  } else {
    sn = (size_t)2 * Ne * n * n;
    sf = (size_t)(2 * Ne + Ex) * n;
  }
  if (cudaMalloc(&c->d_snode, sizeof(double) * sn) != cudaSuccess ||
      cudaMalloc(&c->d_sface, sizeof(double) * sf) != cudaSuccess ||
      cudaMalloc(&c->d_work, sizeof(double) * c->n_state) != cudaSuccess ||
      cudaMalloc(&c->d_state, sizeof(DevState)) != cudaSuccess) {
    free_buffers(c);
    cudaGetLastError();
    return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
  }
  c->limit_mode = CRKFR_LIMITER_NONE;
  {
    const size_t cn = dim == 1 ? (size_t)Ne * n : (size_t)Ne * n * n;
    if (cudaMalloc(&c->d_cnode, sizeof(double) * cn) != cudaSuccess ||
        cudaMalloc(&c->d_alpha_raw, sizeof(double) * Ne) != cudaSuccess ||
        cudaMalloc(&c->d_alpha, sizeof(double) * Ne) != cudaSuccess) {
      free_buffers(c);
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
    CK(c, cudaMemset(c->d_alpha, 0, sizeof(double) * Ne));
  }
  if (dim == 2) {
    const size_t trx = (size_t)7 * 2 * Ne * n;
    const size_t try_ = (size_t)7 * 2 * (Ey + 2) * Ex * n;
    if (cudaMalloc(&c->d_trx, sizeof(double) * trx) != cudaSuccess ||
        cudaMalloc(&c->d_try, sizeof(double) * try_) != cudaSuccess) {
      free_buffers(c);
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
  }
  CK(c, cudaMemset(c->d_state, 0, sizeof(DevState)));
  c->nstep = 0;
  c->dim = dim;
  return CRKFR_OK;
}

crkfr_status crkfr_sizes(const crkfr_ctx* c, int64_t* n_state, int64_t* n_coef) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return CRKFR_ERR_STATE;
  if (n_state) *n_state = c->n_state;
  if (n_coef) *n_coef = c->n_coef;
  return CRKFR_OK;
}

crkfr_status crkfr_get_nodes(const crkfr_ctx* c, double* xi, double* w) {
  if (!c || !xi || !w) return CRKFR_ERR_ARG;
  for (int i = 0; i < c->basis.n; ++i) {
    xi[i] = c->basis.xi[i];
    w[i] = c->basis.w[i];
  }
  return CRKFR_OK;
}

crkfr_status crkfr_get_cfl(const crkfr_ctx* c, double* cfl) {
  if (!c || !cfl) return CRKFR_ERR_ARG;
  *cfl = c->cfl;
  return CRKFR_OK;
}

crkfr_status crkfr_set_coefficients(crkfr_ctx* c, const double* coef, void* stream) {
  if (!c || !coef) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  crkfr_status st = check_device(c);
  if (st != CRKFR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int e;
  e = timed(c, CRKFR_KERNEL_COEF, s, [&] {
    if (c->dim == 1 && c->subdomain) {
      // coef[E + 2][n]: the left neighbour element, the subdomain, the right
      // neighbour element; the neighbours' static terms go to the ghosts
      const int n = c->basis.n, gs = ghost_stride_1d(c->M, n), gd = ghost_dyn_1d(c->M, n);
      int r = launch_coef_1d(c->cfg.system, c->cfg.degree, c->Ex, coef + n, c->d_snode,
                             c->d_sface, c->tab, s);
      for (int side = 0; side < 2 && !r; ++side) {
        double* g = c->d_ghost + side * gs;
        const double* ce = coef + (side ? c->Ex + 1 : 0) * n;
        r = launch_coef_1d(c->cfg.system, c->cfg.degree, 1, ce, g + gd, g + gd + n, c->tab, s);
        // the nodal c of the ghost element (the limiter's first-order fluxes)
        if (!r)
          r = (int)cudaMemcpyAsync(g + gd + n + 2, ce, sizeof(double) * n,
                                   cudaMemcpyDeviceToDevice, s);
      }
      return r;
    }
    if (c->dim == 1)
      return launch_coef_1d(c->cfg.system, c->cfg.degree, c->Ex, coef, c->d_snode, c->d_sface,
                            c->tab, s);
    return launch_coef_2d(c->cfg.degree, c->cfg.nodes == CRKFR_NODES_GLL, c->Ex, c->Ey, coef,
                          c->subdomain, c->d_snode, c->d_sface, c->tab, s);
  });
  if (e) return cuda_fail(c, e, "coefficient kernel");
  c->launches += 1;
  // the limiter's first-order fluxes read the nodal field of the context's
  // own elements (a subdomain's coefficients start with a halo row/element)
  const int64_t halo = !c->subdomain ? 0 : c->dim == 2 ? c->Ex * c->basis.n * c->basis.n
                                                      : c->basis.n;
  CK(c, cudaMemcpyAsync(c->d_cnode, coef + halo, sizeof(double) * c->n_coef,
                        cudaMemcpyDeviceToDevice, s));
  c->coef_set = true;
  return CRKFR_OK;
}

crkfr_status crkfr_set_limiter(crkfr_ctx* c, int32_t mode, double alpha) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  if (mode < CRKFR_LIMITER_NONE || mode > CRKFR_LIMITER_FIXED)
    return fail(c, CRKFR_ERR_ARG, "unknown limiter mode");
  if (mode != CRKFR_LIMITER_NONE) {
    if (c->cfg.degree < 1) return fail(c, CRKFR_ERR_UNSUPPORTED, "the limiter needs N >= 1");
    if (c->subdomain) {
      crkfr_status hs = check_limited_slab(c);
      if (hs != CRKFR_OK) return hs;
    }
  }
  if (mode == CRKFR_LIMITER_FIXED && !(alpha >= 0.0 && alpha <= 1.0))
    return fail(c, CRKFR_ERR_ARG, "alpha must lie in [0, 1]");
  if (mode != CRKFR_LIMITER_NONE && c->dim == 2 && !c->d_ulo) {
    const int64_t n = c->basis.n, Ne = c->Ex * c->Ey;
    const size_t lx = (size_t)8 * 2 * Ne * n, ly = (size_t)8 * 2 * (c->Ey + 2) * c->Ex * n;
    if (cudaMalloc(&c->d_ulo, sizeof(double) * c->n_state) != cudaSuccess ||
        cudaMalloc(&c->d_lx, sizeof(double) * lx) != cudaSuccess ||
        cudaMalloc(&c->d_ly, sizeof(double) * ly) != cudaSuccess) {
      cudaFree(c->d_ulo);
      cudaFree(c->d_lx);
      cudaFree(c->d_ly);
      c->d_ulo = c->d_lx = c->d_ly = nullptr;
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
  }
  c->limit_mode = mode;
  c->alpha_fixed = mode == CRKFR_LIMITER_FIXED ? alpha : 0.0;
  return CRKFR_OK;
}

crkfr_status crkfr_set_tile_1d(crkfr_ctx* c, int32_t threads) {
  if (!c) return CRKFR_ERR_ARG;
  if (sys_is_2d(c->cfg.system))
    return fail(c, CRKFR_ERR_UNSUPPORTED, "the tile size is a setting of the 1D step");
  if (threads != 0 && threads != 64 && threads != 96 && threads != 128)
    return fail(c, CRKFR_ERR_ARG, "threads must be 0, 64, 96 or 128");
  c->tile_1d = threads;
  return CRKFR_OK;
}

crkfr_status crkfr_limiter_alpha(crkfr_ctx* c, double* alpha_dev, void* stream) {
  if (!c || !alpha_dev) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  CK(c, cudaMemcpyAsync(alpha_dev, c->d_alpha, sizeof(double) * c->Ex * c->Ey,
                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return CRKFR_OK;
}

crkfr_status crkfr_compute_dt(crkfr_ctx* c, const double* u, double* dt_host, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (!u || !dt_host) return fail(c, CRKFR_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  // slot 0 is free between calls: every stepping call re-initialises its slots
  st = launch_rate(c, u, 0, s);
  if (st != CRKFR_OK) return st;
  unsigned long long bits = 0;
  CK(c, cudaMemcpyAsync(&bits, &c->d_state->rate[0], sizeof(bits), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  double rate;
  std::memcpy(&rate, &bits, sizeof(rate));
  if (!(rate > 0.0) || !std::isfinite(rate)) {
    *dt_host = 0.0;
    return fail(c, CRKFR_ERR_NONPHYSICAL, "wave-speed rate is not positive and finite");
  }
  *dt_host = (c->cfg.cfl_safety * c->cfl) / rate;
  return CRKFR_OK;
}

crkfr_status crkfr_residual(crkfr_ctx* c, const double* u, double dt, double* r, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->subdomain) return fail(c, CRKFR_ERR_STATE, "subdomain: use crkfr_step_local / faces");
  if (!u || !r) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  const size_t bytes = sizeof(double) * c->n_state;
  const char *a = (const char*)u, *b = (const char*)r;
  if (a < b + bytes && b < a + bytes) return fail(c, CRKFR_ERR_ARG, "u and r overlap");
  cudaStream_t s = (cudaStream_t)stream;
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.residual = 1;
  int e;
  if (c->dim == 1) {
    Launch1D L = make1d(c);
    L.ctl = ctl;
    L.u_in = u;
    L.u_out = r;
    e = timed(c, CRKFR_KERNEL_STEP_1D, s, [&] { return launch_step_1d(L, s); });
    c->launches += 1;
  } else {
    Launch2D L = make2d(c);
    L.ctl = ctl;
    L.u_in = u;
    L.u_out = r;
    e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(L, s); });
    if (!e) e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(L, s); });
    c->launches += 2;
  }
  if (e) return cuda_fail(c, e, "residual kernels");
  return CRKFR_OK;
}

crkfr_status crkfr_step(crkfr_ctx* c, double* u, double dt, int64_t nsteps, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->subdomain) return fail(c, CRKFR_ERR_STATE, "subdomain: use crkfr_step_local / faces");
  if (!u) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (nsteps < 0) return fail(c, CRKFR_ERR_ARG, "nsteps must be >= 0");
  if (std::isnan(dt) || (std::isinf(dt) && dt > 0.0))
    return fail(c, CRKFR_ERR_ARG, "dt must be finite (or <= 0 for the CFL step)");
  return run_steps(c, u, dt, nsteps, std::numeric_limits<double>::infinity(),
                   (cudaStream_t)stream);
}

crkfr_status crkfr_advance(crkfr_ctx* c, double* u, double t_end, int64_t max_steps,
                           int64_t* steps_taken, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->subdomain) return fail(c, CRKFR_ERR_STATE, "subdomain: use crkfr_step_local / faces");
  if (!u || !std::isfinite(t_end) || max_steps < 0) return fail(c, CRKFR_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int64_t done = 0;
  double t = 0.0;
  unsigned long long nadv0 = 0, nadv = 0;
  const int64_t chunk = 16;
  for (int first = 1;; first = 0) {
    DevState h;
    CK(c, cudaMemcpyAsync(&h, c->d_state, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    t = h.time[c->nstep % 2];
    nadv = h.nadv;
    if (first) nadv0 = nadv;
    if (t >= t_end) break;
    if (done >= max_steps) break;
    const int64_t k = (max_steps - done) < chunk ? (max_steps - done) : chunk;
    st = run_steps(c, u, 0.0, k, t_end, s);
    if (st != CRKFR_OK) return st;
    done += k;
  }
  if (steps_taken) *steps_taken = (int64_t)(nadv - nadv0);
  if (t < t_end) return fail(c, CRKFR_ERR_ARG, "t_end not reached within max_steps");
  return CRKFR_OK;
}

crkfr_status crkfr_step_host(crkfr_ctx* c, const double* u_in, double* u_out, double dt,
                             int64_t nsteps, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->subdomain) return fail(c, CRKFR_ERR_STATE, "subdomain: use crkfr_step_local / faces");
  if (!u_in || !u_out || nsteps < 0) return fail(c, CRKFR_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * c->n_state;
  if (!c->d_stage) {
    if (cudaMalloc(&c->d_stage, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
  }
  // 2D standard form: the upload runs in parts, overlapped with the rate and
  // the first stage's local operator of the parts already there; otherwise
  // one copy.  The last step's rows are read back while the face kernel
  // finishes the rows after them.
  const bool ahead = c->dim == 2 && nsteps > 0 && c->cfg.system == CRKFR_SYS_SWE_2D &&
                     c->cfg.source == CRKFR_SRC_NONE && c->limit_mode == CRKFR_LIMITER_NONE;
  if (ahead) {
    st = upload_ahead(c, u_in, c->d_stage, !(dt > 0.0), s);
    if (st != CRKFR_OK) {
      if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
      cudaStreamSynchronize(s);
      return st;
    }
  } else {
    CK(c, cudaMemcpyAsync(c->d_stage, u_in, bytes, cudaMemcpyHostToDevice, s));
  }
  bool copied = false;
  st = run_steps(c, c->d_stage, dt, nsteps, std::numeric_limits<double>::infinity(), s,
                 c->dim == 2 ? u_out : nullptr, &copied, ahead);
  if (st != CRKFR_OK) {
    // copies already queued on the copy stream still target u_out
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    cudaStreamSynchronize(s);
    return st;
  }
  if (!copied) CK(c, cudaMemcpyAsync(u_out, c->d_stage, bytes, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  return CRKFR_OK;
}

crkfr_status crkfr_set_subdomain(crkfr_ctx* c, int32_t enable) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  if (enable && c->limit_mode != CRKFR_LIMITER_NONE) {
    crkfr_status hs = check_limited_slab(c);
    if (hs != CRKFR_OK) return hs;
  }
  if (enable && c->dim == 1 && !c->d_ghost) {
    const int n = c->basis.n;
    if (cudaMalloc(&c->d_ghost, sizeof(double) * 2 * ghost_stride_1d(c->M, n)) != cudaSuccess ||
        cudaMalloc(&c->d_send, sizeof(double) * 2 * ghost_dyn_1d(c->M, n)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
    CK(c, cudaMemset(c->d_ghost, 0, sizeof(double) * 2 * ghost_stride_1d(c->M, n)));
  }
  c->subdomain = enable != 0;
  c->coef_set = false;
  return CRKFR_OK;
}

crkfr_status crkfr_halo_buffers(crkfr_ctx* c, double** send_bottom, double** send_top,
                                double** recv_bottom, double** recv_top, int64_t* count) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 1) {
    // the end elements' states (left = bottom, right = top) and the ghosts
    if (!c->subdomain || !c->d_ghost) return fail(c, CRKFR_ERR_STATE, "not a 1D subdomain");
    const int64_t gd = ghost_dyn_1d(c->M, c->basis.n);
    if (send_bottom) *send_bottom = c->d_send;
    if (send_top) *send_top = c->d_send + gd;
    if (recv_bottom) *recv_bottom = c->d_ghost;
    if (recv_top) *recv_top = c->d_ghost + ghost_stride_1d(c->M, c->basis.n);
    if (count) *count = gd;
    return CRKFR_OK;
  }
  if (c->dim != 2) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  const int64_t n = c->basis.n;
  const int64_t block = 7 * c->Ex * n;           // one (row, side) block of the y traces
  double* base = c->d_try;
  auto at = [&](int64_t row, int side) { return base + (row * 2 + side) * block; };
  if (send_bottom) *send_bottom = at(1, 0);       // bottom row, bottom side
  if (send_top) *send_top = at(c->Ey, 1);         // top row, top side
  if (recv_bottom) *recv_bottom = at(0, 1);       // halo below: top side of the row below
  if (recv_top) *recv_top = at(c->Ey + 1, 0);     // halo above: bottom side of the row above
  if (count) *count = block;
  return CRKFR_OK;
}

crkfr_status crkfr_step_local(crkfr_ctx* c, const double* u, double dt, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->limit_mode != CRKFR_LIMITER_NONE && !c->subdomain)
    return fail(c, CRKFR_ERR_UNSUPPORTED, "limited steps of a whole mesh run through crkfr_step");
  if (!u) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->dim == 1) {
    // 1D: the fused step recomputes the neighbours' stages itself, so the
    // local phase only packs this range's end elements for the exchange,
    // with the limiter's raw indicator of the two elements at each end
    if (!c->subdomain) return fail(c, CRKFR_ERR_STATE, "phased 1D steps need a subdomain");
    const bool raw = c->limit_mode == CRKFR_LIMITER_BLEND;
    if (raw) {
      Launch1D L = make1d(c);
      L.u_in = u;
      int ea = timed(c, CRKFR_KERNEL_INDICATOR, s,
                     [&] { return launch_alpha_1d(L, c->d_alpha_raw, s); });
      if (ea) return cuda_fail(c, ea, "indicator kernel");
      c->launches += 1;
    }
    const int n = c->basis.n, total = 2 * ghost_dyn_1d(c->M, n);
    k_pack_ends_1d<<<(total + 127) / 128, 128, 0, s>>>(u, raw ? c->d_alpha_raw : nullptr,
                                                       c->d_send, c->Ex, c->M, n);
    CK(c, cudaGetLastError());
    c->launches += 1;
    c->sub_dt = dt;
    return CRKFR_OK;
  }
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.cs_cfl = c->cfg.cfl_safety * c->cfl;
  ctl.t_end = std::numeric_limits<double>::infinity();
  ctl.slot_read = (int)(c->nstep % 3);
  ctl.slot_write = (int)((c->nstep + 1) % 3);
  ctl.slot_reset = (int)((c->nstep + 2) % 3);
  ctl.tslot = (int)(c->nstep % 2);
  Launch2D L = make2d(c);
  fill_limit_2d(c, L);
  L.ctl = ctl;
  L.u_in = u;
  L.u_out = nullptr;
  if (c->limit_mode != CRKFR_LIMITER_NONE) {
    // the blending coefficient of the slab's rows and of the rows next to it,
    // from the raw indicator of crkfr_step_indicator and the neighbours' rows
    int ea = timed(c, CRKFR_KERNEL_INDICATOR, s, [&] {
      return launch_smooth_2d_halo(L, c->d_alpha_raw, c->d_araw_halo, c->d_araw_halo + 2 * c->Ex,
                                   c->d_alpha, c->d_alpha_halo, s);
    });
    if (ea) return cuda_fail(c, ea, "indicator smoothing kernel");
    c->launches += 1;
  }
  int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D local kernel");
  c->launches += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_step_indicator(crkfr_ctx* c, const double* u, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (!u) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (c->dim != 2 || !c->subdomain) return fail(c, CRKFR_ERR_STATE, "not a 2D slab");
  if (c->limit_mode == CRKFR_LIMITER_NONE) return fail(c, CRKFR_ERR_STATE, "no limiter set");
  cudaStream_t s = (cudaStream_t)stream;
  Launch2D L = make2d(c);
  fill_limit_2d(c, L);
  L.u_in = u;
  int e = timed(c, CRKFR_KERNEL_INDICATOR, s,
                [&] { return launch_indicator_2d(L, c->d_alpha_raw, s); });
  if (e) return cuda_fail(c, e, "indicator kernel");
  if (c->limit_mode == CRKFR_LIMITER_BLEND) c->launches += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_limiter_halo_buffers(crkfr_ctx* c, int32_t kind, double** send_bottom,
                                        double** send_top, double** recv_bottom,
                                        double** recv_top, int64_t* count) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim != 2 || !c->subdomain) return fail(c, CRKFR_ERR_STATE, "not a 2D slab");
  if (c->limit_mode == CRKFR_LIMITER_NONE || !c->d_araw_halo || !c->d_ly)
    return fail(c, CRKFR_ERR_STATE, "no limiter set");
  const int64_t Ex = c->Ex, Ey = c->Ey, n = c->basis.n;
  if (kind == 0) {
    // raw indicator: rows 0, 1 go down, rows Ey-2, Ey-1 go up; rows -2, -1
    // and Ey, Ey+1 come in
    if (send_bottom) *send_bottom = c->d_alpha_raw;
    if (send_top) *send_top = c->d_alpha_raw + (Ey - 2) * Ex;
    if (recv_bottom) *recv_bottom = c->d_araw_halo;
    if (recv_top) *recv_top = c->d_araw_halo + 2 * Ex;
    if (count) *count = 2 * Ex;
    return CRKFR_OK;
  }
  if (kind != 1) return fail(c, CRKFR_ERR_ARG, "kind must be 0 (indicator) or 1 (face data)");
  // y-face data, rows as the y traces: one (row, side) block of 8 fields
  const int64_t block = 8 * Ex * n;
  auto at = [&](int64_t row, int side) { return c->d_ly + (row * 2 + side) * block; };
  if (send_bottom) *send_bottom = at(1, 0);
  if (send_top) *send_top = at(Ey, 1);
  if (recv_bottom) *recv_bottom = at(0, 1);
  if (recv_top) *recv_top = at(Ey + 1, 0);
  if (count) *count = block;
  return CRKFR_OK;
}

crkfr_status crkfr_step_faces(crkfr_ctx* c, double* u, void* stream) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->limit_mode != CRKFR_LIMITER_NONE && !c->subdomain)
    return fail(c, CRKFR_ERR_UNSUPPORTED, "limited steps of a whole mesh run through crkfr_step");
  if (!u) return fail(c, CRKFR_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->dim == 1) {
    // 1D: the whole fused step with the received ghosts, into the work
    // buffer (the step reads neighbour elements of the same time level),
    // then back into u
    if (!c->subdomain) return fail(c, CRKFR_ERR_STATE, "phased 1D steps need a subdomain");
    if (!(c->sub_dt > 0.0)) return fail(c, CRKFR_ERR_STATE, "crkfr_step_local first");
    StepCtl ctl{};
    ctl.dt_fixed = c->sub_dt;
    ctl.cs_cfl = c->cfg.cfl_safety * c->cfl;
    ctl.t_end = std::numeric_limits<double>::infinity();
    ctl.slot_read = (int)(c->nstep % 3);
    ctl.slot_write = (int)((c->nstep + 1) % 3);
    ctl.slot_reset = (int)((c->nstep + 2) % 3);
    ctl.tslot = (int)(c->nstep % 2);
    Launch1D L = make1d(c);
    L.ctl = ctl;
    L.u_in = u;
    L.u_out = c->d_work;
    int e = timed(c, CRKFR_KERNEL_STEP_1D, s, [&] { return launch_step_1d(L, s); });
    if (e) return cuda_fail(c, e, "1D step kernel");
    CK(c, cudaMemcpyAsync(u, c->d_work, sizeof(double) * c->n_state, cudaMemcpyDeviceToDevice, s));
    c->launches += 1;
    c->nstep += 1;
    c->sub_dt = 0.0;
    return CRKFR_OK;
  }
  StepCtl ctl{};
  ctl.dt_fixed = 1.0;   // the face kernel reads the step size the local phase stored
  ctl.slot_write = (int)((c->nstep + 1) % 3);
  ctl.want_rate = 0;
  Launch2D L = make2d(c);
  fill_limit_2d(c, L);
  L.ctl = ctl;
  L.u_in = u;
  L.u_out = u;
  int e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D face kernel");
  c->launches += 1;
  c->nstep += 1;
  return CRKFR_OK;
}

}  // extern "C"

namespace {

// The contexts the adjoint (and the recorded step) support.
crkfr_status adjoint_context(crkfr_ctx* c, bool slab = false) {
  crkfr_status st = ready(c);
  if (st != CRKFR_OK) return st;
  if (c->dim != 2 || c->cfg.system != CRKFR_SYS_SWE_2D)
    return fail(c, CRKFR_ERR_UNSUPPORTED,
                "the adjoint step is built for 2D shallow water in its standard form");
  if (c->cfg.nodes != CRKFR_NODES_GL) return fail(c, CRKFR_ERR_UNSUPPORTED, "GL nodes only");
  if (c->cfg.source != CRKFR_SRC_NONE)
    return fail(c, CRKFR_ERR_UNSUPPORTED, "the adjoint step has no source term");
  if (c->subdomain != slab)
    return fail(c, CRKFR_ERR_STATE, slab ? "the phased adjoint is a step of a 2D slab"
                                         : "subdomain: use crkfr_adjoint_local / faces");
  if (c->limit_mode != CRKFR_LIMITER_NONE)
    return fail(c, CRKFR_ERR_UNSUPPORTED, "the adjoint step has no limiter");
  return CRKFR_OK;
}

// Parts of a step record: x-face traces, y-face traces (with the two halo
// rows), inner stage values 1..S-1 (doubles each).
void record_parts(const crkfr_ctx* c, int64_t* ntx, int64_t* nty, int64_t* nst) {
  const int64_t n = c->basis.n, Ne = c->Ex * c->Ey;
  *ntx = 7 * 2 * Ne * n;
  *nty = 7 * 2 * (c->Ey + 2) * c->Ex * n;
  *nst = (int64_t)(tab_stages(c->cfg.degree) - 1) * 3 * Ne * n * n;
}

// A 2D slab's buffers of the adjoint's y-correction sums (sent and received).
crkfr_status ensure_adjoint_sums(crkfr_ctx* c) {
  if (c->d_adj_send) return CRKFR_OK;
  const int64_t sums = (int64_t)2 * 3 * c->Ex * c->basis.n;
  if (cudaMalloc(&c->d_adj_send, sizeof(double) * sums) != cudaSuccess ||
      cudaMalloc(&c->d_adj_recv, sizeof(double) * sums) != cudaSuccess) {
    cudaFree(c->d_adj_send);
    cudaFree(c->d_adj_recv);
    c->d_adj_send = c->d_adj_recv = nullptr;
    cudaGetLastError();
    return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
  }
  CK(c, cudaMemset(c->d_adj_recv, 0, sizeof(double) * sums));
  return CRKFR_OK;
}

// The adjoint kernels of one step whose forward traces of u^n are in
// (trx, try_) and whose stage values are in `stages` (null: recomputed).
crkfr_status launch_adjoint(crkfr_ctx* c, const double* u, const double* ubar1, double* ubar0,
                            double* bbar, double dt, const double* trx, const double* try_,
                            const double* stages, cudaStream_t s) {
  Launch2DAdj A{};
  A.N = c->cfg.degree;
  A.Ex = c->Ex;
  A.Ey = c->Ey;
  A.dt = dt;
  A.u = u;
  A.ubar1 = ubar1;
  A.ubar0 = ubar0;
  A.bbar = bbar;
  A.snode = c->d_snode;
  A.sface = c->d_sface;
  A.trx = trx;
  A.try_ = try_;
  A.atrx = c->d_atrx;
  A.atry = c->d_atry;
  A.gbar = c->d_gbar;
  A.stages = stages;
  if (c->subdomain) {
    A.sums_below = c->d_adj_recv;
    A.sums_above = c->d_adj_recv + 3 * c->Ex * c->basis.n;
  }
  A.tab = c->tab;
  int e = timed(c, CRKFR_KERNEL_ADJOINT_2D, s, [&] { return launch_adjoint_2d(A, s); });
  if (e) return cuda_fail(c, e, "2D adjoint kernels");
  c->launches += 2;
  return CRKFR_OK;
}

crkfr_status adjoint_args(crkfr_ctx* c, const double* u, const double* ubar1, double* ubar0,
                          double* bbar, double dt) {
  if (!u || !ubar1 || !ubar0 || !bbar) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  const size_t bytes = sizeof(double) * c->n_state;
  const char *a = (const char*)ubar1, *o = (const char*)ubar0;
  if (a < o + bytes && o < a + bytes) return fail(c, CRKFR_ERR_ARG, "ubar1 and ubar0 overlap");
  const int64_t n = c->basis.n, Ne = c->Ex * c->Ey;
  if (!c->d_atrx) {
    const size_t tr = (size_t)7 * 2 * Ne * n;
    if (cudaMalloc(&c->d_atrx, sizeof(double) * tr) != cudaSuccess ||
        cudaMalloc(&c->d_atry, sizeof(double) * tr) != cudaSuccess ||
        cudaMalloc(&c->d_gbar, sizeof(double) * (2 * Ne + c->Ex) * n) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CRKFR_ERR_ALLOC, "device allocation failed");
    }
  }
  return CRKFR_OK;
}

}  // namespace

extern "C" {

crkfr_status crkfr_step_adjoint(crkfr_ctx* c, const double* u, const double* ubar1, double* ubar0,
                                double* bbar, double dt, void* stream) {
  crkfr_status st = adjoint_context(c);
  if (st == CRKFR_OK) st = adjoint_args(c, u, ubar1, ubar0, bbar, dt);
  if (st != CRKFR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // forward traces of u^n: the local kernel in its residual form (same traces,
  // no time bookkeeping)
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.residual = 1;
  Launch2D L = make2d(c);
  L.ctl = ctl;
  L.u_in = u;
  int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D local kernel");
  c->launches += 1;
  return launch_adjoint(c, u, ubar1, ubar0, bbar, dt, c->d_trx, c->d_try, nullptr, s);
}

// The adjoint step of a 2D slab in phases.  Each slab recomputes the face
// adjoints of both its boundary faces (the slab below has the same face at
// its top), so what crosses a slab boundary is the forward traces (the
// exchange of crkfr_halo_buffers) and the y-correction sums of ubar1 of the
// rows next to the slab; the bathymetry gradient of a slab's elements stays
// with that slab.
crkfr_status crkfr_adjoint_local(crkfr_ctx* c, const double* u, const double* ubar1, double dt,
                                 void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st != CRKFR_OK) return st;
  if (!u || !ubar1) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  st = ensure_adjoint_sums(c);
  if (st != CRKFR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // forward traces of u^n (the local kernel in its residual form) and the
  // sums the neighbouring slabs need
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.residual = 1;
  Launch2D L = make2d(c);
  L.ctl = ctl;
  L.u_in = u;
  int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D local kernel");
  e = launch_adjoint_sums_2d(c->cfg.degree, c->Ex, c->Ey, ubar1, c->tab, c->d_adj_send, s);
  if (e) return cuda_fail(c, e, "adjoint sums kernel");
  c->launches += 2;
  return CRKFR_OK;
}

crkfr_status crkfr_adjoint_halo_buffers(crkfr_ctx* c, double** send_bottom, double** send_top,
                                        double** recv_bottom, double** recv_top,
                                        int64_t* count) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim != 2 || !c->subdomain) return fail(c, CRKFR_ERR_STATE, "not a 2D slab");
  if (!c->d_adj_send) return fail(c, CRKFR_ERR_STATE, "crkfr_adjoint_local first");
  const int64_t per = 3 * c->Ex * c->basis.n;
  if (send_bottom) *send_bottom = c->d_adj_send;
  if (send_top) *send_top = c->d_adj_send + per;
  if (recv_bottom) *recv_bottom = c->d_adj_recv;
  if (recv_top) *recv_top = c->d_adj_recv + per;
  if (count) *count = per;
  return CRKFR_OK;
}

crkfr_status crkfr_adjoint_faces(crkfr_ctx* c, const double* u, const double* ubar1,
                                 double* ubar0, double* bbar, double dt, void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st == CRKFR_OK) st = adjoint_args(c, u, ubar1, ubar0, bbar, dt);
  if (st != CRKFR_OK) return st;
  if (!c->d_adj_send) return fail(c, CRKFR_ERR_STATE, "crkfr_adjoint_local first");
  return launch_adjoint(c, u, ubar1, ubar0, bbar, dt, c->d_trx, c->d_try, nullptr,
                        (cudaStream_t)stream);
}

// Recorded steps of a 2D slab: the local phase writes the face traces and
// the inner stage values into the record, the record's halo rows of y traces
// are exchanged, and the face phase reads the traces from the record.
crkfr_status crkfr_step_local_record(crkfr_ctx* c, const double* u, double dt, double* record,
                                     int32_t advance, void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st != CRKFR_OK) return st;
  if (!u || !record) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  if (advance != 0 && advance != 1) return fail(c, CRKFR_ERR_ARG, "advance must be 0 or 1");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  const size_t rbytes = sizeof(double) * (size_t)(tx + ty + ns);
  const size_t ubytes = sizeof(double) * c->n_state;
  const char *a = (const char*)u, *r = (const char*)record;
  if (a < r + rbytes && r < a + ubytes) return fail(c, CRKFR_ERR_ARG, "u and record overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Launch2D L = make2d(c);
  L.trx = record;
  L.try_ = record + tx;
  L.stages = record + tx + ty;
  L.u_in = u;
  L.u_out = nullptr;
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.cs_cfl = c->cfg.cfl_safety * c->cfl;
  ctl.t_end = std::numeric_limits<double>::infinity();
  if (!advance) {
    ctl.residual = 1;   // traces and stages only, no time bookkeeping
  } else {
    ctl.slot_read = (int)(c->nstep % 3);
    ctl.slot_write = (int)((c->nstep + 1) % 3);
    ctl.slot_reset = (int)((c->nstep + 2) % 3);
    ctl.tslot = (int)(c->nstep % 2);
  }
  L.ctl = ctl;
  int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d_stages(L, s); });
  if (e) return cuda_fail(c, e, "2D local kernel");
  c->launches += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_record_halo_buffers(crkfr_ctx* c, double* record, double** send_bottom,
                                       double** send_top, double** recv_bottom, double** recv_top,
                                       int64_t* count) {
  if (!c || !record) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (c->dim != 2 || !c->subdomain) return fail(c, CRKFR_ERR_STATE, "not a 2D slab");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  const int64_t block = 7 * c->Ex * c->basis.n;   // as crkfr_halo_buffers, in the record
  auto at = [&](int64_t row, int side) { return record + tx + (row * 2 + side) * block; };
  if (send_bottom) *send_bottom = at(1, 0);
  if (send_top) *send_top = at(c->Ey, 1);
  if (recv_bottom) *recv_bottom = at(0, 1);
  if (recv_top) *recv_top = at(c->Ey + 1, 0);
  if (count) *count = block;
  return CRKFR_OK;
}

crkfr_status crkfr_step_faces_record(crkfr_ctx* c, double* u, const double* record,
                                     void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st != CRKFR_OK) return st;
  if (!u || !record) return fail(c, CRKFR_ERR_ARG, "null argument");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  cudaStream_t s = (cudaStream_t)stream;
  StepCtl ctl{};
  ctl.dt_fixed = 1.0;   // the face kernel reads the step size the local phase stored
  ctl.slot_write = (int)((c->nstep + 1) % 3);
  ctl.want_rate = 0;
  Launch2D L = make2d(c);
  // (the face kernel only reads the traces)
  L.trx = const_cast<double*>(record);
  L.try_ = const_cast<double*>(record) + tx;
  L.ctl = ctl;
  L.u_in = u;
  L.u_out = u;
  int e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D face kernel");
  c->launches += 1;
  c->nstep += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_adjoint_sums(crkfr_ctx* c, const double* ubar1, void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st != CRKFR_OK) return st;
  if (!ubar1) return fail(c, CRKFR_ERR_ARG, "null argument");
  st = ensure_adjoint_sums(c);
  if (st != CRKFR_OK) return st;
  int e = launch_adjoint_sums_2d(c->cfg.degree, c->Ex, c->Ey, ubar1, c->tab, c->d_adj_send,
                                 (cudaStream_t)stream);
  if (e) return cuda_fail(c, e, "adjoint sums kernel");
  c->launches += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_adjoint_faces_recorded(crkfr_ctx* c, const double* u, const double* record,
                                          const double* ubar1, double* ubar0, double* bbar,
                                          double dt, void* stream) {
  crkfr_status st = adjoint_context(c, true);
  if (st == CRKFR_OK) st = adjoint_args(c, u, ubar1, ubar0, bbar, dt);
  if (st != CRKFR_OK) return st;
  if (!record) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!c->d_adj_send) return fail(c, CRKFR_ERR_STATE, "crkfr_adjoint_sums first");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  return launch_adjoint(c, u, ubar1, ubar0, bbar, dt, record, record + tx, record + tx + ty,
                        (cudaStream_t)stream);
}

crkfr_status crkfr_record_size(const crkfr_ctx* c, int64_t* count) {
  if (!c || !count) return CRKFR_ERR_ARG;
  if (c->dim != 2) return CRKFR_ERR_STATE;
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  *count = tx + ty + ns;
  return CRKFR_OK;
}

crkfr_status crkfr_step_record(crkfr_ctx* c, double* u, double dt, double* record,
                               int32_t advance, void* stream) {
  crkfr_status st = adjoint_context(c);
  if (st != CRKFR_OK) return st;
  if (!u || !record) return fail(c, CRKFR_ERR_ARG, "null argument");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, CRKFR_ERR_ARG, "dt must be positive");
  if (advance != 0 && advance != 1) return fail(c, CRKFR_ERR_ARG, "advance must be 0 or 1");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  const size_t rbytes = sizeof(double) * (size_t)(tx + ty + ns);
  const size_t ubytes = sizeof(double) * c->n_state;
  const char *a = (const char*)u, *r = (const char*)record;
  if (a < r + rbytes && r < a + ubytes) return fail(c, CRKFR_ERR_ARG, "u and record overlap");
  cudaStream_t s = (cudaStream_t)stream;
  Launch2D L = make2d(c);
  L.trx = record;
  L.try_ = record + tx;
  L.stages = record + tx + ty;
  L.u_in = u;
  L.u_out = u;
  StepCtl ctl{};
  ctl.dt_fixed = dt;
  ctl.cs_cfl = c->cfg.cfl_safety * c->cfl;
  ctl.t_end = std::numeric_limits<double>::infinity();
  if (!advance) {
    // traces and stages only (residual form: no time bookkeeping, u unchanged)
    ctl.residual = 1;
    L.ctl = ctl;
    int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d_stages(L, s); });
    if (e) return cuda_fail(c, e, "2D local kernel");
    c->launches += 1;
    return CRKFR_OK;
  }
  ctl.slot_read = (int)(c->nstep % 3);
  ctl.slot_write = (int)((c->nstep + 1) % 3);
  ctl.slot_reset = (int)((c->nstep + 2) % 3);
  ctl.tslot = (int)(c->nstep % 2);
  L.ctl = ctl;
  int e = timed(c, CRKFR_KERNEL_LOCAL_2D, s, [&] { return launch_local_2d_stages(L, s); });
  if (e) return cuda_fail(c, e, "2D local kernel");
  e = timed(c, CRKFR_KERNEL_FACE_2D, s, [&] { return launch_face_2d(L, s); });
  if (e) return cuda_fail(c, e, "2D face kernel");
  c->launches += 2;
  c->nstep += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_step_adjoint_recorded(crkfr_ctx* c, const double* u, const double* record,
                                         const double* ubar1, double* ubar0, double* bbar,
                                         double dt, void* stream) {
  crkfr_status st = adjoint_context(c);
  if (st == CRKFR_OK) st = adjoint_args(c, u, ubar1, ubar0, bbar, dt);
  if (st != CRKFR_OK) return st;
  if (!record) return fail(c, CRKFR_ERR_ARG, "null argument");
  int64_t tx, ty, ns;
  record_parts(c, &tx, &ty, &ns);
  return launch_adjoint(c, u, ubar1, ubar0, bbar, dt, record, record + tx, record + tx + ty,
                        (cudaStream_t)stream);
}

crkfr_status crkfr_get_time(crkfr_ctx* c, double* t_host, double* last_dt_host, void* stream) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  crkfr_status st = check_device(c);
  if (st != CRKFR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DevState h;
  CK(c, cudaMemcpyAsync(&h, c->d_state, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  if (t_host) *t_host = h.time[c->nstep % 2];
  if (last_dt_host) *last_dt_host = h.dt_last;
  return CRKFR_OK;
}

crkfr_status crkfr_set_time(crkfr_ctx* c, double t, void* stream) {
  if (!c || !std::isfinite(t)) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  crkfr_status st = check_device(c);
  if (st != CRKFR_OK) return st;
  k_set_time<<<1, 1, 0, (cudaStream_t)stream>>>(c->d_state, (int)(c->nstep % 2), t);
  CK(c, cudaGetLastError());
  c->launches += 1;
  return CRKFR_OK;
}

crkfr_status crkfr_math_check(const double* x, double* out, int64_t n, int32_t op, void* stream) {
  if (!x || !out || n < 0 || op < 0 || op > 2) return CRKFR_ERR_ARG;
  if (n == 0) return CRKFR_OK;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffff) return CRKFR_ERR_ARG;
  k_math_check<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, out, n, op);
  return cudaGetLastError() == cudaSuccess ? CRKFR_OK : CRKFR_ERR_CUDA;
}

crkfr_status crkfr_profile_enable(crkfr_ctx* c, int32_t enable) {
  if (!c) return CRKFR_ERR_ARG;
  crkfr_status st = drain_profile(c, false);
  for (int k = 0; k < CRKFR_KERNEL_KINDS; ++k) {
    c->prof_n[k] = 0;
    c->prof_ms[k] = 0.0;
  }
  c->prof = enable != 0;
  return st;
}

crkfr_status crkfr_profile_read(crkfr_ctx* c, int32_t kind, int64_t* launches, double* total_ms) {
  if (!c || kind < 0 || kind >= CRKFR_KERNEL_KINDS) return CRKFR_ERR_ARG;
  crkfr_status st = drain_profile(c, true);
  if (launches) *launches = c->prof_n[kind];
  if (total_ms) *total_ms = c->prof_ms[kind];
  return st;
}

crkfr_status crkfr_get_status(crkfr_ctx* c, void* stream) {
  if (!c) return CRKFR_ERR_ARG;
  if (c->dim == 0) return fail(c, CRKFR_ERR_STATE, "no mesh set");
  crkfr_status st = check_device(c);
  if (st != CRKFR_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned int flag = 0;
  CK(c, cudaMemcpyAsync(&flag, &c->d_state->status, sizeof(flag), cudaMemcpyDeviceToHost, s));
  CK(c, cudaMemsetAsync(&c->d_state->status, 0, sizeof(flag), s));
  CK(c, cudaStreamSynchronize(s));
  if (flag) return fail(c, CRKFR_ERR_NONPHYSICAL, "non-physical state produced");
  return CRKFR_OK;
}

}  // extern "C"
