// Ragged ensembles of independent 1D meshes (C ABI crkfr_batch_*).
//
// All instances share one system, node family and CFL safety factor; each has
// its own degree N, element count, interval and coefficient field, and its own
// time step when stepping with the CFL step.  A step of the whole ensemble is
// one kernel launch per degree class: every block takes one (instance, tile)
// pair from the class's work list and runs the same fused tile body as the
// single-mesh step, with the instance's 1/dx as a scalar, so small instances
// do not leave the GPU idle and no per-instance launch is needed.  A call of
// many steps can be captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "crkfr.h"
#include "crkfr_internal.h"
#include "tableau.h"

using namespace crkfr;

struct crkfr_batch {
  crkfr_config cfg{};
  int n_inst = 0;
  int M = 1;
  std::vector<int> deg;
  std::vector<int64_t> E, u_off, c_off, sf_off;
  std::vector<double> lo, hi;
  int64_t n_state = 0, n_coef = 0, n_sface = 0;
  HostBasis basis[kMaxNodes];
  Tables tab[kMaxNodes];
  double cfl[kMaxNodes] = {};
  bool have[kMaxNodes] = {};
  BatchInstance* d_inst = nullptr;
  WorkItem* d_work[kMaxNodes] = {};
  int64_t nwork[kMaxNodes] = {};
  double* d_snode = nullptr;
  double* d_sface = nullptr;
  double* d_swap = nullptr;
  DevState* d_states = nullptr;
  bool coef_set = false;
  int device = -1;
  int64_t launches = 0;
  std::string err;
  // graph of the last captured call
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double* g_u = nullptr;
  double g_dt = 0.0;
  int64_t g_nsteps = -1;
};

namespace {

crkfr_status bfail(crkfr_batch* b, crkfr_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define BCK(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail(b, CRKFR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__global__ void k_batch_prepare(DevState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) st[i].rate[0] = st[i].rate[1] = st[i].rate[2] = 0ull;
}

// after an odd number of steps the time sits in slot 1: move it to slot 0 so
// that every call starts from slot 0
__global__ void k_batch_finish(DevState* st, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) st[i].time[0] = st[i].time[1];
}

void free_all(crkfr_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaFree(b->d_inst);
  for (int k = 0; k < kMaxNodes; ++k) cudaFree(b->d_work[k]);
  cudaFree(b->d_snode);
  cudaFree(b->d_sface);
  cudaFree(b->d_swap);
  cudaFree(b->d_states);
}

LaunchBatch1D make(crkfr_batch* b, int N) {
  LaunchBatch1D B{};
  B.system = b->cfg.system;
  B.N = N;
  B.gll = b->cfg.nodes == CRKFR_NODES_GLL;
  B.imex = b->cfg.source != CRKFR_SRC_NONE;
  B.inst = b->d_inst;
  B.work = b->d_work[N];
  B.nwork = b->nwork[N];
  B.snode = b->d_snode;
  B.sface = b->d_sface;
  B.tab = b->tab[N];
  return B;
}

// the launches of one call: [prepare + rates], [copy], nsteps x classes, [finish]
crkfr_status record(crkfr_batch* b, double* u, double dt, int64_t nsteps, cudaStream_t s) {
  const bool cfl_mode = !(dt > 0.0);
  const int nb = (b->n_inst + 127) / 128;
  if (cfl_mode) {
    k_batch_prepare<<<nb, 128, 0, s>>>(b->d_states, b->n_inst);
    BCK(b, cudaGetLastError());
    b->launches += 1;
    for (int N = 0; N < kMaxNodes; ++N) {
      if (!b->nwork[N]) continue;
      LaunchBatch1D B = make(b, N);
      B.u_in = u;
      if (launch_rate_1d_batch(B, 0, s)) return bfail(b, CRKFR_ERR_CUDA, "batch rate kernel");
      b->launches += 1;
    }
  }
  double* bufs[2] = {u, b->d_swap};
  int cur = 0;
  if (nsteps % 2 == 1) {
    BCK(b, cudaMemcpyAsync(b->d_swap, u, sizeof(double) * b->n_state, cudaMemcpyDeviceToDevice, s));
    cur = 1;
  }
  StepCtl ctl{};
  ctl.dt_fixed = cfl_mode ? 0.0 : dt;
  ctl.t_end = std::numeric_limits<double>::infinity();
  ctl.want_rate = cfl_mode ? 1 : 0;
  for (int64_t k = 0; k < nsteps; ++k) {
    ctl.slot_read = (int)(k % 3);
    ctl.slot_write = (int)((k + 1) % 3);
    ctl.slot_reset = (int)((k + 2) % 3);
    ctl.tslot = (int)(k % 2);
    for (int N = 0; N < kMaxNodes; ++N) {
      if (!b->nwork[N]) continue;
      LaunchBatch1D B = make(b, N);
      ctl.cs_cfl = b->cfg.cfl_safety * b->cfl[N];
      B.ctl = ctl;
      B.u_in = bufs[cur];
      B.u_out = bufs[cur ^ 1];
      if (launch_step_1d_batch(B, s)) return bfail(b, CRKFR_ERR_CUDA, "batch step kernel");
      b->launches += 1;
    }
    cur ^= 1;
  }
  if (nsteps % 2 == 1) {
    k_batch_finish<<<nb, 128, 0, s>>>(b->d_states, b->n_inst);
    BCK(b, cudaGetLastError());
    b->launches += 1;
  }
  return CRKFR_OK;
}

crkfr_status ready(crkfr_batch* b) {
  if (!b) return CRKFR_ERR_ARG;
  if (!b->coef_set) return bfail(b, CRKFR_ERR_STATE, "no coefficients set");
  int d = -1;
  BCK(b, cudaGetDevice(&d));
  if (d != b->device) return bfail(b, CRKFR_ERR_STATE, "current device differs from the batch's");
  return CRKFR_OK;
}

}  // namespace

extern "C" {

crkfr_status crkfr_batch_create(crkfr_batch** out, const crkfr_config* cfg, int32_t n,
                                const int32_t* degrees, const int64_t* n_elem, const double* lo,
                                const double* hi) {
  if (!out) return CRKFR_ERR_ARG;
  *out = nullptr;
  if (!cfg || !degrees || !n_elem || !lo || !hi || n <= 0) return CRKFR_ERR_ARG;
  if (!sys_valid(cfg->system) || sys_is_2d(cfg->system)) return CRKFR_ERR_UNSUPPORTED;
  if (cfg->nodes != CRKFR_NODES_GL && cfg->nodes != CRKFR_NODES_GLL) return CRKFR_ERR_ARG;
  if (crkfr_status sst = check_source(cfg); sst != CRKFR_OK) return sst;
  const bool imex = cfg->source != CRKFR_SRC_NONE;
  if (!(cfg->cfl_safety > 0.0) || cfg->cfl_safety > 1.0) return CRKFR_ERR_ARG;
  if (sys_is_swe(cfg->system) && !(cfg->gravity > 0.0)) return CRKFR_ERR_ARG;
  const bool gll = cfg->nodes == CRKFR_NODES_GLL;
  crkfr_batch* b = new (std::nothrow) crkfr_batch();
  if (!b) return CRKFR_ERR_ALLOC;
  b->cfg = *cfg;
  b->n_inst = n;
  b->M = sys_vars(cfg->system);
  const double g = cfg->system == CRKFR_SYS_VARADV_1D ? 0.0 : cfg->gravity;
  std::vector<std::vector<WorkItem>> work(kMaxNodes);
  for (int i = 0; i < n; ++i) {
    const int N = degrees[i];
    if (N < (gll ? 1 : 0) || N > kMaxN) {
      delete b;
      return CRKFR_ERR_UNSUPPORTED;
    }
    if (n_elem[i] <= 0 || !(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i])) {
      delete b;
      return CRKFR_ERR_ARG;
    }
    if (!b->have[N]) {
      build_basis(N, gll, &b->basis[N]);
      fill_tables(b->basis[N], 1.0, 0.0, g, imex, source_coef(*cfg), &b->tab[N]);
      b->cfl[N] = cfg->cfl_number > 0.0 ? cfg->cfl_number : von_neumann_cfl(b->basis[N], imex);
      b->have[N] = true;
    }
    const int64_t nn = N + 1;
    b->deg.push_back(N);
    b->E.push_back(n_elem[i]);
    b->lo.push_back(lo[i]);
    b->hi.push_back(hi[i]);
    b->u_off.push_back(b->n_state);
    b->c_off.push_back(b->n_coef);
    b->sf_off.push_back(b->n_sface);
    b->n_state += b->M * n_elem[i] * nn;
    b->n_coef += n_elem[i] * nn;
    b->n_sface += 2 * n_elem[i];
    const int64_t tiles = (n_elem[i] + kTile1D - 1) / kTile1D;
    if (tiles > 0x7fffffff) {
      delete b;
      return CRKFR_ERR_ARG;
    }
    for (int64_t t = 0; t < tiles; ++t) work[N].push_back({(int32_t)i, (int32_t)t});
  }
  b->u_off.push_back(b->n_state);
  b->c_off.push_back(b->n_coef);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return CRKFR_ERR_CUDA;
  }
  bool ok = cudaMalloc(&b->d_inst, sizeof(BatchInstance) * n) == cudaSuccess &&
            cudaMalloc(&b->d_snode, sizeof(double) * b->n_coef) == cudaSuccess &&
            cudaMalloc(&b->d_sface, sizeof(double) * b->n_sface) == cudaSuccess &&
            cudaMalloc(&b->d_swap, sizeof(double) * b->n_state) == cudaSuccess &&
            cudaMalloc(&b->d_states, sizeof(DevState) * n) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int N = 0; ok && N < kMaxNodes; ++N) {
    b->nwork[N] = (int64_t)work[N].size();
    if (b->nwork[N]) {
      ok = cudaMalloc(&b->d_work[N], sizeof(WorkItem) * b->nwork[N]) == cudaSuccess &&
           cudaMemcpy(b->d_work[N], work[N].data(), sizeof(WorkItem) * b->nwork[N],
                      cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (ok) {
    std::vector<BatchInstance> inst(n);
    for (int i = 0; i < n; ++i) {
      inst[i].E = b->E[i];
      inst[i].u_off = b->u_off[i];
      inst[i].sn_off = b->c_off[i];
      inst[i].sf_off = b->sf_off[i];
      inst[i].xs = (double)b->E[i] / (b->hi[i] - b->lo[i]);
      inst[i].st = b->d_states + i;
    }
    ok = cudaMemcpy(b->d_inst, inst.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemset(b->d_states, 0, sizeof(DevState) * n) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    free_all(b);
    delete b;
    return CRKFR_ERR_ALLOC;
  }
  *out = b;
  return CRKFR_OK;
}

void crkfr_batch_destroy(crkfr_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_all(b);
  delete b;
}

crkfr_status crkfr_batch_layout(const crkfr_batch* b, int64_t* state_offsets,
                                int64_t* coef_offsets) {
  if (!b) return CRKFR_ERR_ARG;
  for (int i = 0; i <= b->n_inst; ++i) {
    if (state_offsets) state_offsets[i] = b->u_off[i];
    if (coef_offsets) coef_offsets[i] = b->c_off[i];
  }
  return CRKFR_OK;
}

crkfr_status crkfr_batch_set_coefficients(crkfr_batch* b, const double* c, void* stream) {
  if (!b || !c) return CRKFR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < b->n_inst; ++i) {
    const int N = b->deg[i];
    if (launch_coef_1d(b->cfg.system, N, b->E[i], c + b->c_off[i], b->d_snode + b->c_off[i],
                       b->d_sface + b->sf_off[i], b->tab[N], s))
      return bfail(b, CRKFR_ERR_CUDA, "coefficient kernel");
    b->launches += 1;
  }
  b->coef_set = true;
  return CRKFR_OK;
}

crkfr_status crkfr_batch_step(crkfr_batch* b, double* u, double dt, int64_t nsteps,
                              int32_t use_graph, void* stream) {
  crkfr_status st = ready(b);
  if (st != CRKFR_OK) return st;
  if (!u || nsteps < 0) return bfail(b, CRKFR_ERR_ARG, "bad argument");
  if (!std::isfinite(dt) && dt > 0.0) return bfail(b, CRKFR_ERR_ARG, "dt must be finite");
  if (nsteps == 0) return CRKFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return record(b, u, dt, nsteps, s);
  const bool same = b->gexec && b->g_u == u && b->g_nsteps == nsteps &&
                    ((dt > 0.0) == (b->g_dt > 0.0)) && (!(dt > 0.0) || dt == b->g_dt);
  if (!same) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    const int64_t before = b->launches;
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    st = record(b, u, dt, nsteps, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != CRKFR_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return bfail(b, CRKFR_ERR_CUDA, "graph capture failed");
    b->graph = g;
    BCK(b, cudaGraphInstantiate(&b->gexec, g, 0));
    b->g_u = u;
    b->g_dt = dt;
    b->g_nsteps = nsteps;
    b->launches = before;   // counted when the graph runs
  }
  const int64_t per_call = [&] {
    int64_t k = 0, classes = 0;
    for (int N = 0; N < kMaxNodes; ++N) classes += b->nwork[N] ? 1 : 0;
    k = nsteps * classes + (nsteps % 2 == 1 ? 1 : 0);
    if (!(dt > 0.0)) k += 1 + classes;
    return k;
  }();
  BCK(b, cudaGraphLaunch(b->gexec, s));
  b->launches += per_call;
  return CRKFR_OK;
}

crkfr_status crkfr_batch_get_times(crkfr_batch* b, double* t_host, void* stream) {
  if (!b || !t_host) return CRKFR_ERR_ARG;
  std::vector<DevState> h(b->n_inst);
  cudaStream_t s = (cudaStream_t)stream;
  BCK(b, cudaMemcpyAsync(h.data(), b->d_states, sizeof(DevState) * b->n_inst,
                         cudaMemcpyDeviceToHost, s));
  BCK(b, cudaStreamSynchronize(s));
  for (int i = 0; i < b->n_inst; ++i) t_host[i] = h[i].time[0];
  return CRKFR_OK;
}

crkfr_status crkfr_batch_get_status(crkfr_batch* b, void* stream) {
  if (!b) return CRKFR_ERR_ARG;
  std::vector<DevState> h(b->n_inst);
  cudaStream_t s = (cudaStream_t)stream;
  BCK(b, cudaMemcpyAsync(h.data(), b->d_states, sizeof(DevState) * b->n_inst,
                         cudaMemcpyDeviceToHost, s));
  BCK(b, cudaStreamSynchronize(s));
  bool bad = false;
  for (auto& x : h) bad |= x.status != 0;
  if (bad) {
    for (int i = 0; i < b->n_inst; ++i)
      BCK(b, cudaMemsetAsync(&b->d_states[i].status, 0, sizeof(unsigned int), s));
    BCK(b, cudaStreamSynchronize(s));
    return bfail(b, CRKFR_ERR_NONPHYSICAL, "non-physical state produced");
  }
  return CRKFR_OK;
}

int64_t crkfr_batch_launch_count(const crkfr_batch* b) { return b ? b->launches : 0; }

const char* crkfr_batch_last_error(const crkfr_batch* b) { return b ? b->err.c_str() : "null"; }

}  // extern "C"
