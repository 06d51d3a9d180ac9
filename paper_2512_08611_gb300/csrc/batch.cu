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
//
// Launch shape (tuned per ensemble by crkfr_batch_autotune, which times the
// candidates as captured graphs on a scratch copy of the state): the number
// of tiles each block runs in turn (tiles per block), the order of the work
// lists (instance order, or the tiles of the largest instances first so that
// the last wave is made of small tiles), and whether the degree classes,
// which share no data, run as one serial chain of launches or as concurrent
// branches (one stream each, forked and joined around the K steps).
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
  // launch shape (crkfr_batch_set_tuning / crkfr_batch_autotune)
  std::vector<WorkItem> work_h[kMaxNodes];   // work lists in instance order
  int tpb = 1;            // tiles per block
  int order = 0;          // 0 instance order, 1 largest instances first
  int parallel = 0;       // 1: degree classes on concurrent branches
  double tune_ms = 0.0;   // time per step of the chosen shape (autotune), 0 if not tuned
  cudaStream_t side[kMaxNodes] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxNodes] = {};
  // graph of the last captured call
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double* g_u = nullptr;
  double g_dt = 0.0;
  int64_t g_nsteps = -1;
  // kernel timing of calls without a graph (crkfr_batch_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;   // pairs (start, end) of the recorded launches
  int64_t prof_n = 0;
  double prof_ms = 0.0;
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

void drop_graph(crkfr_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->g_u = nullptr;
  b->g_nsteps = -1;
}

void free_all(crkfr_batch* b) {
  drop_graph(b);
  for (auto e : b->prof_ev) cudaEventDestroy(e);
  b->prof_ev.clear();
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int k = 0; k < kMaxNodes; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
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
  B.grid = (b->nwork[N] + b->tpb - 1) / b->tpb;
  B.snode = b->d_snode;
  B.sface = b->d_sface;
  B.tab = b->tab[N];
  return B;
}

// rate launch of one degree class
crkfr_status class_rates(crkfr_batch* b, int N, double* u, cudaStream_t s) {
  LaunchBatch1D B = make(b, N);
  B.u_in = u;
  if (launch_rate_1d_batch(B, 0, s)) return bfail(b, CRKFR_ERR_CUDA, "batch rate kernel");
  b->launches += 1;
  return CRKFR_OK;
}

// step k of one degree class (timed with an event pair when profiling a
// call that is not captured)
crkfr_status class_step(crkfr_batch* b, int N, StepCtl ctl, int64_t k, double* const* bufs,
                        int cur, cudaStream_t s, bool timed) {
  ctl.slot_read = (int)(k % 3);
  ctl.slot_write = (int)((k + 1) % 3);
  ctl.slot_reset = (int)((k + 2) % 3);
  ctl.tslot = (int)(k % 2);
  ctl.cs_cfl = b->cfg.cfl_safety * b->cfl[N];
  LaunchBatch1D B = make(b, N);
  B.ctl = ctl;
  B.u_in = bufs[cur];
  B.u_out = bufs[cur ^ 1];
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (timed) {
    for (auto& e : ev) BCK(b, cudaEventCreate(&e));
    b->prof_ev.push_back(ev[0]);
    b->prof_ev.push_back(ev[1]);
    BCK(b, cudaEventRecord(ev[0], s));
  }
  if (launch_step_1d_batch(B, s)) return bfail(b, CRKFR_ERR_CUDA, "batch step kernel");
  if (timed) BCK(b, cudaEventRecord(ev[1], s));
  b->launches += 1;
  return CRKFR_OK;
}

// sums the recorded kernel times (synchronises on the events) and frees them
crkfr_status drain_profile(crkfr_batch* b) {
  crkfr_status st = CRKFR_OK;
  for (size_t i = 0; i + 1 < b->prof_ev.size(); i += 2) {
    float ms = 0.0f;
    if (st == CRKFR_OK) {
      cudaError_t e = cudaEventSynchronize(b->prof_ev[i + 1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->prof_ev[i], b->prof_ev[i + 1]);
      if (e != cudaSuccess) st = bfail(b, CRKFR_ERR_CUDA, "profile events");
    }
    b->prof_n += 1;
    b->prof_ms += ms;
    cudaEventDestroy(b->prof_ev[i]);
    cudaEventDestroy(b->prof_ev[i + 1]);
  }
  b->prof_ev.clear();
  return st;
}

// the launches of one call: [prepare], [copy], per class [rates] and nsteps
// steps (interleaved by step, or one concurrent branch per class), [finish]
crkfr_status record(crkfr_batch* b, double* u, double dt, int64_t nsteps, cudaStream_t s,
                    bool timed = false) {
  const bool cfl_mode = !(dt > 0.0);
  const int nb = (b->n_inst + 127) / 128;
  if (cfl_mode) {
    k_batch_prepare<<<nb, 128, 0, s>>>(b->d_states, b->n_inst);
    BCK(b, cudaGetLastError());
    b->launches += 1;
  }
  double* bufs[2] = {u, b->d_swap};
  int cur0 = 0;
  if (nsteps % 2 == 1) {
    BCK(b, cudaMemcpyAsync(b->d_swap, u, sizeof(double) * b->n_state, cudaMemcpyDeviceToDevice, s));
    cur0 = 1;
  }
  StepCtl ctl{};
  ctl.dt_fixed = cfl_mode ? 0.0 : dt;
  ctl.t_end = std::numeric_limits<double>::infinity();
  ctl.want_rate = cfl_mode ? 1 : 0;
  if (b->parallel) {
    BCK(b, cudaEventRecord(b->ev_fork, s));
    for (int N = 0; N < kMaxNodes; ++N) {
      if (!b->nwork[N]) continue;
      cudaStream_t q = b->side[N];
      BCK(b, cudaStreamWaitEvent(q, b->ev_fork, 0));
      if (cfl_mode) {
        crkfr_status st = class_rates(b, N, u, q);
        if (st != CRKFR_OK) return st;
      }
      int cur = cur0;
      for (int64_t k = 0; k < nsteps; ++k) {
        crkfr_status st = class_step(b, N, ctl, k, bufs, cur, q, timed);
        if (st != CRKFR_OK) return st;
        cur ^= 1;
      }
      BCK(b, cudaEventRecord(b->ev_join[N], q));
      BCK(b, cudaStreamWaitEvent(s, b->ev_join[N], 0));
    }
  } else {
    if (cfl_mode) {
      for (int N = 0; N < kMaxNodes; ++N) {
        if (!b->nwork[N]) continue;
        crkfr_status st = class_rates(b, N, u, s);
        if (st != CRKFR_OK) return st;
      }
    }
    int cur = cur0;
    for (int64_t k = 0; k < nsteps; ++k) {
      for (int N = 0; N < kMaxNodes; ++N) {
        if (!b->nwork[N]) continue;
        crkfr_status st = class_step(b, N, ctl, k, bufs, cur, s, timed);
        if (st != CRKFR_OK) return st;
      }
      cur ^= 1;
    }
  }
  if (nsteps % 2 == 1) {
    k_batch_finish<<<nb, 128, 0, s>>>(b->d_states, b->n_inst);
    BCK(b, cudaGetLastError());
    b->launches += 1;
  }
  return CRKFR_OK;
}

// capture one call into a graph (on the batch's capture stream)
crkfr_status capture(crkfr_batch* b, double* u, double dt, int64_t nsteps, cudaGraph_t* graph,
                     cudaGraphExec_t* exec) {
  *graph = nullptr;
  *exec = nullptr;
  BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  crkfr_status st = record(b, u, dt, nsteps, b->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != CRKFR_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return bfail(b, CRKFR_ERR_CUDA, "graph capture failed");
  if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return bfail(b, CRKFR_ERR_CUDA, "graph instantiation failed");
  }
  *graph = g;
  return CRKFR_OK;
}

// upload the work lists in the chosen order
crkfr_status apply_order(crkfr_batch* b) {
  for (int N = 0; N < kMaxNodes; ++N) {
    if (!b->nwork[N]) continue;
    std::vector<WorkItem> w = b->work_h[N];
    if (b->order == 1)
      std::stable_sort(w.begin(), w.end(), [&](const WorkItem& x, const WorkItem& y) {
        return b->E[x.inst] > b->E[y.inst];
      });
    BCK(b, cudaMemcpy(b->d_work[N], w.data(), sizeof(WorkItem) * w.size(),
                      cudaMemcpyHostToDevice));
  }
  return CRKFR_OK;
}

int64_t launches_per_call(const crkfr_batch* b, double dt, int64_t nsteps) {
  int64_t classes = 0;
  for (int N = 0; N < kMaxNodes; ++N) classes += b->nwork[N] ? 1 : 0;
  int64_t k = nsteps * classes + (nsteps % 2 == 1 ? 1 : 0);
  if (!(dt > 0.0)) k += 1 + classes;
  return k;
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
  clear_global_error();
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
    if (crkfr_status so = check_options(cfg, N); so != CRKFR_OK) {
      delete b;
      return so;
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
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int N = 0; ok && N < kMaxNodes; ++N)
    ok = cudaStreamCreateWithFlags(&b->side[N], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join[N], cudaEventDisableTiming) == cudaSuccess;
  for (int N = 0; ok && N < kMaxNodes; ++N) {
    b->work_h[N] = work[N];
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
  if (std::isnan(dt) || (std::isinf(dt) && dt > 0.0))
    return bfail(b, CRKFR_ERR_ARG, "dt must be finite (or <= 0 for the CFL step)");
  if (nsteps == 0) return CRKFR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return record(b, u, dt, nsteps, s, b->prof);
  const bool same = b->gexec && b->g_u == u && b->g_nsteps == nsteps &&
                    ((dt > 0.0) == (b->g_dt > 0.0)) && (!(dt > 0.0) || dt == b->g_dt);
  if (!same) {
    drop_graph(b);
    const int64_t before = b->launches;
    st = capture(b, u, dt, nsteps, &b->graph, &b->gexec);
    b->launches = before;   // counted when the graph runs
    if (st != CRKFR_OK) return st;
    b->g_u = u;
    b->g_dt = dt;
    b->g_nsteps = nsteps;
  }
  BCK(b, cudaGraphLaunch(b->gexec, s));
  b->launches += launches_per_call(b, dt, nsteps);
  return CRKFR_OK;
}

crkfr_status crkfr_batch_set_tuning(crkfr_batch* b, int32_t tiles_per_block, int32_t order,
                                    int32_t parallel) {
  if (!b) return CRKFR_ERR_ARG;
  if (tiles_per_block < 1 || tiles_per_block > 1024 || order < 0 || order > 1 || parallel < 0 ||
      parallel > 1)
    return bfail(b, CRKFR_ERR_ARG, "bad tuning");
  b->tpb = tiles_per_block;
  b->order = order;
  b->parallel = parallel;
  b->tune_ms = 0.0;
  drop_graph(b);
  return apply_order(b);
}

crkfr_status crkfr_batch_get_tuning(const crkfr_batch* b, int32_t* tiles_per_block,
                                    int32_t* order, int32_t* parallel, double* ms_per_step) {
  if (!b) return CRKFR_ERR_ARG;
  if (tiles_per_block) *tiles_per_block = b->tpb;
  if (order) *order = b->order;
  if (parallel) *parallel = b->parallel;
  if (ms_per_step) *ms_per_step = b->tune_ms;
  return CRKFR_OK;
}

crkfr_status crkfr_batch_autotune(crkfr_batch* b, const double* u, int32_t steps, void* stream) {
  crkfr_status st = ready(b);
  if (st != CRKFR_OK) return st;
  if (!u || steps < 1) return bfail(b, CRKFR_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  // scratch state and a copy of the stepping states, restored afterwards
  double* scratch = nullptr;
  DevState* saved = nullptr;
  if (cudaMalloc(&scratch, sizeof(double) * b->n_state) != cudaSuccess ||
      cudaMalloc(&saved, sizeof(DevState) * b->n_inst) != cudaSuccess) {
    cudaFree(scratch);
    cudaGetLastError();
    return bfail(b, CRKFR_ERR_ALLOC, "device allocation failed");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  BCK(b, cudaMemcpyAsync(saved, b->d_states, sizeof(DevState) * b->n_inst,
                         cudaMemcpyDeviceToDevice, s));
  const int64_t launches0 = b->launches;
  const int tpbs[] = {1, 2, 4, 8};
  double best = std::numeric_limits<double>::infinity();
  int bt = 1, bo = 0, bp = 0;
  st = CRKFR_OK;
  for (int par = 0; par <= 1 && st == CRKFR_OK; ++par)
    for (int ord = 0; ord <= 1 && st == CRKFR_OK; ++ord)
      for (int t : tpbs) {
        b->tpb = t;
        b->order = ord;
        b->parallel = par;
        st = apply_order(b);
        if (st != CRKFR_OK) break;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        st = capture(b, scratch, 0.0, steps, &g, &x);
        if (st != CRKFR_OK) break;
        float ms = 0.0f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {   // warm, then timed
          ok = cudaMemcpyAsync(scratch, u, sizeof(double) * b->n_state, cudaMemcpyDeviceToDevice,
                               s) == cudaSuccess &&
               cudaMemcpyAsync(b->d_states, saved, sizeof(DevState) * b->n_inst,
                               cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
               cudaEventRecord(e0, s) == cudaSuccess && cudaGraphLaunch(x, s) == cudaSuccess &&
               cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
               cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        }
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        if (!ok) {
          cudaGetLastError();
          st = bfail(b, CRKFR_ERR_CUDA, "autotune trial failed");
          break;
        }
        if (ms / steps < best) {
          best = ms / steps;
          bt = t;
          bo = ord;
          bp = par;
        }
      }
  cudaMemcpyAsync(b->d_states, saved, sizeof(DevState) * b->n_inst, cudaMemcpyDeviceToDevice, s);
  cudaStreamSynchronize(s);
  cudaFree(scratch);
  cudaFree(saved);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->launches = launches0;
  if (st != CRKFR_OK) return st;
  st = crkfr_batch_set_tuning(b, bt, bo, bp);
  b->tune_ms = best;
  return st;
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

crkfr_status crkfr_batch_profile_enable(crkfr_batch* b, int32_t enable) {
  if (!b) return CRKFR_ERR_ARG;
  crkfr_status st = drain_profile(b);
  b->prof_n = 0;
  b->prof_ms = 0.0;
  b->prof = enable != 0;
  return st;
}

crkfr_status crkfr_batch_profile_read(crkfr_batch* b, int64_t* launches, double* total_ms) {
  if (!b) return CRKFR_ERR_ARG;
  crkfr_status st = drain_profile(b);
  if (launches) *launches = b->prof_n;
  if (total_ms) *total_ms = b->prof_ms;
  return st;
}

const char* crkfr_batch_last_error(const crkfr_batch* b) { return b ? b->err.c_str() : "null"; }

}  // extern "C"
