// crkfr_step_1d_noalloc: the fused 1D step for callers that cannot allocate
// device memory.  Every buffer the step needs beyond the caller's input and
// output (the static coefficient terms, the second state of the ping-pong,
// the device stepping state) lives in one file-scope __device__ array of
// fixed size, so the call performs no cudaMalloc/cudaFree.  It launches the
// same kernels as crkfr_step on a 1D context.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "crkfr.h"
#include "crkfr_internal.h"

using namespace crkfr;

namespace {

// 2^21 doubles = 16 MiB per device that loads the library, held until exit.
constexpr int64_t kNoAllocDoubles = (int64_t)1 << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name
// g_noalloc_scratch in host code is only a host-side stand-in, so the
// address is looked up once per device with that device current.
cudaError_t scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = (double*)p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

extern "C" crkfr_status crkfr_step_1d_noalloc(const crkfr_config* cfg, int64_t n_elem, double lo,
                                              double hi, const double* c_dev,
                                              const double* u_in_dev, double* u_out_dev,
                                              double dt, int64_t nsteps, void* stream) {
  clear_global_error();
  if (!cfg || !c_dev || !u_in_dev || !u_out_dev) return CRKFR_ERR_ARG;
  if (!sys_valid(cfg->system) || sys_is_2d(cfg->system)) return CRKFR_ERR_UNSUPPORTED;
  if (cfg->nodes < CRKFR_NODES_GL || cfg->nodes > CRKFR_NODES_GLL) return CRKFR_ERR_ARG;
  if (crkfr_status sst = check_source(cfg); sst != CRKFR_OK) return sst;
  const bool imex = cfg->source != CRKFR_SRC_NONE;
  const bool gll = cfg->nodes == CRKFR_NODES_GLL;
  if (cfg->degree < (gll ? 1 : 0) || cfg->degree > kMaxN) return CRKFR_ERR_UNSUPPORTED;
  if (crkfr_status so = check_options(cfg, cfg->degree); so != CRKFR_OK) return so;
  if (!(cfg->cfl_safety > 0.0) || cfg->cfl_safety > 1.0) return CRKFR_ERR_ARG;
  if (sys_is_swe(cfg->system) && !(cfg->gravity > 0.0)) return CRKFR_ERR_ARG;
  if (n_elem <= 0 || nsteps < 0 || !(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
    return CRKFR_ERR_ARG;
  if (std::isnan(dt) || (std::isinf(dt) && dt > 0.0)) return CRKFR_ERR_ARG;

  HostBasis b;
  if (!build_basis(cfg->degree, gll, &b)) return CRKFR_ERR_UNSUPPORTED;
  const int n = b.n;
  const int M = sys_vars(cfg->system);
  const int64_t E = n_elem;
  // scratch layout (in doubles): snode [E n] | sface [2E] | state [M E n] | DevState
  const int64_t o_sface = round_up(E * n, 32);
  const int64_t o_state = o_sface + round_up(2 * E, 32);
  const int64_t o_dev = o_state + round_up((int64_t)M * E * n, 32);
  const int64_t need = o_dev + round_up((int64_t)((sizeof(DevState) + 7) / 8), 32);
  if (need > kNoAllocDoubles) return CRKFR_ERR_ARG;  // mesh too large for the static scratch

  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return CRKFR_ERR_CUDA;
  double* snode = scratch;
  double* sface = scratch + o_sface;
  double* state = scratch + o_state;
  DevState* st = reinterpret_cast<DevState*>(scratch + o_dev);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t state_bytes = sizeof(double) * (size_t)M * E * n;
  {
    const char *a = (const char*)u_in_dev, *o = (const char*)u_out_dev;
    if (a != o && a < o + state_bytes && o < a + state_bytes) return CRKFR_ERR_ARG;
  }

  Tables T;   // reference element; 1/dx goes with the launch
  fill_tables(b, 1.0, 0.0, cfg->system == CRKFR_SYS_VARADV_1D ? 0.0 : cfg->gravity, imex,
              source_coef(*cfg), &T);
  const double xs = (double)E / (hi - lo);

  // the array keeps the previous call's contents: reset the stepping state
  if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return CRKFR_ERR_CUDA;
  if (launch_coef_1d(cfg->system, cfg->degree, E, c_dev, snode, sface, T, s)) return CRKFR_ERR_CUDA;
  if (nsteps == 0) {
    if (u_out_dev != u_in_dev &&
        cudaMemcpyAsync(u_out_dev, u_in_dev, state_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return CRKFR_ERR_CUDA;
    return CRKFR_OK;
  }

  const bool cfl_mode = !(dt > 0.0);
  double cfl = cfg->cfl_number;
  if (cfl_mode && !(cfl > 0.0)) cfl = von_neumann_cfl(b, imex);

  Launch1D L{};
  L.system = cfg->system;
  L.N = cfg->degree;
  L.gll = gll;
  L.imex = imex;
  L.E = E;
  L.snode = snode;
  L.sface = sface;
  L.st = st;
  L.tab = T;
  L.xs = xs;
  // ping-pong between the caller's output and the scratch state, ending in
  // the output; an input that is also the output is first moved to scratch
  // (an odd count in place starts from a copy in scratch: the first step may
  // not write the buffer it reads)
  const double* src = u_in_dev;
  double* bufs[2] = {u_out_dev, state};
  int cur_dst = (nsteps % 2 == 1) ? 0 : 1;
  if (u_in_dev == u_out_dev && nsteps % 2 == 1) {
    if (cudaMemcpyAsync(state, u_in_dev, state_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return CRKFR_ERR_CUDA;
    src = state;
  }
  if (cfl_mode) {
    L.u_in = src;
    if (launch_rate_1d(L, 0, s)) return CRKFR_ERR_CUDA;
  }
  StepCtl ctl{};
  ctl.dt_fixed = cfl_mode ? 0.0 : dt;
  ctl.cs_cfl = cfg->cfl_safety * cfl;
  ctl.t_end = INFINITY;
  ctl.want_rate = cfl_mode ? 1 : 0;
  for (int64_t k = 0; k < nsteps; ++k) {
    ctl.slot_read = (int)(k % 3);
    ctl.slot_write = (int)((k + 1) % 3);
    ctl.slot_reset = (int)((k + 2) % 3);
    ctl.tslot = (int)(k % 2);
    L.ctl = ctl;
    L.u_in = src;
    L.u_out = bufs[cur_dst];
    if (launch_step_1d(L, s)) return CRKFR_ERR_CUDA;
    src = bufs[cur_dst];
    cur_dst ^= 1;
  }
  return CRKFR_OK;
}
