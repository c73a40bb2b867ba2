// Objective evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at evaluation time: a real-time control loop that
// must not allocate after start-up (cudaMalloc can synchronize the device and its latency
// is unbounded), or a host framework whose own allocator owns all device memory and
// forbids allocations by libraries.  For them, ocp_eval_obj_noalloc evaluates the
// objective without a handle and without any allocation: the per-tile partial sums and the
// completion ticket of the deterministic reduction live in one file-scope device array.
//
// That array exists once per device that loads this library and stays allocated until the
// process exits.  Every call on a device shares it, so calls that overlap on the GPU race
// (issue them on one stream, or wait between them).  The array keeps the last call's
// contents; the ticket that must start at zero is cleared by each call before its launch.
// The array's device address is looked up once per device and cached for the life of the
// process; it is stale after cudaDeviceReset, so the entry point is not for processes that
// reset a device they used it on.
#include <cstring>
#include <mutex>

#include "ocp_internal.h"

using namespace ocpg;

// Maximum number of reduction tiles: 65536 tiles of 31 (heat) to 255 (Van der Pol) nodes.
// The array holds the ticket in its first 256 bytes and one partial sum per tile after it.
#define OCP_NOALLOC_MAX_TILES 65536
static __device__ __align__(256) double g_noalloc_scratch[32 + OCP_NOALLOC_MAX_TILES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};
}  // namespace

extern "C" ocp_status ocp_eval_obj_noalloc(const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N,
                                           double T, const double* x, double* f, void* stream) {
  OCP_RANGE();
  if (!x || !f) return set_err(nullptr, OCP_EINVAL, "x and f are required");
  if (((uintptr_t)x & 7u) || ((uintptr_t)f & 7u)) return set_err(nullptr, OCP_EINVAL, "x or f is not 8-byte aligned");
  ocp prob;  // host-side description only; no device allocation
  ocp_status st = init_host(&prob, dyn, cost, nx, nu, N, T);
  if (st != OCP_OK) return st;
  if (prob.model == OCP_MODEL_GODDARD)
    return set_err(nullptr, OCP_EMODEL, "ocp_eval_obj_noalloc: the Goddard objective is a terminal cost set on a handle");
  const int64_t ntiles = objective_tiles(prob.model, N + 1);
  if (ntiles < 1 || ntiles > OCP_NOALLOC_MAX_TILES)
    return set_err(nullptr, OCP_EDIM,
                   "ocp_eval_obj_noalloc: N too large for the static scratch (at most 65536 reduction tiles; "
                   "use eval_obj with a handle)");
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_err(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_err(nullptr, OCP_EINVAL, "device index out of range");
  double* base = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
        return cuda_err(nullptr, e, "cudaGetSymbolAddress(static scratch)");
      g_scratch_ptr[dev] = (double*)p;
    }
    base = g_scratch_ptr[dev];
  }
  if ((e = cudaDeviceGetAttribute(&prob.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_err(nullptr, e, "cudaDeviceGetAttribute");
  prob.device = dev;
  prob.d_counter = (unsigned*)base;
  prob.d_partials = base + 32;
  prob.max_partials = OCP_NOALLOC_MAX_TILES;
  if ((e = cudaMemsetAsync(prob.d_counter, 0, sizeof(unsigned), (cudaStream_t)stream)) != cudaSuccess)
    return cuda_err(nullptr, e, "cudaMemsetAsync(ticket)");
  EvalCall c;
  c.B = 0;
  c.E = N + 1;
  c.x = x;
  c.f = f;
  st = dispatch_eval(&prob, O_F, c, stream);
  if (st != OCP_OK) return set_err(nullptr, st, prob.err);
  return OCP_OK;
}
