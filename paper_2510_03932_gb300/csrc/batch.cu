// Batched evaluation: many problems of one model (different horizons, cost weights and
// boundary values) evaluated by ONE persistent launch over the concatenation of their tiles.
//
// Layout: instance i's variables, constraints, gradient, Jacobian and Hessian values start at
// the prefix offsets xoff[i], coff[i], xoff[i], joff[i], hoff[i] of the concatenated arrays
// and are laid out exactly as for its own handle, so every instance slice is bit-identical to
// the plain evaluator's output (same per-node arithmetic; only the objective's summation
// tiles may differ when the tile size differs).
//
// Work decomposition: instance i is cut into tiles of NPT*TILE nodes (owning NPT*TILE-1); the
// tiles of all instances form one index space.  A persistent grid of (CTAs per SM) x (SMs)
// CTAs takes tiles from an atomic work counter (dynamic balance; no CTA ever waits for
// another); a CTA maps its tile to the instance by binary search over the tile prefix sums,
// copies that instance's argument block into shared memory, and runs the same tile body as
// the plain kernel.  Each tile's objective term goes to its own slot; the CTA completing an
// instance's last tile (per-instance completion counter) sums that instance's slots in tile
// order, so the objective does not depend on the scheduling.  Counters are reset in-kernel.
//
// Tuning: threads per CTA (64, 128, 256), nodes per thread (1, 2: nodes per warp 32 or 64) and
// CTAs per SM are chosen by ocp_batch_autotune, which times every candidate on the caller's
// data.  ocp_batch_graph_capture records one launch in a CUDA graph for cheap replay.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "model_cartpole.cuh"
#include "model_dint.cuh"
#include "model_quad.cuh"
#include "model_vdp.cuh"
#include "node_kernels.cuh"
#include "ocp_internal.h"

using namespace ocpg;

namespace ocpg {

template <class M>
struct BatchArgs {
  const NodeArgs<M>* inst;
  const int64_t* tileoff;  // count + 1
  const int64_t* xoff;
  const int64_t* coff;
  const int64_t* joff;
  const int64_t* hoff;
  const double* x;
  const double* y;
  double *f, *c, *g, *jv, *hv;
  double* partials;
  unsigned* counter;             // CTAs that finished (reset by the last one)
  unsigned long long* work;      // next tile to take (reset by the last CTA)
  unsigned* icount;              // per instance: tiles completed (reset by the finishing CTA)
  double sigma;
  int64_t ntiles;
  int count;
};

template <class M, int TILE, int NPT>
__global__ void __launch_bounds__(TILE) k_batch_eval(const __grid_constant__ BatchArgs<M> b) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double sEdge[2 * (TILE / 32 + 1) * M::NX];
  __shared__ NodeArgs<M> sa;
  __shared__ long long s_tile;
  __shared__ int s_inst, s_fin;
  static_assert(sizeof(NodeArgs<M>) % 8 == 0, "argument block is copied in 8-byte words");
  for (;;) {
    // dynamic tile scheduling: results do not depend on which CTA takes which tile
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(b.work, 1ull);
    __syncthreads();
    const int64_t gt = s_tile;
    if (gt >= b.ntiles) break;
    if (threadIdx.x == 0) {
      int lo = 0, hi = b.count - 1;  // last instance whose first tile is <= gt
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(b.tileoff + mid) <= gt) lo = mid; else hi = mid - 1;
      }
      s_inst = lo;
    }
    __syncthreads();
    const int i = s_inst;
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(b.inst + i);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sa);
      for (int w = threadIdx.x; w < (int)(sizeof(NodeArgs<M>) / 8); w += TILE) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      sa.x = b.x + __ldg(b.xoff + i);
      sa.y = b.y ? b.y + __ldg(b.coff + i) : nullptr;
      sa.f = b.f;
      sa.c = b.c ? b.c + __ldg(b.coff + i) : nullptr;
      sa.g = b.g ? b.g + __ldg(b.xoff + i) : nullptr;
      sa.jv = b.jv ? b.jv + __ldg(b.joff + i) : nullptr;
      sa.hv = b.hv ? b.hv + __ldg(b.hoff + i) : nullptr;
      for (int v = 0; v < M::NZ; ++v) {  // the argument blocks hold sigma = 1 coefficients
        sa.cq_in[v] *= b.sigma;
        sa.cq_end[v] *= b.sigma;
      }
    }
    __syncthreads();
    const ModelConst K = sa.K;
    const int64_t t0 = __ldg(b.tileoff + i), t1 = __ldg(b.tileoff + i + 1);
    node_eval_tile<M, TILE, NPT, O_ALL>(sa, K, gt - t0, sm, sEdge, b.partials + gt);
    if (b.f) {
      // the CTA that completes an instance's last tile sums its tile terms in tile order
      if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(b.icount + i, 1u);
        s_fin = (done == (unsigned)(t1 - t0 - 1));
      }
      __syncthreads();
      if (s_fin) {
        __threadfence();
        double s = 0.0;
        for (int64_t t = t0 + threadIdx.x; t < t1; t += TILE) s = s + __ldcg(b.partials + t);
        s = cta_sum<TILE>(s, sm);
        if (threadIdx.x == 0) {
          b.f[i] = 0.5 * s;
          b.icount[i] = 0u;
        }
      }
      __syncthreads();
    }
  }
  // the last CTA to leave resets the work counter for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned left = atomicAdd(b.counter, 1u);
    if (left == gridDim.x - 1) {
      *b.work = 0ull;
      *b.counter = 0u;
      __threadfence();
    }
  }
}

struct BatchConfig {
  int threads, npt;
};
static const BatchConfig kConfigs[] = {{64, 1}, {128, 1}, {256, 1}, {64, 2}, {128, 2}, {256, 2}};

// Largest CTA (threads x nodes per thread) of a model's batched kernel: the tile's staged
// Jacobian rows must fit the shared memory (the quadrotor's 68 entries per node: 128 nodes).
template <class M>
constexpr int batch_max_nodes() { return jrow_total<M>() > 32 ? 128 : 512; }

template <class M, int TILE, int NPT>
static const void* batch_kernel() {
  if constexpr (TILE * NPT <= batch_max_nodes<M>()) return (const void*)k_batch_eval<M, TILE, NPT>;
  else return nullptr;
}

template <class M>
static const void* kernel_for(int threads, int npt) {
  if (npt == 1) {
    if (threads == 64) return batch_kernel<M, 64, 1>();
    if (threads == 128) return batch_kernel<M, 128, 1>();
    if (threads == 256) return batch_kernel<M, 256, 1>();
  } else {
    if (threads == 64) return batch_kernel<M, 64, 2>();
    if (threads == 128) return batch_kernel<M, 128, 2>();
    if (threads == 256) return batch_kernel<M, 256, 2>();
  }
  return nullptr;
}

template <class M>
static size_t smem_bytes(int threads, int npt) {
  return sizeof(double) * ((size_t)jrow_total<M>() * (npt * threads - 1) + threads);
}

}  // namespace ocpg

struct ocp_batch_impl {
  int model = 0, count = 0, device = 0, num_sms = 0;
  std::vector<ocp*> items;
  std::vector<int64_t> xoff, coff, joff, hoff, tileoff;
  int threads = 128, npt = 1, ctas_per_sm = 0;
  int64_t ntiles = 0;
  void* d_inst = nullptr;
  int64_t *d_tileoff = nullptr, *d_xoff = nullptr, *d_coff = nullptr, *d_joff = nullptr, *d_hoff = nullptr;
  double* d_partials = nullptr;
  int64_t partials_cap = 0;
  unsigned* d_counter = nullptr;
  cudaGraphExec_t graph = nullptr;
  // set when the tile offsets failed to reach the device after a configuration change: the
  // device tables then disagree with the host's and every evaluation refuses the batch until
  // a configuration is set successfully
  bool unusable = false;
  std::string err;
};

struct ocp_batch : ocp_batch_impl {};

// Autotuning cache (OCP_AUTOTUNE_CACHE = path of a text file): one line per tuned batch shape,
// "key<TAB>threads npt ctas_per_sm ms", the key naming the model, the instance count, the total
// and the largest horizon, the requested outputs and the GPU (SM count, compute capability).
// A batch of a shape already in the file takes the stored configuration without timing; the
// last line of a key wins.  Lines that do not parse are ignored.
static std::mutex g_tune_mu;

static std::string tune_key(const ocp_batch* b, unsigned outs) {
  int64_t nodes = 0, maxn = 0;
  for (const ocp* h : b->items) { nodes += h->N + 1; maxn = std::max<int64_t>(maxn, h->N + 1); }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, b->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, b->device);
  char buf[256];
  std::snprintf(buf, sizeof(buf), "model=%d count=%d nodes=%lld maxnodes=%lld outputs=%u sms=%d cc=%d.%d", b->model,
                b->count, (long long)nodes, (long long)maxn, outs, b->num_sms, major, minor);
  return buf;
}

static bool tune_lookup(const char* path, const std::string& key, int& threads, int& npt, int& ctas, float& ms) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  FILE* fh = std::fopen(path, "r");
  if (!fh) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof(line), fh)) {
    char* tab = std::strchr(line, '\t');
    if (!tab || std::string(line, tab - line) != key) continue;
    int t = 0, n = 0, c = 0;
    float m = 0.f;
    if (std::sscanf(tab + 1, "%d %d %d %f", &t, &n, &c, &m) == 4 && (t == 64 || t == 128 || t == 256) &&
        (n == 1 || n == 2) && c >= 0) {
      threads = t; npt = n; ctas = c; ms = m; found = true;
    }
  }
  std::fclose(fh);
  return found;
}

static void tune_store(const char* path, const std::string& key, int threads, int npt, int ctas, float ms) {
  std::lock_guard<std::mutex> g(g_tune_mu);
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;   // the cache is an optimisation: a write failure is not an error
  std::fprintf(fh, "%s\t%d %d %d %.6f\n", key.c_str(), threads, npt, ctas, ms);
  std::fclose(fh);
}

static ocp_status berr(ocp_batch* b, ocp_status st, const std::string& m) {
  const ocp_status s = set_err(nullptr, st, m);  // (marks a fault injected by OCP_FAULT)
  if (b) b->err = ocp_last_error(nullptr);
  return s;
}

template <class M>
static ocp_status batch_upload_inst(ocp_batch* b) {
  std::vector<NodeArgs<M>> inst(b->count);
  for (int i = 0; i < b->count; ++i) {
    fill_args<M>(b->items[i], 1.0, inst[i]);
    inst[i].B = 0;
    inst[i].E = b->items[i]->N + 1;
    inst[i].p0_dev = nullptr;
  }
  cudaError_t e = ocpg::dev_malloc(&b->d_inst, sizeof(NodeArgs<M>) * b->count);
  if (e != cudaSuccess) return berr(b, OCP_ENOMEM, "cudaMalloc(batch instances)");
  e = ocpg::dev_upload(b->d_inst, inst.data(), sizeof(NodeArgs<M>) * b->count);
  if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  // allow the largest shared-memory request of every configuration once
  for (const auto& cf : kConfigs) {
    if (!kernel_for<M>(cf.threads, cf.npt)) continue;   // not provided for this model
    e = cudaFuncSetAttribute(kernel_for<M>(cf.threads, cf.npt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<M>(cf.threads, cf.npt));
    if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  }
  return OCP_OK;
}

static ocp_status batch_tiles(ocp_batch* b) {
  const int64_t owned = (int64_t)b->npt * b->threads - 1;
  b->tileoff.assign(b->count + 1, 0);
  for (int i = 0; i < b->count; ++i) b->tileoff[i + 1] = b->tileoff[i] + (b->items[i]->N + 1 + owned - 1) / owned;
  b->ntiles = b->tileoff[b->count];
  if (b->ntiles > b->partials_cap) return berr(b, OCP_EDIM, "tile count exceeds the partial-sum buffer");
  cudaError_t e = ocpg::dev_upload(b->d_tileoff, b->tileoff.data(), sizeof(int64_t) * (b->count + 1));
  if (e != cudaSuccess) {
    b->unusable = true;
    return berr(b, OCP_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  }
  b->unusable = false;   // a later successful configuration makes the batch usable again
  return OCP_OK;
}

template <class M>
static int max_ctas_per_sm(const ocp_batch* b) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel_for<M>(b->threads, b->npt), b->threads,
                                                    smem_bytes<M>(b->threads, b->npt)) != cudaSuccess || per < 1)
    per = 1;
  return per;
}

template <class M>
static ocp_status batch_launch(ocp_batch* b, const double* x, const double* y, double sigma, double* f, double* c,
                               double* g, double* jv, double* hv, cudaStream_t s) {
  BatchArgs<M> a;
  memset(&a, 0, sizeof(a));
  a.inst = (const NodeArgs<M>*)b->d_inst;
  a.tileoff = b->d_tileoff; a.xoff = b->d_xoff; a.coff = b->d_coff; a.joff = b->d_joff; a.hoff = b->d_hoff;
  a.x = x; a.y = y; a.f = f; a.c = c; a.g = g; a.jv = jv; a.hv = hv;
  a.partials = b->d_partials; a.counter = b->d_counter;
  a.work = (unsigned long long*)(b->d_counter + 2);
  a.icount = b->d_counter + 4;
  a.sigma = sigma;
  a.ntiles = b->ntiles;
  a.count = b->count;
  const int per = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, max_ctas_per_sm<M>(b)) : max_ctas_per_sm<M>(b);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(b->ntiles, (int64_t)per * b->num_sms));
  const size_t sm = smem_bytes<M>(b->threads, b->npt);
  const int T = b->threads;
  auto go = [&](auto tt, auto pp) {
    constexpr int TT = decltype(tt)::value, PP = decltype(pp)::value;
    if constexpr (TT * PP <= batch_max_nodes<M>()) k_batch_eval<M, TT, PP><<<grid, TT, sm, s>>>(a);
  };
  using I64 = std::integral_constant<int, 64>;
  using I128 = std::integral_constant<int, 128>;
  using I256 = std::integral_constant<int, 256>;
  using P1 = std::integral_constant<int, 1>;
  using P2 = std::integral_constant<int, 2>;
  if (!kernel_for<M>(T, b->npt)) return berr(b, OCP_EINVAL, "configuration not provided for this model");
  if (b->npt == 1) {
    if (T == 64) go(I64{}, P1{}); else if (T == 128) go(I128{}, P1{}); else go(I256{}, P1{});
  } else {
    if (T == 64) go(I64{}, P2{}); else if (T == 128) go(I128{}, P2{}); else go(I256{}, P2{});
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return OCP_OK;
}

// Calls fn with a value of the batch's model type (the node models the batched form serves).
template <class Fn>
static auto with_model(int model, Fn&& fn) {
  switch (model) {
    case OCP_MODEL_CARTPOLE: return fn(CartPole{});
    case OCP_MODEL_DINT: return fn(Dint{});
    case OCP_MODEL_QUADROTOR: return fn(Quadrotor{});
    default: return fn(VdP{});
  }
}

static ocp_status dispatch_batch(ocp_batch* b, const double* x, const double* y, double sigma, double* f, double* c,
                                 double* g, double* jv, double* hv, cudaStream_t s) {
  return with_model(b->model, [&](auto m) {
    return batch_launch<decltype(m)>(b, x, y, sigma, f, c, g, jv, hv, s);
  });
}

static bool config_provided(const ocp_batch* b, int threads, int npt) {
  return with_model(b->model, [&](auto m) { return kernel_for<decltype(m)>(threads, npt) != nullptr; });
}

static void batch_free(ocp_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->d_inst); cudaFree(b->d_tileoff); cudaFree(b->d_xoff); cudaFree(b->d_coff); cudaFree(b->d_joff);
  cudaFree(b->d_hoff); cudaFree(b->d_partials); cudaFree(b->d_counter);
  delete b;
}

extern "C" {

ocp_status ocp_batch_create(ocp_t* const* items, int count, ocp_batch_t** out) {
  OCP_RANGE();
  if (!out) return set_err(nullptr, OCP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!items || count < 1) return set_err(nullptr, OCP_EINVAL, "need at least one problem");
  const int model = items[0] ? items[0]->model : 0;
  if (model != OCP_MODEL_CARTPOLE && model != OCP_MODEL_VDP && model != OCP_MODEL_DINT && model != OCP_MODEL_QUADROTOR)
    return set_err(nullptr, OCP_EMODEL,
                   "batched evaluation is provided for the Van der Pol, cart-pole, double-integrator and quadrotor models");
  for (int i = 0; i < count; ++i) {
    if (!items[i]) return set_err(nullptr, OCP_EINVAL, "NULL problem in the batch");
    if (items[i]->unusable) return set_err(nullptr, OCP_EINVAL, "a problem of the batch is unusable after a failed setter");
    if (items[i]->model != model) return set_err(nullptr, OCP_EMODEL, "all problems of a batch must share the model");
    if (items[i]->scheme != OCP_SCHEME_TRAPEZOID)
      return set_err(nullptr, OCP_EMODEL, "batched evaluation is provided for the trapezoidal scheme");
    if (items[i]->npath > 0) return set_err(nullptr, OCP_EMODEL, "batched evaluation has no path inequalities");
    if (items[i]->nbin > 0) return set_err(nullptr, OCP_EMODEL, "batched evaluation has no boundary inequalities");
    if (items[i]->has_bol) return set_err(nullptr, OCP_EMODEL, "batched evaluation has no boundary cost");
    if (items[i]->device != items[0]->device) return set_err(nullptr, OCP_EINVAL, "problems on different devices");
  }
  ocp_batch* b = new (std::nothrow) ocp_batch();
  if (!b) return set_err(nullptr, OCP_ENOMEM, "host allocation failed");
  b->model = model; b->count = count; b->device = items[0]->device; b->num_sms = items[0]->num_sms;
  b->items.assign(items, items + count);
  b->xoff.assign(count + 1, 0); b->coff.assign(count + 1, 0); b->joff.assign(count + 1, 0); b->hoff.assign(count + 1, 0);
  int64_t cap = 0;
  for (int i = 0; i < count; ++i) {
    const Pattern& P = items[i]->pat;
    b->xoff[i + 1] = b->xoff[i] + P.n;
    b->coff[i + 1] = b->coff[i] + P.m;
    b->joff[i + 1] = b->joff[i] + P.nnzj;
    b->hoff[i + 1] = b->hoff[i] + P.nnzh;
    cap += (items[i]->N + 1 + 62) / 63;  // tiles of the smallest configuration (64 threads, 1 node)
  }
  b->partials_cap = cap;
  cudaError_t e = cudaSuccess;
  auto up = [&](int64_t** d, const std::vector<int64_t>& h) -> cudaError_t {
    const cudaError_t r = ocpg::dev_malloc(d, sizeof(int64_t) * h.size());
    return r != cudaSuccess ? r : ocpg::dev_upload(*d, h.data(), sizeof(int64_t) * h.size());
  };
  if ((e = up(&b->d_xoff, b->xoff)) != cudaSuccess || (e = up(&b->d_coff, b->coff)) != cudaSuccess ||
      (e = up(&b->d_joff, b->joff)) != cudaSuccess || (e = up(&b->d_hoff, b->hoff)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&b->d_tileoff, sizeof(int64_t) * (count + 1))) != cudaSuccess ||
      (e = ocpg::dev_malloc(&b->d_partials, sizeof(double) * cap)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&b->d_counter, sizeof(unsigned) * (4 + count))) != cudaSuccess ||
      (e = cudaMemset(b->d_counter, 0, sizeof(unsigned) * (4 + count))) != cudaSuccess) {
    batch_free(b);
    return cuda_err(nullptr, e, "batch tables");   // OCP_ENOMEM for a failed allocation
  }
  ocp_status st = with_model(model, [&](auto m) { return batch_upload_inst<decltype(m)>(b); });
  if (st == OCP_OK) st = batch_tiles(b);
  if (st != OCP_OK) { batch_free(b); return st; }
  *out = b;
  return OCP_OK;
}

void ocp_batch_destroy(ocp_batch_t* b) { batch_free(b); }

ocp_status ocp_batch_offsets(const ocp_batch_t* b, int64_t* xoff, int64_t* coff, int64_t* joff, int64_t* hoff) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  for (int i = 0; i <= b->count; ++i) {
    if (xoff) xoff[i] = b->xoff[i];
    if (coff) coff[i] = b->coff[i];
    if (joff) joff[i] = b->joff[i];
    if (hoff) hoff[i] = b->hoff[i];
  }
  return OCP_OK;
}

ocp_status ocp_batch_set_config(ocp_batch_t* b, int nodes_per_thread, int threads, int ctas_per_sm) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if ((nodes_per_thread != 1 && nodes_per_thread != 2) || (threads != 64 && threads != 128 && threads != 256) ||
      ctas_per_sm < 0)
    return berr(b, OCP_EINVAL, "config: nodes_per_thread in {1,2}, threads in {64,128,256}, ctas_per_sm >= 0");
  if (!config_provided(b, threads, nodes_per_thread))
    return berr(b, OCP_EINVAL, "config: more nodes per CTA than this model's staged Jacobian rows fit in shared memory");
  b->npt = nodes_per_thread;
  b->threads = threads;
  b->ctas_per_sm = ctas_per_sm;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  return batch_tiles(b);
}

ocp_status ocp_batch_get_config(const ocp_batch_t* b, int* nodes_per_thread, int* threads, int* ctas_per_sm) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if (nodes_per_thread) *nodes_per_thread = b->npt;
  if (threads) *threads = b->threads;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  return OCP_OK;
}

ocp_status ocp_batch_eval_all(ocp_batch_t* b, const double* x, const double* y, double sigma, double* f, double* c,
                              double* g, double* jvals, double* hvals, void* stream) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if (b->unusable) return berr(b, OCP_EINVAL, "batch unusable after a failed configuration change");
  if (!x) return berr(b, OCP_EINVAL, "x is NULL");
  if (hvals && !y) return berr(b, OCP_EINVAL, "y is required for Hessian values");
  return dispatch_batch(b, x, y, sigma, f, c, g, jvals, hvals, (cudaStream_t)stream);
}

ocp_status ocp_batch_autotune(ocp_batch_t* b, const double* x, const double* y, double sigma, double* f, double* c,
                              double* g, double* jvals, double* hvals, void* stream, double* best_ms) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if (b->unusable) return berr(b, OCP_EINVAL, "batch unusable after a failed configuration change");
  const char* cache = std::getenv("OCP_AUTOTUNE_CACHE");
  const unsigned outs = (f ? 1u : 0u) | (c ? 2u : 0u) | (g ? 4u : 0u) | (jvals ? 8u : 0u) | (hvals ? 16u : 0u);
  const std::string key = tune_key(b, outs);
  {
    int ct = 0, cn = 0, cc = 0;
    float cms = 0.f;
    if (cache && *cache && tune_lookup(cache, key, ct, cn, cc, cms)) {
      if (best_ms) *best_ms = cms;
      return ocp_batch_set_config(b, cn, ct, cc);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return berr(b, OCP_ECUDA, "cudaEventCreate");
  float best = 1e30f;
  int bt = 128, bn = 1, bc = 0;
  ocp_status st = OCP_OK;
  for (const auto& cf : kConfigs) {
    if (!config_provided(b, cf.threads, cf.npt)) continue;
    b->threads = cf.threads; b->npt = cf.npt; b->ctas_per_sm = 0;
    if ((st = batch_tiles(b)) != OCP_OK) break;
    const int maxc = with_model(b->model, [&](auto m) { return max_ctas_per_sm<decltype(m)>(b); });
    for (int cps = maxc; cps >= 1; cps = (cps > 2 ? cps / 2 : cps - 1)) {
      b->ctas_per_sm = cps;
      if ((st = dispatch_batch(b, x, y, sigma, f, c, g, jvals, hvals, s)) != OCP_OK) break;  // warm-up
      float tms[3];
      for (int r = 0; r < 3 && st == OCP_OK; ++r) {
        cudaEventRecord(e0, s);
        st = dispatch_batch(b, x, y, sigma, f, c, g, jvals, hvals, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&tms[r], e0, e1);
      }
      if (st != OCP_OK) break;
      std::sort(tms, tms + 3);
      if (tms[1] < best) { best = tms[1]; bt = cf.threads; bn = cf.npt; bc = cps; }
    }
    if (st != OCP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != OCP_OK) return st;
  if (best_ms) *best_ms = best;
  if (cache && *cache) tune_store(cache, key, bt, bn, bc, best);
  return ocp_batch_set_config(b, bn, bt, bc);
}

ocp_status ocp_batch_graph_capture(ocp_batch_t* b, const double* x, const double* y, double sigma, double* f, double* c,
                                   double* g, double* jvals, double* hvals, void* stream) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if (b->unusable) return berr(b, OCP_EINVAL, "batch unusable after a failed configuration change");
  if (!stream) return berr(b, OCP_EINVAL, "graph capture needs a created (non-default) stream");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  ocp_status st = dispatch_batch(b, x, y, sigma, f, c, g, jvals, hvals, s);
  e = cudaStreamEndCapture(s, &gr);
  if (st != OCP_OK) { if (gr) cudaGraphDestroy(gr); return st; }
  if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) { b->graph = nullptr; return berr(b, OCP_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)); }
  return OCP_OK;
}

ocp_status ocp_batch_graph_launch(ocp_batch_t* b, void* stream) {
  OCP_RANGE();
  if (!b) return OCP_EINVAL;
  if (b->unusable) return berr(b, OCP_EINVAL, "batch unusable after a failed configuration change");
  if (!b->graph) return berr(b, OCP_EINVAL, "no captured graph");
  cudaError_t e = cudaGraphLaunch(b->graph, (cudaStream_t)stream);
  if (e != cudaSuccess) return berr(b, OCP_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  return OCP_OK;
}

const char* ocp_batch_last_error(const ocp_batch_t* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
