// C-ABI of the evaluator (declarations and contracts in include/ocp.h).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <unordered_map>

#include "ocp_internal.h"

using namespace ocpg;

static thread_local std::string g_create_err;

namespace ocpg {

ocp_status set_err(ocp* h, ocp_status st, const std::string& msg) {
  const std::string m = take_injected() ? msg + " (injected by OCP_FAULT)" : msg;
  if (h) h->err = m;
  else g_create_err = m;
  return st;
}

ocp_status cuda_err(ocp* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return OCP_OK;
  return set_err(h, e == cudaErrorMemoryAllocation ? OCP_ENOMEM : OCP_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

ocp_status unusable_err(const ocp* h) {
  ocp* m = const_cast<ocp*>(h);
  if (m->err.rfind("handle unusable", 0) != 0) m->err = "handle unusable after a failed setter: " + m->err;
  return OCP_EINVAL;
}

// One CTA per tile: the hardware block scheduler balances the tail.  (Results do not depend
// on the grid: reductions are per tile and summed in tile order.)
int occupancy_grid(ocp* h, const void* kernel, int threads, size_t smem, int64_t work_tiles) {
  (void)h; (void)kernel; (void)threads; (void)smem;
  if (work_tiles < 1) return 1;
  if (work_tiles > 0x7fffffff) return 0x7fffffff;
  return (int)work_tiles;
}

int64_t objective_tiles(int model, int64_t nodes) {
  int owned = 0;
  switch (model) {
    case OCP_MODEL_VDP: owned = TILE_VDP - 1; break;
    case OCP_MODEL_CARTPOLE: owned = TILE_CARTPOLE - 1; break;
    case OCP_MODEL_DINT: owned = TILE_DINT - 1; break;
    case OCP_MODEL_QUADROTOR: owned = TILE_QUAD_EVAL - 1; break;
    case OCP_MODEL_HEAT1D: owned = HEAT_TILE_NODES - 1; break;
    default: return -1;
  }
  return (nodes + owned - 1) / owned;
}

// Time-varying state reference, tabulated once per node: for the tracked components i,
//   out[ntrk j + i] = (xref + xslope t_j) + xamp sin(xfreq t_j),  t_j = j h
// (plain operations in this order, no FMA).  One thread per table entry.
// The start point: one value per state and control component at every node, then tf.
struct StartArgs {
  double* x;
  int64_t nX, nXU, n;     // ends of the X block, of the U block, of x
  int nx, nu;
  double tf;
  double xs[128], us[8];
};
__global__ void k_start_point(const __grid_constant__ StartArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
    a.x[i] = i < a.nX ? a.xs[i % a.nx] : (i < a.nXU ? a.us[(i - a.nX) % a.nu] : a.tf);
}

struct TrackArgs {
  double* out;
  int64_t N;
  double h;
  int ntrk;
  double ref[kMaxTrack], slope[kMaxTrack], amp[kMaxTrack], freq[kMaxTrack];
};

__global__ void k_fill_tracking(const __grid_constant__ TrackArgs a) {
  const int64_t total = (a.N + 1) * a.ntrk;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int64_t j = idx / a.ntrk;
    const int i = (int)(idx - j * a.ntrk);
    const double t = (double)j * a.h;
    const double lin = a.ref[i] + a.slope[i] * t;
    a.out[idx] = lin + a.amp[i] * sin(a.freq[i] * t);
  }
}

ocp_status fill_tracking(ocp* h) {
  TrackArgs a;
  memset(&a, 0, sizeof(a));
  a.out = h->d_xtrack; a.N = h->N; a.h = h->h; a.ntrk = h->ntrk;
  for (int i = 0; i < h->ntrk; ++i) {
    const int k = h->trk_comp[i];
    a.ref[i] = h->xref[k]; a.slope[i] = h->xslope[k]; a.amp[i] = h->xamp[k]; a.freq[i] = h->xfreq[k];
  }
  const int64_t total = (h->N + 1) * h->ntrk;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)h->num_sms * 8);
  k_fill_tracking<<<(int)std::max<int64_t>(blocks, 1), 256>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return cuda_err(h, e, "tracking table");
}

}  // namespace ocpg

// ---------------------------------------------------------------------------------------
static bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

static ocp_status upload_tables(ocp* h) {
  ocpg::scatter_map_free(h);  // built from the previous pattern
  cudaFree(h->d_rowtmpl); cudaFree(h->d_jbase); cudaFree(h->d_hent); cudaFree(h->d_fin); cudaFree(h->d_tcol);
  cudaFree(h->d_kcbase);
  h->d_rowtmpl = nullptr; h->d_jbase = nullptr; h->d_hent = nullptr; h->d_fin = nullptr; h->d_tcol = nullptr;
  h->d_kcbase = nullptr;
  const Pattern& P = h->pat;
  std::vector<int32_t> rt((size_t)RT_STRIDE * P.nx, -1);
  for (int k = 0; k < P.nx; ++k) {
    int32_t* t = rt.data() + (size_t)RT_STRIDE * k;
    t[0] = P.rows[k].rx;
    t[1] = P.rows[k].ru;
    for (int e = 0; e < RT_XV; ++e) t[2 + e] = P.rows[k].xv[e];
    for (int e = 0; e < RT_UV; ++e) t[2 + RT_XV + e] = P.rows[k].uv[e];
  }
  std::vector<int32_t> he;
  for (auto& e : P.hent) { he.push_back(e.first); he.push_back(e.second); }
  if (he.empty()) he.push_back(0);
  cudaError_t e;
  if ((e = ocpg::dev_malloc(&h->d_rowtmpl, rt.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_malloc(&h->d_jbase, P.jbase.size() * sizeof(int64_t))) != cudaSuccess) return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_malloc(&h->d_hent, he.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_upload(h->d_rowtmpl, rt.data(), rt.size() * 4)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  if ((e = ocpg::dev_upload(h->d_jbase, P.jbase.data(), P.jbase.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  if ((e = ocpg::dev_upload(h->d_hent, he.data(), he.size() * 4)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  std::vector<int32_t> fin(P.fin.begin(), P.fin.end()), tcol(P.tcol.begin(), P.tcol.end());
  if (fin.empty()) fin.push_back(0);
  if (tcol.empty()) tcol.push_back(0);
  if ((e = ocpg::dev_malloc(&h->d_fin, fin.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_malloc(&h->d_tcol, tcol.size() * sizeof(int32_t))) != cudaSuccess) return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_upload(h->d_fin, fin.data(), fin.size() * 4)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  if ((e = ocpg::dev_upload(h->d_tcol, tcol.data(), tcol.size() * 4)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  if ((e = ocpg::dev_malloc(&h->d_kcbase, P.kcbase.size() * sizeof(int64_t))) != cudaSuccess)
    return cuda_err(h, e, "cudaMalloc");
  if ((e = ocpg::dev_upload(h->d_kcbase, P.kcbase.data(), P.kcbase.size() * 8)) != cudaSuccess)
    return cuda_err(h, e, "cudaMemcpy");
  ocp_status st = path_upload(h);
  return st == OCP_OK ? bin_upload(h) : st;
}

// Rebuilds the pattern and its device tables after a setter changed the problem; a failure
// part-way leaves the handle unusable.
static ocp_status rebuild(ocp* h) {
  std::string why;
  ocp_status st = build_pattern(h, why) ? upload_tables(h) : set_err(h, OCP_EDIM, why);
  if (st != OCP_OK) h->unusable = true;
  return st;
}

static int model_nparams(int model) {
  switch (model) {
    case OCP_MODEL_VDP: return 1;
    case OCP_MODEL_CARTPOLE: return 4;
    case OCP_MODEL_HEAT1D: return 1;
    case OCP_MODEL_DINT: return 0;
    case OCP_MODEL_QUADROTOR: return 1;
    case OCP_MODEL_GODDARD: return 4;
  }
  return -1;
}

// Dynamics parameters with a derivative (the leading entries of params): the heat model's
// cell count is structural and the double integrator has none.
static int model_nderiv(int model) {
  switch (model) {
    case OCP_MODEL_VDP: return 1;
    case OCP_MODEL_CARTPOLE: return 4;
    case OCP_MODEL_GODDARD: return 4;
    case OCP_MODEL_QUADROTOR: return 1;
  }
  return 0;
}

static void free_handle(ocp* h) {
  if (!h) return;
  ocpg::host_step_free(h);
  ocpg::scatter_map_free(h);
  cudaFree(h->d_rowtmpl); cudaFree(h->d_jbase); cudaFree(h->d_hent); cudaFree(h->d_fin); cudaFree(h->d_tcol);
  cudaFree(h->d_kcbase);
  cudaFree(h->d_poff); cudaFree(h->d_pv); cudaFree(h->d_pcoef); cudaFree(h->d_pbase);
  cudaFree(h->d_boff); cudaFree(h->d_bv); cudaFree(h->d_bcoef); cudaFree(h->d_bbase);
  cudaFree(h->d_partials); cudaFree(h->d_counter); cudaFree(h->d_xtrack);
  delete h;
}

namespace ocpg {

// Host part of ocp_create: validation, parameters and the pattern; no device work.
ocp_status init_host(ocp* h, const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N, double T) {
  if (!dyn || !cost) return set_err(nullptr, OCP_EINVAL, "dynamics or cost is NULL");
  const int np = model_nparams(dyn->model);
  if (np < 0) return set_err(nullptr, OCP_EMODEL, "unknown model id");
  if (cost->kind != OCP_COST_DIAG_QUADRATIC) return set_err(nullptr, OCP_EMODEL, "unknown cost kind");
  if (dyn->nparams != np || (np > 0 && !dyn->params))
    return set_err(nullptr, OCP_EDIM, "wrong number of model parameters");
  int enx = 0, enu = 1;
  switch (dyn->model) {
    case OCP_MODEL_VDP: enx = 2; break;
    case OCP_MODEL_CARTPOLE: enx = 4; break;
    case OCP_MODEL_DINT: enx = 2; break;
    case OCP_MODEL_QUADROTOR: enx = 9; enu = 4; break;
    case OCP_MODEL_GODDARD: enx = 3; break;
    case OCP_MODEL_HEAT1D: {
      const double c = dyn->params[0];
      if (!(c >= 2.0 && c <= 128.0) || c != std::floor(c))
        return set_err(nullptr, OCP_EDIM, "heat model: ncell must be an integer in [2, 128]");
      enx = (int)c;
      break;
    }
  }
  if (nx != enx || nu != enu) return set_err(nullptr, OCP_EDIM, "wrong bound dimension: nx/nu disagree with the model");
  if (N < 1) return set_err(nullptr, OCP_EDIM, "N must be >= 1");
  if (!(T > 0.0) || !std::isfinite(T)) return set_err(nullptr, OCP_EINVAL, "T must be positive and finite");
  if (!cost->q || !cost->r) return set_err(nullptr, OCP_EINVAL, "cost weights q and r are required");
  if (dyn->model == OCP_MODEL_GODDARD) {
    for (int k = 0; k < nx; ++k)
      if (cost->q[k] != 0.0) return set_err(nullptr, OCP_EMODEL, "Goddard: the objective is a terminal cost (q and r must be zero)");
    for (int i = 0; i < nu; ++i)
      if (cost->r[i] != 0.0) return set_err(nullptr, OCP_EMODEL, "Goddard: the objective is a terminal cost (q and r must be zero)");
    for (int k = 0; k < nx && cost->xref; ++k)
      if (cost->xref[k] != 0.0) return set_err(nullptr, OCP_EMODEL, "Goddard: no running-cost reference");
    for (int i = 0; i < nu && cost->uref; ++i)
      if (cost->uref[i] != 0.0) return set_err(nullptr, OCP_EMODEL, "Goddard: no running-cost reference");
  }
  h->model = dyn->model; h->nx = nx; h->nu = nu; h->N = N; h->T = T;
  h->h = T / (double)N;
  h->hh = h->h / 2.0;
  h->params.assign(8, 0.0);
  for (int i = 0; i < np; ++i) h->params[i] = dyn->params[i];
  h->q.assign(cost->q, cost->q + nx);
  h->r.assign(cost->r, cost->r + nu);
  h->xref.assign(nx, 0.0);
  h->uref.assign(nu, 0.0);
  if (cost->xref) h->xref.assign(cost->xref, cost->xref + nx);
  if (cost->uref) h->uref.assign(cost->uref, cost->uref + nu);
  for (double v : h->xref) if (v != 0.0) h->has_ref = true;
  for (double v : h->uref) if (v != 0.0) h->has_ref = true;
  h->x0.assign(nx, 0.0);
  {
    const double inf = std::numeric_limits<double>::infinity();
    h->xlo.assign(nx, -inf); h->xhi.assign(nx, inf); h->ulo.assign(nu, -inf); h->uhi.assign(nu, inf);
    h->tflo = -inf; h->tfhi = inf;
  }
  std::string why;
  if (!build_pattern(h, why)) return set_err(nullptr, OCP_EDIM, why);
  return OCP_OK;
}

}  // namespace ocpg

extern "C" {

ocp_status ocp_create(const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N, double T,
                      ocp_t** out) {
  OCP_RANGE();
  if (!out) return set_err(nullptr, OCP_EINVAL, "out is NULL");
  *out = nullptr;
  ocp* h = new (std::nothrow) ocp();
  if (!h) return set_err(nullptr, OCP_ENOMEM, "host allocation failed");
  {
    ocp_status st = init_host(h, dyn, cost, nx, nu, N, T);
    if (st != OCP_OK) { delete h; return st; }
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { free_handle(h); return cuda_err(nullptr, e, "cudaGetDevice"); }
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
    free_handle(h);
    return cuda_err(nullptr, e, "cudaDeviceGetAttribute");
  }
  // one partial per tile of the smallest tile (31 owned nodes), plus slack: this also holds the
  // four parameter sums per 128-node chunk of the cart-pole's and six series per 255-node tile
  // of the Goddard model's (dc/dp)^T w
  h->max_partials = (int)((N + 1) / 31 + 8);
  if ((e = ocpg::dev_malloc(&h->d_partials, sizeof(double) * h->max_partials)) != cudaSuccess ||
      (e = ocpg::dev_malloc(&h->d_counter, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMemset(h->d_counter, 0, sizeof(unsigned))) != cudaSuccess) {
    free_handle(h);
    return set_err(nullptr, OCP_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  ocp_status st = upload_tables(h);
  if (st != OCP_OK) { std::string m = h->err; free_handle(h); return set_err(nullptr, st, m); }
  *out = h;
  return OCP_OK;
}

void ocp_destroy(ocp_t* h) { free_handle(h); }

ocp_status ocp_set_boundary(ocp_t* h, const double* x0, const double* xf) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  h->x0.assign(h->nx, 0.0);
  if (x0) h->x0.assign(x0, x0 + h->nx);
  const bool fin = xf != nullptr;
  if (fin) h->xf.assign(xf, xf + h->nx);
  else h->xf.clear();
  if (fin != h->has_final || !h->fin_comp.empty()) {
    h->has_final = fin;
    h->fin_comp.clear();
    return rebuild(h);
  }
  return OCP_OK;
}

ocp_status ocp_dims(const ocp_t* h, int64_t* n, int64_t* m, int64_t* nnzj, int64_t* nnzh) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (n) *n = h->pat.n;
  if (m) *m = h->pat.m;
  if (nnzj) *nnzj = h->pat.nnzj;
  if (nnzh) *nnzh = h->pat.nnzh;
  return OCP_OK;
}

ocp_status ocp_bounds(const ocp_t* h, double* lvar, double* uvar, double* lcon, double* ucon) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const double inf = std::numeric_limits<double>::infinity();
  const int64_t nxN = (int64_t)h->nx * (h->N + 1), nX = nxN + (int64_t)h->nu * h->pat.nun;
  for (int64_t i = 0; i < h->pat.n; ++i) {
    double lo, hi;
    if (i < nxN) { lo = h->xlo[i % h->nx]; hi = h->xhi[i % h->nx]; }
    else if (i < nX) { lo = h->ulo[(i - nxN) % h->nu]; hi = h->uhi[(i - nxN) % h->nu]; }
    else { lo = h->tflo; hi = h->tfhi; }  // the free final time
    if (lvar) lvar[i] = lo;
    if (uvar) uvar[i] = hi;
  }
  const int64_t nfin = h->pat.nb - h->nx;
  // path inequalities, then the boundary inequalities: (-inf, 0]
  const int64_t prow0 = h->pat.nb + (int64_t)h->nx * h->N;
  for (int64_t i = 0; i < h->pat.m; ++i) {
    double lo = 0.0, hi = 0.0;
    if (i < h->nx) lo = hi = h->x0[i];
    else if (i < h->nx + nfin) lo = hi = h->xf[i - h->nx];
    else if (i >= prow0) lo = -inf;
    if (lcon) lcon[i] = lo;
    if (ucon) ucon[i] = hi;
  }
  return OCP_OK;
}

}  // extern "C"

static ocp_status model_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  switch (h->model) {
    case OCP_MODEL_VDP: return node_eval_vdp(h, out, c, s);
    case OCP_MODEL_CARTPOLE: return node_eval_cartpole(h, out, c, s);
    case OCP_MODEL_DINT: return node_eval_dint(h, out, c, s);
    case OCP_MODEL_QUADROTOR: return node_eval_quad(h, out, c, s);
    case OCP_MODEL_GODDARD: return goddard_eval(h, out, c, s);
    case OCP_MODEL_HEAT1D: return heat_eval(h, out, c, s);
  }
  return set_err(h, OCP_EMODEL, "unknown model");
}

// The model's kernel, then (same stream) the path rows, then the boundary inequalities, with
// their updates.
ocp_status ocpg::dispatch_eval(ocp* h, unsigned out, const EvalCall& c, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  ocp_status st = model_eval(h, out, c, s);
  if (st == OCP_OK && h->pat.npath > 0) st = path_eval(h, out, c, s);
  if (st == OCP_OK && h->pat.nbin > 0) st = bin_eval(h, out, c, s);
  if (st == OCP_OK && h->has_bol) st = bol_eval(h, c, s);
  return st;
}

static ocp_status model_prod(ocp* h, const ProdCall& c, cudaStream_t s) {
  switch (h->model) {
    case OCP_MODEL_VDP: return node_prod_vdp(h, c, s);
    case OCP_MODEL_CARTPOLE: return node_prod_cartpole(h, c, s);
    case OCP_MODEL_DINT: return node_prod_dint(h, c, s);
    case OCP_MODEL_QUADROTOR: return node_prod_quad(h, c, s);
    case OCP_MODEL_GODDARD: return goddard_prod(h, c, s);
    case OCP_MODEL_HEAT1D: return heat_prod(h, c, s);
  }
  return set_err(h, OCP_EMODEL, "unknown model");
}

static ocp_status dispatch_prod(ocp* h, const ProdCall& c, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  ocp_status st = model_prod(h, c, s);
  if (st == OCP_OK && h->pat.npath > 0) st = path_prod(h, c, s);
  if (st == OCP_OK && h->pat.nbin > 0) st = bin_prod(h, c, s);
  if (st == OCP_OK && h->has_bol) st = bol_prod(h, c, s);
  return st;
}

static ocp_status need(ocp* h, const void* p, const char* name) {
  if (!p) return set_err(h, OCP_EINVAL, std::string(name) + " is NULL");
  if (!aligned8(p)) return set_err(h, OCP_EINVAL, std::string(name) + " is not 8-byte aligned");
  return OCP_OK;
}

#define NEED(p) do { ocp_status _s = need(h, (p), #p); if (_s != OCP_OK) return _s; } while (0)
#define OPT(p) do { if ((p) && !aligned8(p)) return set_err(h, OCP_EINVAL, #p " is not 8-byte aligned"); } while (0)

static EvalCall full_call(const ocp* h) {
  EvalCall c;
  c.B = 0;
  c.E = h->N + 1;
  return c;
}

// Sum of `count` doubles in index order by one thread (the rank-ordered combination of the
// shards' partial objectives and parameter derivatives: the same bits on every rank).
__global__ void k_sum_ordered(const double* parts, int count, double* out) {
  double s = 0.0;
  for (int i = 0; i < count; ++i) s = s + parts[i];
  *out = s;
}

extern "C" {

ocp_status eval_obj(ocp_t* h, const double* x, double* f, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(f);
  EvalCall c = full_call(h);
  c.x = x; c.f = f;
  return dispatch_eval(h, O_F, c, stream);
}

ocp_status eval_cons(ocp_t* h, const double* x, double* cv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(cv);
  EvalCall c = full_call(h);
  c.x = x; c.c = cv;
  return dispatch_eval(h, O_C, c, stream);
}

ocp_status eval_grad(ocp_t* h, const double* x, double* g, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(g);
  EvalCall c = full_call(h);
  c.x = x; c.g = g;
  return dispatch_eval(h, O_G, c, stream);
}

ocp_status jac_coo_structure(const ocp_t* h, int32_t* rows, int32_t* cols, void* stream) {
  OCP_RANGE();
  if (!h || !rows || !cols) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  return launch_jac_structure(h, rows, cols, (cudaStream_t)stream);
}

ocp_status jac_coo_values(ocp_t* h, const double* x, double* vals, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(vals);
  EvalCall c = full_call(h);
  c.x = x; c.jv = vals;
  return dispatch_eval(h, O_J, c, stream);
}

ocp_status hess_coo_structure(const ocp_t* h, int32_t* rows, int32_t* cols, void* stream) {
  OCP_RANGE();
  if (!h || !rows || !cols) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  return launch_hess_structure(h, rows, cols, (cudaStream_t)stream);
}

ocp_status hess_coo_values(ocp_t* h, const double* x, const double* y, double sigma, double* vals, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(y); NEED(vals);
  EvalCall c = full_call(h);
  c.x = x; c.y = y; c.sigma = sigma; c.hv = vals;
  return dispatch_eval(h, O_H, c, stream);
}

ocp_status jprod(ocp_t* h, const double* x, const double* v, double* Jv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(v); NEED(Jv);
  ProdCall c;
  c.kind = P_JPROD; c.x = x; c.v = v; c.out = Jv;
  return dispatch_prod(h, c, stream);
}

ocp_status jtprod(ocp_t* h, const double* x, const double* v, double* Jtv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(v); NEED(Jtv);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = v; c.out = Jtv;
  return dispatch_prod(h, c, stream);
}

ocp_status hprod(ocp_t* h, const double* x, const double* y, double sigma, const double* v, double* Hv,
                 void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(y); NEED(v); NEED(Hv);
  ProdCall c;
  c.kind = P_HPROD; c.x = x; c.y = y; c.sigma = sigma; c.v = v; c.out = Hv;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_eval_all(ocp_t* h, const double* x, const double* y, double sigma, double* f, double* cv, double* g,
                        double* jvals, double* hvals, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x);
  OPT(f); OPT(cv); OPT(g); OPT(jvals); OPT(hvals);
  if (hvals) NEED(y);
  unsigned out = (f ? O_F : 0u) | (cv ? O_C : 0u) | (g ? O_G : 0u) | (jvals ? O_J : 0u) | (hvals ? O_H : 0u);
  if (!out) return OCP_OK;
  EvalCall c = full_call(h);
  c.x = x; c.y = y; c.sigma = sigma; c.f = f; c.c = cv; c.g = g; c.jv = jvals; c.hv = hvals;
  // subsets without a dedicated kernel run the full kernel, which skips the NULL outputs
  return dispatch_eval(h, out, c, stream);
}

ocp_status ocp_eval_step(ocp_t* h, const double* x, const double* y, double sigma, const double* vn, const double* vm,
                         double* f, double* cv, double* g, double* jvals, double* hvals, double* Jv, double* Jtv,
                         double* Hv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(y); NEED(vn); NEED(vm); NEED(f); NEED(cv); NEED(g); NEED(jvals); NEED(hvals);
  NEED(Jv); NEED(Jtv); NEED(Hv);
  if (h->model == OCP_MODEL_HEAT1D) {
    // the heat model runs two kernels in sequence: the evaluation, and Jv, J^T w and H v in one
    // launch; then each product's path, boundary-inequality and boundary-cost terms as in the
    // separate calls (each array's own operations in the same order: the same bits)
    ocp_status st = ocp_eval_all(h, x, y, sigma, f, cv, g, jvals, hvals, stream);
    ProdCall a, b, c;
    a.kind = P_JPROD; a.x = x; a.v = vn; a.out = Jv;
    b.kind = P_JTPROD; b.x = x; b.v = vm; b.out = Jtv;
    c.kind = P_HPROD; c.x = x; c.y = y; c.sigma = sigma; c.v = vn; c.out = Hv;
    cudaStream_t s = (cudaStream_t)stream;
    if (st == OCP_OK) st = heat_prod2(h, a, b, &c, s);
    for (const ProdCall* pc : {&a, &b, &c}) {
      if (st == OCP_OK && h->pat.npath > 0) st = path_prod(h, *pc, s);
      if (st == OCP_OK && h->pat.nbin > 0) st = bin_prod(h, *pc, s);
      if (st == OCP_OK && h->has_bol) st = bol_prod(h, *pc, s);
    }
    return st;
  }
  EvalCall c = full_call(h);
  c.x = x; c.y = y; c.sigma = sigma; c.f = f; c.c = cv; c.g = g; c.jv = jvals; c.hv = hvals;
  c.vn = vn; c.vm = vm; c.ojv = Jv; c.ojtv = Jtv; c.ohv = Hv;
  return dispatch_eval(h, O_STEP, c, stream);
}

ocp_status ocp_eval_all_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x, const double* y,
                              double sigma, double* f, double* cv, double* g, double* jvals, double* hvals,
                              void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (node_begin < 0 || node_end > h->N + 1 || node_begin >= node_end)
    return set_err(h, OCP_EDIM, "node range outside [0, N+1) or empty");
  if (h->model == OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "node ranges are not provided for the Goddard model (tf couples every node)");
  if (h->nbin > 0)
    return set_err(h, OCP_EMODEL, "node ranges are not provided with boundary inequalities (they couple nodes 0 and N)");
  if (h->has_bol)
    return set_err(h, OCP_EMODEL, "node ranges are not provided with a boundary cost (it couples nodes 0 and N)");
  NEED(x); NEED(y); NEED(f); NEED(cv); NEED(g); NEED(jvals); NEED(hvals);
  EvalCall c;
  c.B = node_begin; c.E = node_end; c.range = true;
  c.x = x; c.y = y; c.sigma = sigma; c.f = f; c.c = cv; c.g = g; c.jv = jvals; c.hv = hvals;
  return dispatch_eval(h, O_ALL, c, stream);
}

// The node ranges of the sharded evaluation: [B, E) inside [0, N+1), node models with the
// trapezoidal scheme, nothing that couples node 0 with node N.
static ocp_status check_range(ocp* h, int64_t B, int64_t E, bool products) {
  if (B < 0 || E > h->N + 1 || B >= E) return set_err(h, OCP_EDIM, "node range outside [0, N+1) or empty");
  if (h->model == OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "node ranges are not provided for the Goddard model (tf couples every node)");
  if (products && h->model == OCP_MODEL_HEAT1D)
    return set_err(h, OCP_EMODEL, "node ranges of the fused step are provided for the node models, not the heat model");
  if (h->scheme != OCP_SCHEME_TRAPEZOID)
    return set_err(h, OCP_EMODEL, "node ranges are provided for the trapezoidal scheme");
  if (h->nbin > 0)
    return set_err(h, OCP_EMODEL, "node ranges are not provided with boundary inequalities (they couple nodes 0 and N)");
  if (h->has_bol)
    return set_err(h, OCP_EMODEL, "node ranges are not provided with a boundary cost (it couples nodes 0 and N)");
  return OCP_OK;
}

ocp_status ocp_eval_step_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x, const double* y,
                               double sigma, const double* vn, const double* vm, double* f, double* cv, double* g,
                               double* jvals, double* hvals, double* Jv, double* Jtv, double* Hv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  ocp_status st = check_range(h, node_begin, node_end, true);
  if (st != OCP_OK) return st;
  NEED(x); NEED(y); NEED(vn); NEED(vm); NEED(f); NEED(cv); NEED(g); NEED(jvals); NEED(hvals);
  NEED(Jv); NEED(Jtv); NEED(Hv);
  EvalCall c;
  c.B = node_begin; c.E = node_end; c.range = true;
  c.x = x; c.y = y; c.sigma = sigma; c.f = f; c.c = cv; c.g = g; c.jv = jvals; c.hv = hvals;
  c.vn = vn; c.vm = vm; c.ojv = Jv; c.ojtv = Jtv; c.ohv = Hv;
  return dispatch_eval(h, O_STEP, c, stream);
}

ocp_status ocp_vjp_param_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x, const double* w,
                               double* Jtw, double* dmu, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_VDP) return set_err(h, OCP_EMODEL, "parameter derivative is provided for the Van der Pol model");
  ocp_status st = check_range(h, node_begin, node_end, true);
  if (st != OCP_OK) return st;
  NEED(x); NEED(w); NEED(dmu); NEED(Jtw);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = w; c.out = Jtw; c.dmu = dmu;
  c.B = node_begin; c.E = node_end;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_sum_ordered(const double* parts, int count, double* out, void* stream) {
  OCP_RANGE();
  if (!parts || !out || count < 1) return set_err(nullptr, OCP_EINVAL, "ocp_sum_ordered: parts, out and count >= 1 required");
  if (((uintptr_t)parts & 7u) || ((uintptr_t)out & 7u)) return set_err(nullptr, OCP_EINVAL, "ocp_sum_ordered: unaligned pointer");
  k_sum_ordered<<<1, 1, 0, (cudaStream_t)stream>>>(parts, count, out);
  return cuda_err(nullptr, cudaGetLastError(), "k_sum_ordered launch");
}

ocp_status ocp_value_layout(const ocp_t* h, int64_t* nb, int32_t* row_count, int32_t* hx, int32_t* hu) {
  OCP_RANGE();
  if (!h || !nb || !row_count || !hx || !hu) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  *nb = h->pat.nb;
  for (int k = 0; k < h->nx; ++k) row_count[k] = (int32_t)h->pat.row_count(k);
  *hx = h->pat.hx;
  *hu = h->pat.hu;
  return OCP_OK;
}

// The handle reads params[0] from the device scalar p0 for the duration of one call (the
// launch copies the pointer into its arguments, so the previous binding returns right after).
struct ParamScope {
  ocp* h;
  const double* prev;
  ParamScope(ocp* hh, const double* p0) : h(hh), prev(hh->p0_dev) { if (p0) h->p0_dev = p0; }
  ~ParamScope() { h->p0_dev = prev; }
};

ocp_status ocp_eval_cons_p(ocp_t* h, const double* x, const double* p0, double* cv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(cv); OPT(p0);
  if (p0 && h->model != OCP_MODEL_VDP) return set_err(h, OCP_EMODEL, "a device parameter is provided for the Van der Pol model");
  ParamScope ps(h, p0);
  EvalCall c = full_call(h);
  c.x = x; c.c = cv;
  return dispatch_eval(h, O_C, c, stream);
}

ocp_status ocp_vjp_param_p(ocp_t* h, const double* x, const double* w, const double* p0, double* Jtw, double* dmu,
                           void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_VDP) return set_err(h, OCP_EMODEL, "parameter derivative is provided for the Van der Pol model");
  NEED(x); NEED(w); NEED(dmu); NEED(Jtw); OPT(p0);
  ParamScope ps(h, p0);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = w; c.out = Jtw; c.dmu = dmu;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_vjp_params_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x, const double* w,
                                const double* p, double* Jtw, double* dp, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (model_nderiv(h->model) == 0)
    return set_err(h, OCP_EMODEL, "the model has no dynamics parameters with a derivative");
  ocp_status st = check_range(h, node_begin, node_end, true);
  if (st != OCP_OK) return st;
  NEED(x); NEED(w); NEED(Jtw); NEED(dp); OPT(p);
  ParamScope ps(h, p);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = w; c.out = Jtw; c.dmu = dp;
  c.B = node_begin; c.E = node_end;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_param_count(const ocp_t* h, int* np) {
  OCP_RANGE();
  if (!h || !np) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  *np = model_nderiv(h->model);
  return OCP_OK;
}

ocp_status ocp_set_params(ocp_t* h, const double* p, int np) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const int want = model_nderiv(h->model);
  if (want == 0) return set_err(h, OCP_EMODEL, "the model has no dynamics parameters with a derivative");
  if (np != want) return set_err(h, OCP_EDIM, "wrong number of dynamics parameters");
  if (!p) return set_err(h, OCP_EINVAL, "p is NULL");
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(p[i])) return set_err(h, OCP_EINVAL, "parameters must be finite");
  for (int i = 0; i < np; ++i) h->params[i] = p[i];
  return OCP_OK;
}

ocp_status ocp_eval_cons_params(ocp_t* h, const double* x, const double* p, double* cv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(cv); OPT(p);
  if (p && model_nderiv(h->model) == 0)
    return set_err(h, OCP_EMODEL, "the model has no dynamics parameters with a derivative");
  ParamScope ps(h, p);
  EvalCall c = full_call(h);
  c.x = x; c.c = cv;
  return dispatch_eval(h, O_C, c, stream);
}

ocp_status ocp_vjp_params(ocp_t* h, const double* x, const double* w, const double* p, double* Jtw, double* dp,
                          void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (model_nderiv(h->model) == 0)
    return set_err(h, OCP_EMODEL, "the model has no dynamics parameters with a derivative");
  NEED(x); NEED(w); NEED(Jtw); NEED(dp); OPT(p);
  ParamScope ps(h, p);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = w; c.out = Jtw; c.dmu = dp;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_vjp_param(ocp_t* h, const double* x, const double* w, double* Jtw, double* dmu, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_VDP) return set_err(h, OCP_EMODEL, "parameter derivative is provided for the Van der Pol model");
  NEED(x); NEED(w); NEED(dmu); NEED(Jtw);
  ProdCall c;
  c.kind = P_JTPROD; c.x = x; c.v = w; c.out = Jtw; c.dmu = dmu;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_bind_param0(ocp_t* h, const double* p0_dev) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (p0_dev && h->model != OCP_MODEL_VDP)
    return set_err(h, OCP_EMODEL, "a device parameter is provided for the Van der Pol model");
  OPT(p0_dev);
  h->p0_dev = p0_dev;
  return OCP_OK;
}

ocp_status ocp_bind_params(ocp_t* h, const double* p_dev) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (p_dev && model_nderiv(h->model) == 0)
    return set_err(h, OCP_EMODEL, "the model has no dynamics parameters with a derivative");
  OPT(p_dev);
  h->p0_dev = p_dev;
  return OCP_OK;
}

ocp_status ocp_jprod_param(ocp_t* h, const double* x, const double* v, const double* s, double* Jv, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(v); NEED(Jv); OPT(s);
  if (s && h->model != OCP_MODEL_VDP) return set_err(h, OCP_EMODEL, "parameter direction: Van der Pol model only");
  ProdCall c;
  c.kind = P_JPROD; c.x = x; c.v = v; c.out = Jv; c.pdir_dev = s;
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_hprod_param(ocp_t* h, const double* x, const double* y, double sigma, const double* v, const double* s,
                           double* Hv, double* dmu, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(y); NEED(v); NEED(Hv); OPT(s); OPT(dmu);
  if ((s || dmu) && h->model != OCP_MODEL_VDP)
    return set_err(h, OCP_EMODEL, "mixed parameter term: Van der Pol model only");
  if (dmu && !s) return set_err(h, OCP_EINVAL, "dmu needs the scale s (pass a device zero for none)");
  ProdCall c;
  c.kind = P_HPROD; c.x = x; c.y = y; c.sigma = sigma; c.v = v; c.out = Hv;
  if (s) { c.mixw = y; c.mixs = s; c.dmu = dmu; }
  return dispatch_prod(h, c, stream);
}

ocp_status ocp_eval_grad_scaled(ocp_t* h, const double* x, const double* s, double* g, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(s); NEED(g);
  if (h->has_bol) return set_err(h, OCP_EMODEL, "the objective-only kernels do not include a boundary cost");
  return obj_launch(h, false, x, s, nullptr, g, nullptr, (cudaStream_t)stream);
}

ocp_status ocp_obj_hvp(ocp_t* h, const double* x, const double* s, const double* v, double* Hv, double* dot,
                       void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x); NEED(s); NEED(v); NEED(Hv); OPT(dot);
  if (h->has_bol) return set_err(h, OCP_EMODEL, "the objective-only kernels do not include a boundary cost");
  return obj_launch(h, true, x, s, v, Hv, dot, (cudaStream_t)stream);
}

ocp_status ocp_set_param0(ocp_t* h, double value) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (model_nparams(h->model) < 1) return set_err(h, OCP_EMODEL, "model has no parameters");
  if (h->model == OCP_MODEL_HEAT1D) return set_err(h, OCP_EMODEL, "the heat cell count is structural");
  h->params[0] = value;
  return OCP_OK;
}

ocp_status ocp_set_path_constraints(ocp_t* h, int npath, const double* a, const double* b, const double* l,
                                    const double* r) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const int nz = h->nx + h->nu;
  if (npath < 0 || npath > 16) return set_err(h, OCP_EINVAL, "between 0 and 16 path inequalities");
  if (npath > 0 && (!a || !b || !l || !r)) return set_err(h, OCP_EINVAL, "a, b, l and r are required");
  for (int i = 0; i < npath * nz; ++i)
    if (!std::isfinite(a[i]) || !std::isfinite(b[i]) || !std::isfinite(l[i]))
      return set_err(h, OCP_EINVAL, "path coefficients must be finite");
  for (int p = 0; p < npath; ++p) {
    bool any = false;
    for (int v = 0; v < nz; ++v) any = any || a[p * nz + v] != 0.0 || l[p * nz + v] != 0.0;
    if (!any) return set_err(h, OCP_EINVAL, "a path inequality without any variable");
  }
  h->npath = npath;
  h->path_a.assign(a, a + (size_t)npath * nz);
  h->path_b.assign(b, b + (size_t)npath * nz);
  h->path_l.assign(l, l + (size_t)npath * nz);
  h->path_r.assign(r, r + npath);
  return rebuild(h);
}

ocp_status ocp_set_boundary_inequalities(ocp_t* h, int nbin, const double* a, const double* b, const double* l,
                                         const double* r) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const int bz = 2 * h->nx;
  if (nbin < 0 || nbin > 16) return set_err(h, OCP_EINVAL, "between 0 and 16 boundary inequalities");
  if (nbin > 0 && (!a || !b || !l || !r)) return set_err(h, OCP_EINVAL, "a, b, l and r are required");
  if (nbin > 0 && h->scheme == OCP_SCHEME_EULER)
    return set_err(h, OCP_EMODEL, "boundary inequalities are provided for the trapezoidal scheme");
  for (int i = 0; i < nbin * bz; ++i)
    if (!std::isfinite(a[i]) || !std::isfinite(b[i]) || !std::isfinite(l[i]))
      return set_err(h, OCP_EINVAL, "boundary inequality coefficients must be finite");
  for (int q = 0; q < nbin; ++q) {
    if (!std::isfinite(r[q])) return set_err(h, OCP_EINVAL, "boundary inequality coefficients must be finite");
    bool any = false;
    for (int v = 0; v < bz; ++v) any = any || a[q * bz + v] != 0.0 || l[q * bz + v] != 0.0;
    if (!any) return set_err(h, OCP_EINVAL, "a boundary inequality without any variable");
  }
  h->nbin = nbin;
  h->bin_a.assign(a, a + (size_t)nbin * bz);
  h->bin_b.assign(b, b + (size_t)nbin * bz);
  h->bin_l.assign(l, l + (size_t)nbin * bz);
  h->bin_r.assign(r, r + nbin);
  return rebuild(h);
}

ocp_status ocp_start_point(ocp_t* h, const double* xs, const double* us, double tf, double* x, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  NEED(x);
  if (h->nx > 128 || h->nu > 8) return set_err(h, OCP_EDIM, "start point: too many components");
  StartArgs a;
  memset(&a, 0, sizeof(a));
  a.x = x;
  a.nX = (int64_t)h->nx * (h->N + 1);
  a.nXU = a.nX + (int64_t)h->nu * h->pat.nun;
  a.n = h->pat.n;
  a.nx = h->nx; a.nu = h->nu; a.tf = tf;
  for (int k = 0; k < h->nx; ++k) a.xs[k] = xs ? xs[k] : 0.0;
  for (int i = 0; i < h->nu; ++i) a.us[i] = us ? us[i] : 0.0;
  const int64_t blocks = std::min<int64_t>((a.n + 255) / 256, (int64_t)h->num_sms * 8);
  k_start_point<<<(int)std::max<int64_t>(blocks, 1), 256, 0, (cudaStream_t)stream>>>(a);
  return cuda_err(h, cudaGetLastError(), "k_start_point launch");
}

ocp_status ocp_set_boundary_cost(ocp_t* h, const double* a, const double* b, const double* l) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const int bz = 2 * h->nx;
  if (!a && !b && !l) {
    h->has_bol = false;
    h->bol_a.clear(); h->bol_b.clear(); h->bol_l.clear();
    return rebuild(h);
  }
  if (!a || !b || !l) return set_err(h, OCP_EINVAL, "a, b and l are required (all NULL removes the cost)");
  for (int v = 0; v < bz; ++v)
    if (!std::isfinite(a[v]) || !std::isfinite(b[v]) || !std::isfinite(l[v]))
      return set_err(h, OCP_EINVAL, "boundary cost coefficients must be finite");
  if (h->scheme == OCP_SCHEME_EULER)
    for (int k = 0; k < h->nx; ++k)
      if (a[h->nx + k] != 0.0)
        return set_err(h, OCP_EMODEL, "with the Euler scheme the boundary cost is linear in X_N");
  h->has_bol = true;
  h->bol_a.assign(a, a + bz); h->bol_b.assign(b, b + bz); h->bol_l.assign(l, l + bz);
  return rebuild(h);
}

ocp_status ocp_set_scheme(ocp_t* h, int scheme) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (scheme == OCP_SCHEME_EULER && h->has_bol)
    for (int k = 0; k < h->nx; ++k)
      if (h->bol_a[h->nx + k] != 0.0)
        return set_err(h, OCP_EMODEL, "with the Euler scheme the boundary cost is linear in X_N");
  if (scheme != OCP_SCHEME_TRAPEZOID && scheme != OCP_SCHEME_EULER) return set_err(h, OCP_EINVAL, "unknown scheme");
  if (scheme == OCP_SCHEME_EULER && h->nbin > 0)
    return set_err(h, OCP_EMODEL, "boundary inequalities are provided for the trapezoidal scheme");
  if (scheme == OCP_SCHEME_EULER && (h->model == OCP_MODEL_HEAT1D || h->model == OCP_MODEL_GODDARD))
    return set_err(h, OCP_EMODEL, "the Euler scheme is provided for the VDP, CARTPOLE, DINT and QUADROTOR models");
  h->scheme = scheme;
  return rebuild(h);
}

ocp_status ocp_set_free_final_time(ocp_t* h, int enable) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "a free final time is provided for the Goddard model");
  h->free_tf = enable != 0;
  return rebuild(h);
}

ocp_status ocp_set_final_components(ocp_t* h, int count, const int32_t* comps, const double* values) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "final rows on a subset of the state are provided for the Goddard model "
                                  "(ocp_set_boundary sets them on every component)");
  if (count < 0 || count > h->nx || (count > 0 && (!comps || !values)))
    return set_err(h, OCP_EINVAL, "final components: bad count or NULL arrays");
  for (int i = 0; i < count; ++i)
    if (comps[i] < 0 || comps[i] >= h->nx || (i > 0 && comps[i] <= comps[i - 1]))
      return set_err(h, OCP_EINVAL, "final components must be ascending state indices");
  h->fin_comp.assign(comps, comps + count);
  h->xf.assign(values, values + count);
  h->has_final = count > 0;
  if (count == h->nx) h->fin_comp.clear();  // every component: the plain final rows
  return rebuild(h);
}

ocp_status ocp_set_terminal_cost(ocp_t* h, const double* mayer) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model != OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "a terminal cost is provided for the Goddard model");
  if (mayer) h->mayer.assign(mayer, mayer + h->nx);
  else h->mayer.clear();
  return OCP_OK;
}

ocp_status ocp_set_variable_bounds(ocp_t* h, const double* xlo, const double* xhi, const double* ulo,
                                   const double* uhi, double tflo, double tfhi) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const double inf = std::numeric_limits<double>::infinity();
  h->xlo.assign(h->nx, -inf); h->xhi.assign(h->nx, inf); h->ulo.assign(h->nu, -inf); h->uhi.assign(h->nu, inf);
  if (xlo) h->xlo.assign(xlo, xlo + h->nx);
  if (xhi) h->xhi.assign(xhi, xhi + h->nx);
  if (ulo) h->ulo.assign(ulo, ulo + h->nu);
  if (uhi) h->uhi.assign(uhi, uhi + h->nu);
  h->tflo = tflo;
  h->tfhi = tfhi;
  return OCP_OK;
}

ocp_status ocp_set_tracking(ocp_t* h, const double* xslope, const double* xamp, const double* xfreq) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  if (h->model == OCP_MODEL_HEAT1D || h->model == OCP_MODEL_GODDARD)
    return set_err(h, OCP_EMODEL, "a time-varying reference is provided for the node models with a running cost");
  const int nx = h->nx;
  h->xslope.assign(nx, 0.0); h->xamp.assign(nx, 0.0); h->xfreq.assign(nx, 0.0);
  if (xslope) h->xslope.assign(xslope, xslope + nx);
  if (xamp) h->xamp.assign(xamp, xamp + nx);
  if (xfreq) h->xfreq.assign(xfreq, xfreq + nx);
  for (int k = 0; k < nx; ++k)
    if (!std::isfinite(h->xslope[k]) || !std::isfinite(h->xamp[k]) || !std::isfinite(h->xfreq[k]))
      return set_err(h, OCP_EINVAL, "tracking coefficients must be finite");
  h->trk_comp.clear();
  for (int k = 0; k < nx; ++k)
    if (h->xslope[k] != 0.0 || (h->xamp[k] != 0.0 && h->xfreq[k] != 0.0)) h->trk_comp.push_back(k);
  cudaFree(h->d_xtrack);
  h->d_xtrack = nullptr;
  h->ntrk = 0;
  h->has_ref = false;
  for (double v : h->xref) if (v != 0.0) h->has_ref = true;
  for (double v : h->uref) if (v != 0.0) h->has_ref = true;
  if (h->trk_comp.empty()) return OCP_OK;
  if ((int)h->trk_comp.size() > kMaxTrack) return set_err(h, OCP_EDIM, "too many tracked components");
  const size_t bytes = sizeof(double) * (size_t)(h->N + 1) * h->trk_comp.size();
  cudaError_t e = ocpg::dev_malloc(&h->d_xtrack, bytes);
  if (e != cudaSuccess) { h->d_xtrack = nullptr; h->trk_comp.clear(); return cuda_err(h, e, "cudaMalloc(tracking table)"); }
  h->ntrk = (int)h->trk_comp.size();
  h->has_ref = true;
  return fill_tracking(h);
}

const char* ocp_last_error(const ocp_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

}  // extern "C"
