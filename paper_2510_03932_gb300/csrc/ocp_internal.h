// Internal declarations shared by the C-ABI, the host pattern compiler and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "ocp.h"
#include "kernel_config.h"

#include <nvtx3/nvToolsExt.h>

namespace ocpg {

// NVTX range around each C-ABI call (named after the call), for timeline profilers; without a
// profiler attached the push and pop are a few instructions each.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define OCP_RANGE() ::ocpg::NvtxRange ocp_nvtx_range_(__func__)

// Host pattern: sizes, slot offsets and the node templates (paper Sec. 5: the generators
// make one row per state component per interval; the pattern compiler lays out the COO
// slots of every (component, interval) row and of every node's Hessian block).
struct HostStep;    // see host_step.cu
struct ScatterMap;  // see scatter_map.cu

struct Pattern {
  int nx = 0, nu = 0, nz = 0;
  int64_t N = 0, n = 0, m = 0, nb = 0, nnzj = 0, nnzh = 0;
  std::vector<RowTemplate> rows;         // per component k
  std::vector<int64_t> jbase;            // slot of row (k, 0); size nx + 1 (last = nnzj)
  std::vector<std::pair<int, int>> hent; // node Hessian entries (a, b), canonical order
  int hx = 0, hu = 0;                    // entries per node in the X block / U block
  int64_t hbase_u = 0;                   // first slot of the U block = (N+1) * hx
  std::vector<int8_t> hpos;              // per max-template entry: position in its block or -1
  // free final time tf (the last unknown, index n - 1): one more entry closing every defect
  // row (its tf column) and a Hessian row of tf against the node variables tcol (local
  // indices: tx state columns, then tu control columns) of every node
  int free_tf = 0;
  int scheme = 0;                        // OCP_SCHEME_TRAPEZOID or OCP_SCHEME_EULER
  int64_t nun = 0;                       // nodes with controls and Hessian blocks (N+1, or N for Euler)
  int tx = 0, tu = 0;
  std::vector<int> tcol;
  int64_t hbase_t = 0;                   // first slot of the tf row = (N+1) * (hx + hu)
  std::vector<int> fin;                  // components with a final row X_{N,k}, ascending
  int row_count(int k) const {
    return scheme == OCP_SCHEME_EULER ? rows[k].rx + 1 + rows[k].ru : rows[k].count() + free_tf;
  }
  // KKT matrix [H + D, J^T; J, -delta_c I] (lower triangle, sorted by (row, col)): per-node
  // templates of the (1,1) rows, X then U, with the diagonal appended to rows where H has
  // none; src = position in the node's H block or -1 for an added diagonal
  struct KEnt { int src, a, b; };
  std::vector<KEnt> kxt, kut;
  int64_t kb_u = 0, kb_t = 0, kb_c = 0, nnzk = -1;  // slot bases; nnzk = -1: too large for int32
  std::vector<int64_t> kcbase;           // KKT slot of the first defect row of component k (nx + 1)
  // path inequalities: rows nb + nx N + p nun + i; row (p, i) has its entries on the
  // variables psupp[p] (local, ascending) of node i, at jpbase[p] + i * psupp[p].size()
  int npath = 0;
  std::vector<std::vector<int>> psupp;
  std::vector<int64_t> jpbase;           // npath + 1
  std::vector<int64_t> kpbase;           // KKT slots of the path rows (npath + 1)
  std::vector<int> hdiag;                // position of (v, v) in its node block (X or U), or -1
  // boundary inequalities b_q(X_0, X_N) <= 0: rows nb + nx N + npath nun + q (after the path
  // rows); row q has its entries on the variables bsupp[q] of z = (X_0, X_N) (local, ascending:
  // v < nx is X_{0,v}, nx + v is X_{N,v}) at jbbase[q]..; KKT slots kbbase[q]..
  int nbin = 0;
  std::vector<std::vector<int>> bsupp;
  std::vector<int64_t> jbbase;           // nbin + 1
  std::vector<int64_t> kbbase;           // nbin + 1
};

}  // namespace ocpg

struct ocp {
  int model = 0, nx = 0, nu = 0;
  int64_t N = 0;
  double T = 0, h = 0, hh = 0;
  std::vector<double> params, q, r, xref, uref, x0, xf;
  bool has_final = false, has_ref = false;
  // final rows on a subset of the components (fin_comp, ascending; empty: all of them when
  // has_final), a free final time and a linear terminal cost sum_k mayer_k X_{N,k}
  std::vector<int> fin_comp;
  bool free_tf = false;
  int scheme = OCP_SCHEME_TRAPEZOID;
  std::vector<double> mayer;
  // variable bounds reported by ocp_bounds (default -inf / +inf)
  std::vector<double> xlo, xhi, ulo, uhi;
  double tflo = 0, tfhi = 0;
  // path inequalities sum_v [a (z_v - b)^2 + l z_v] - r <= 0 (npath x (nx+nu), row-major)
  int npath = 0;
  std::vector<double> path_a, path_b, path_l, path_r;
  // boundary inequalities sum_v [a (z_v - b)^2 + l z_v] - r <= 0 on z = (X_0, X_N)
  // (nbin x 2 nx, row-major)
  int nbin = 0;
  std::vector<double> bin_a, bin_b, bin_l, bin_r;
  // boundary cost sum_v [a (z_v - b)^2 + l z_v] on z = (X_0, X_N) added to the objective (2 nx)
  bool has_bol = false;
  std::vector<double> bol_a, bol_b, bol_l;
  // device-resident parameters overriding params (or null): params[0] alone for the Van der Pol
  // binding, the model's whole dynamics-parameter vector for one call otherwise
  const double* p0_dev = nullptr;
  // time-varying state reference: xref_k + xslope_k t_j + xamp_k sin(xfreq_k t_j) for the
  // components trk_comp (ntrk of them), tabulated once per node in d_xtrack[(N+1) x ntrk]
  std::vector<double> xslope, xamp, xfreq;
  std::vector<int> trk_comp;
  int ntrk = 0;
  double* d_xtrack = nullptr;
  ocpg::Pattern pat;
  int device = 0, num_sms = 0;
  // device-resident pattern tables for the structure kernels
  int32_t* d_rowtmpl = nullptr;  // nx * RT_STRIDE ints: rx, ru, xv[RT_XV], uv[RT_UV]
  int64_t* d_jbase = nullptr;    // nx + 1
  int32_t* d_hent = nullptr;     // 2 * (hx + hu)
  int32_t* d_fin = nullptr;      // components of the final rows (nb - nx)
  int32_t* d_tcol = nullptr;     // tf-row columns (tx + tu local indices)
  int64_t* d_kcbase = nullptr;   // KKT slot bases of the defect rows (nx + 1)
  // path inequalities on the device: per row p the terms poff[p]..poff[p+1]-1 with variable
  // pv, coefficients pa, pb, pl; pr[p]; and the supports for the structure kernels
  int32_t* d_poff = nullptr;
  int32_t* d_pv = nullptr;
  double* d_pcoef = nullptr;     // pa, pb, pl of every term (3 per term), then pr (npath)
  int64_t* d_pbase = nullptr;    // jpbase (npath + 1) then kpbase (npath + 1)
  // boundary inequalities on the device: row q's terms boff[q]..boff[q+1]-1 with variable bv
  // (local index of z = (X_0, X_N)) and coefficients a, b, l; then r (nbin)
  int32_t* d_boff = nullptr;
  int32_t* d_bv = nullptr;
  double* d_bcoef = nullptr;
  int64_t* d_bbase = nullptr;    // jbbase (nbin + 1) then kbbase (nbin + 1)
  // scratch: per-CTA partial sums and the completion ticket of the last-block reduction
  double* d_partials = nullptr;
  unsigned* d_counter = nullptr;
  int max_partials = 0;
  // device mirrors, copy streams and events of ocp_eval_step_host (allocated on first use)
  ocpg::HostStep* hstep = nullptr;
  // the Jacobian's per-variable scatter map for ocp_jtprod_coo (built on first use, dropped
  // when the pattern is rebuilt)
  ocpg::ScatterMap* smap = nullptr;
  // set when a setter failed after it had started to rebuild the pattern or its device tables:
  // the handle is then inconsistent and every call but ocp_destroy / ocp_last_error refuses it
  bool unusable = false;
  std::string err;
};


namespace ocpg {

ocp_status set_err(ocp* h, ocp_status st, const std::string& msg);
// Refusal of a handle made unusable by a failed setter (OCP_EINVAL, message kept).
ocp_status unusable_err(const ocp* h);
// Device allocations and table uploads of the library (see fault.cu: host-side fault injection).
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) { return dev_malloc_raw(reinterpret_cast<void**>(p), bytes); }
cudaError_t dev_upload(void* dst, const void* src, size_t bytes);
bool fault_dims();      // the armed 'dims' fault fires here (once)
bool take_injected();   // whether the last failure on this thread was an injected one (clears it)
ocp_status cuda_err(ocp* h, cudaError_t e, const char* what);
int occupancy_grid(ocp* h, const void* kernel, int threads, size_t smem, int64_t work_tiles);

// Host pattern compiler.
bool build_pattern(ocp* h, std::string& why);
// Host part of ocp_create (validation, parameters, pattern); no device allocation.
ocp_status init_host(ocp* h, const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N, double T);

struct EvalCall {
  const double* x = nullptr;
  const double* y = nullptr;
  double sigma = 1.0;
  double *f = nullptr, *c = nullptr, *g = nullptr, *jv = nullptr, *hv = nullptr;
  // fused step only: directions and product outputs
  const double* vn = nullptr;  // length n: for J vn and H vn
  const double* vm = nullptr;  // length m: for J^T vm
  double *ojv = nullptr, *ojtv = nullptr, *ohv = nullptr;
  int64_t B = 0, E = 0;  // owned node range [B, E)
  bool range = false;    // f receives the partial sum of this range
};

enum ProdKind { P_JPROD = 0, P_JTPROD = 1, P_HPROD = 2 };
struct ProdCall {
  int kind = 0;
  const double* x = nullptr;
  const double* y = nullptr;
  double sigma = 1.0;
  const double* v = nullptr;
  double* out = nullptr;
  double* dmu = nullptr;  // jtprod: (dc/dp)^T v, one double per dynamics parameter (or null)
  // autograd extensions (Van der Pol): parameter-direction terms
  double pdir = 0.0;            // jprod: adds (dc/dp0) * pdir  (host scalar)
  const double* pdir_dev = nullptr;  // jprod: same with a device scalar
  const double* mixw = nullptr; // hprod: adds (d2 c / dp0 dx)^T mixw * mixs
  const double* mixs = nullptr; // device scalar
  // jtprod only: the nodes [B, E) whose entries are written (E < 0: every node); dmu then
  // receives the partial sum over these nodes
  int64_t B = 0, E = -1;
};

// Per-model dispatchers (node models: VDP, CARTPOLE, DINT, QUADROTOR; HEAT1D separate).
ocp_status node_eval_vdp(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status node_eval_cartpole(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status node_eval_dint(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status node_eval_quad(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status node_prod_vdp(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status node_prod_cartpole(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status node_prod_dint(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status node_prod_quad(ocp* h, const ProdCall& c, cudaStream_t s);
// Tabulate the time-varying state reference of the handle into h->d_xtrack.
ocp_status fill_tracking(ocp* h);
ocp_status goddard_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status goddard_prod(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status heat_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status heat_prod(ocp* h, const ProdCall& c, cudaStream_t s);
// The heat model's Jv (jp), J^T w (jt) and, unless hp is null, H v (hp) in one launch.
ocp_status heat_prod2(ocp* h, const ProdCall& jp, const ProdCall& jt, const ProdCall* hp, cudaStream_t s);

struct EvalCall;
ocp_status dispatch_eval(ocp* h, unsigned out, const EvalCall& c, void* stream);
// Tiles of the objective reduction for a problem of this model and horizon.
int64_t objective_tiles(int model, int64_t nodes);

ocp_status launch_jac_structure(const ocp* h, int32_t* rows, int32_t* cols, cudaStream_t s);
ocp_status launch_hess_structure(const ocp* h, int32_t* rows, int32_t* cols, cudaStream_t s);

// Max-template of the node Hessian for node models (see node_kernels.cuh) and the
// per-model Jacobian row templates, for the pattern compiler.
void model_row_templates(int model, int nx, std::vector<RowTemplate>& rows);
void model_hess_max_template(int model, int nx, std::vector<std::pair<int, int>>& ent,
                             std::vector<int>& is_dyn);

ocp_status obj_launch(ocp* h, bool hvp, const double* x, const double* s, const double* v, double* out,
                      double* dot, cudaStream_t st);

// Path inequalities: rows, Jacobian entries and the updates of H, J^T w and H v that belong
// to them, after the model's own kernel on the same stream (see path_kernels.cu).
ocp_status path_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status path_prod(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status path_upload(ocp* h);
// Boundary inequalities: their rows, Jacobian entries and the updates of H (nodes 0 and N),
// J^T w and H v, after the path rows' kernel on the same stream (see bineq_kernels.cu).
ocp_status bin_eval(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s);
ocp_status bin_prod(ocp* h, const ProdCall& c, cudaStream_t s);
ocp_status bin_upload(ocp* h);
// The boundary cost: its value, gradient and Hessian terms after the other kernels.
ocp_status bol_eval(ocp* h, const EvalCall& c, cudaStream_t s);
ocp_status bol_prod(ocp* h, const ProdCall& c, cudaStream_t s);
// Releases the scatter map (called on every pattern rebuild and by ocp_destroy).
void scatter_map_free(ocp* h);
// Releases what ocp_eval_step_host allocated (called by ocp_destroy).
void host_step_free(ocp* h);


}  // namespace ocpg
