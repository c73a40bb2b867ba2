/*
 * ocp.h — C-ABI of the GB300 (sm_103a) FP64 evaluator for trapezoidal direct transcriptions
 * of optimal control problems.
 *
 * The problem (paper, Sec. 3 and Sec. 5):  minimise  int_0^T f0(x(t), u(t)) dt  subject to
 * x' = f(x, u), x(0) = x0 (and optionally x(T) = xf), transcribed on the uniform grid
 * t_j = j h, h = T/N, j = 0..N, with the trapezoidal rule for both the dynamics and the cost.
 *
 * Unknown vector (length n = (nx+nu)(N+1); Sec. 3 unknowns, Sec. 5 variable layout):
 *     x = [ X_0, X_1, ..., X_N, U_0, U_1, ..., U_N ],   X_j in R^nx, U_j in R^nu,
 *   i.e. X_{j,k} at index k + nx*j and U_{j,i} at index nx*(N+1) + i + nu*j (0-based);
 *   with a free final time tf is appended (n grows by one, h = tf / N).
 * Constraints (length m = nb + nx*N, declaration order of Sec. 5):
 *     rows 0..nx-1         : X_{0,k}                (the expression; bounds are x0)
 *     rows nx..nb-1        : X_{N,k}                (final rows: every component, or those set
 *                                                   by ocp_set_final_components; nb = nx + count)
 *     row  nb + k*N + j    : (X_{j+1,k} - X_{j,k}) - h/2 (f_k(z_j) + f_k(z_{j+1})),  z_j = (X_j, U_j)
 *     then the path inequalities, if any (ocp_set_path_constraints)
 *     then the boundary inequalities, if any (ocp_set_boundary_inequalities)
 * Objective (Sec. 5 trapezoidal cost): F = sum_j w_j f0(z_j), w_0 = w_N = h/2, else w_j = h,
 *   plus the terminal cost (ocp_set_terminal_cost) and the boundary cost g(X_0, X_N)
 *   (ocp_set_boundary_cost), if set.
 * Lagrangian Hessian: H = sigma * Hess F + sum_r y_r Hess c_r (lower triangle stored).
 * Sparse matrices are COO, 0-based, one entry per structural nonzero (a derivative that is
 * not identically zero, whatever its value at x, y, sigma), sorted by (row, col).
 *
 * Conventions for every call below:
 *   - Array arguments of the evaluation calls are caller-owned, contiguous FP64 (or int32)
 *     DEVICE pointers; the handle owns only its pattern tables and a small scratch area.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  The status reports argument and launch errors only.
 *   - Calls on one handle must not overlap on the GPU (they share the handle's scratch);
 *     use one handle per concurrent stream.
 *   - No call aborts the process.  On failure the status is non-zero and
 *     ocp_last_error(handle) (or ocp_last_error(NULL) for ocp_create / ocp_batch_create)
 *     returns a message.
 */
#ifndef OCP_GB300_H
#define OCP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ocp ocp_t;             /* opaque; created by ocp_create, owned by the library */
typedef struct ocp_batch ocp_batch_t; /* opaque; many problems evaluated in one launch */

typedef enum {
  OCP_OK = 0,
  OCP_EINVAL = 1,   /* null or malformed argument, unaligned pointer */
  OCP_EDIM = 2,     /* dimensions disagree with the model, or a size does not fit int32 */
  OCP_ENOMEM = 3,   /* device or host allocation failed */
  OCP_ECUDA = 4,    /* a CUDA runtime call or kernel launch failed */
  OCP_EMODEL = 5,   /* unknown model, cost kind, or operation not provided for this model */
  OCP_ETIMEOUT = 6  /* a bounded device wait ran out (reserved; no current kernel waits) */
} ocp_status;

/* Models.  Parameters (params[], nparams):
 *   VDP      (nx=2, nu=1): mu.         x1' = x2,  x2' = mu (1 - x1^2) x2 - x1 + u
 *   CARTPOLE (nx=4, nu=1): mc, mp, l, g.  state (p, p', th, th'), th from the downward
 *            vertical, point-mass pole:  D = mc + mp sin^2 th,
 *            p''  = (u + mp sin th (l th'^2 + g cos th)) / D,
 *            th'' = (-u cos th - mp l th'^2 cos th sin th - (mc+mp) g sin th) / (l D)
 *   HEAT1D   (nx=ncell, nu=1): ncell.  x_k' = (x_{k-1} - 2 x_k + x_{k+1}) / dx^2 - x_k^3,
 *            dx = 1/ncell, ghost x_0 = u (Dirichlet control), x_{ncell+1} = x_ncell (Neumann)
 *   DINT     (nx=2, nu=1): none.       x1' = x2,  x2' = u   (the paper's Sec. 5 example)
 *   QUADROTOR (nx=9, nu=4): g.  The quadrotor of the paper's appendix: positions x1, x3, x5 with
 *            velocities x2, x4, x6, attitude angles x7, x8, x9, thrust u1, angle-rate inputs
 *            u2..u4 (ck = cos xk, sk = sin xk):
 *            x1' = x2, x3' = x4, x5' = x6,
 *            x2' = u1 (c7 s8 c9 + s7 s9),  x4' = u1 (c7 s8 s9 - s7 c9),  x6' = u1 c7 c8 - g,
 *            x7' = (u2 c7 + u3 s7) / c8,  x8' = u3 c7 - u2 s7,  x9' = (u2 c7 + u3 s7) tan x8 + u4.
 *            Values are finite for |x8| < pi/2; the kernels do not check the singularity.
 *   GODDARD  (nx=3, nu=1): Cd, beta, Tmax, b.  The Goddard rocket of the paper's appendix:
 *            state (r, v, m) = altitude, speed, mass; u = normalised thrust:
 *            r' = v,  v' = -Cd v^2 exp(-beta (r - 1)) / m - 1/r^2 + u Tmax / m,  m' = -b Tmax u.
 *            The objective is a terminal cost (ocp_set_terminal_cost; q and r must be zero);
 *            the final time may be free (ocp_set_free_final_time) and the final condition may
 *            cover part of the state (ocp_set_final_components).  Its kernels are dedicated
 *            (tf couples every node); node ranges, the batched form, the differentiation
 *            form and ocp_eval_obj_noalloc are not provided for it (OCP_EMODEL). */
enum {
  OCP_MODEL_VDP = 1,
  OCP_MODEL_CARTPOLE = 2,
  OCP_MODEL_HEAT1D = 3,
  OCP_MODEL_DINT = 4,
  OCP_MODEL_QUADROTOR = 5,
  OCP_MODEL_GODDARD = 6
};

/* Running cost kinds.  DIAG_QUADRATIC: f0 = sum_k q_k (x_k - xref_k)^2 + sum_i r_i (u_i - uref_i)^2.
 * q, r are required; xref, uref may be NULL (zero).  ocp_set_tracking makes the state reference
 * time-varying. */
enum { OCP_COST_DIAG_QUADRATIC = 0 };

/* One-step schemes of the transcription (paper Sec. 3 / Sec. 5). */
enum { OCP_SCHEME_TRAPEZOID = 0, OCP_SCHEME_EULER = 1 };

typedef struct { int model; const double* params; int nparams; } ocp_dynamics;
typedef struct { int kind; const double* q; const double* r; const double* xref; const double* uref; } ocp_cost;

/* Build a problem (Sec. 5, the generated model constructor: scheme = trapezoid, grid size N,
 * uniform grid).  Host pointers in `dyn` and `cost` are copied.  Runs the host pattern
 * compiler and uploads the pattern once.  Errors: OCP_EMODEL (unknown model or cost kind),
 * OCP_EDIM (nx/nu/nparams disagree with the model, N < 1, T <= 0, or n, m, nnz >= 2^31),
 * OCP_ENOMEM, OCP_ECUDA.  Binds to the current CUDA device. */
ocp_status ocp_create(const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N,
                      double T, ocp_t** out);
void ocp_destroy(ocp_t* h);

/* Boundary values (Sec. 5 boundary generator: lcon = ucon = x0).  Host pointers of length nx.
 * xf == NULL leaves the problem without final rows; a non-NULL xf adds the nx rows X_{N,k}
 * (this changes m and nnz_J; call it before asking for dimensions or structure).
 * x0 == NULL keeps zeros. */
ocp_status ocp_set_boundary(ocp_t* h, const double* x0, const double* xf);

/* Time-varying state reference (the quadrotor's tracking terms, paper appendix): the running
 * cost uses, at node time t_j = j h,
 *     xref_k(t_j) = xref_k + xslope_k t_j + xamp_k sin(xfreq_k t_j)
 * instead of the constant xref_k.  Host arrays of length nx; NULL means zeros; all three NULL
 * (or all coefficients zero) returns to the constant reference.  The values are tabulated once
 * on the device, (N+1) doubles per tracked component (a component is tracked when its slope is
 * non-zero, or its amplitude and frequency both are); the call synchronizes the device.  Only
 * F, its gradient and the objective kernels of the differentiation form depend on it (the
 * Hessian of the cost does not).  A batch created earlier from this handle keeps using the
 * table it saw: re-create the batch after changing the reference.  Errors: OCP_EMODEL for
 * HEAT1D, OCP_EINVAL for non-finite coefficients, OCP_ENOMEM / OCP_ECUDA. */
ocp_status ocp_set_tracking(ocp_t* h, const double* xslope, const double* xamp, const double* xfreq);

/* Scheme (paper Sec. 3: the transcription is parametrised by the one-step scheme).
 * OCP_SCHEME_TRAPEZOID (default): as described at the top of this file.
 * OCP_SCHEME_EULER: forward Euler,  defect (k, j) = (X_{j+1,k} - X_{j,k}) - h f_k(X_j, U_j),
 *   j = 0..N-1; cost sum_{j<N} h f0(z_j) (rectangle rule); the unknowns are X_0..X_N and
 *   U_0..U_{N-1} (n = nx (N+1) + nu N, U_j at nx (N+1) + nu j).  Row (k, j) lists its entries
 *   on X_j (the model's template, identity merged), then X_{j+1,k}, then U_j; the Hessian has
 *   the blocks of nodes 0..N-1 only (X rows of those nodes, then their U rows), built from the
 *   own rows' multipliers y_{k,j}.
 * Rebuilds the pattern.  Euler is provided for VDP, CARTPOLE, DINT and QUADROTOR (OCP_EMODEL
 * otherwise); node ranges, the batched form, the parameter derivatives and the objective
 * kernels of the differentiation form are provided for the trapezoidal scheme only. */
ocp_status ocp_set_scheme(ocp_t* h, int scheme);

/* Path inequalities (paper Sec. 3: c(X_i, U_i) <= 0, i over the nodes with a control), in the
 * quadratic-plus-linear family
 *     c_p(z) = sum_v [ a[p,v] (z_v - b[p,v])^2 + l[p,v] z_v ] - r[p] <= 0,   z = (x, u) of the node,
 * (half-spaces, bounds, ellipsoids, keep-out regions with a < 0).  Host arrays a, b, l of
 * npath x (nx+nu) (row-major) and r of npath; npath = 0 removes them (at most 16).  The rows
 * come after the defects: row nb + nx N + p nun + i (nun = N+1, or N for Euler), bounds
 * (-inf, 0] in ocp_bounds.  Row (p, i) has one Jacobian entry per variable with a or l non-zero
 * (columns ascending); the squared terms add 2 a y on the Hessian diagonal of node i (the
 * entry becomes structural if it was not).  Every evaluation and product includes them (a
 * kernel after the model's on the same stream).  Rebuilds the pattern.  Not in the batched
 * form.  Errors: OCP_EINVAL (bad counts, NULL or non-finite arrays, an empty row). */
ocp_status ocp_set_path_constraints(ocp_t* h, int npath, const double* a, const double* b, const double* l,
                                    const double* r);

/* Boundary inequalities (paper Sec. 3: b(X_0, X_N) <= 0) in the same family over the first
 * and the last state, z = (X_0, X_N) (2 nx variables: v < nx is X_{0,v}, nx + v is X_{N,v}):
 *     b_q(z) = sum_v [ a[q,v] (z_v - b[q,v])^2 + l[q,v] z_v ] - r[q] <= 0
 * (terminal sets, coupling of the start and the end).  Host arrays a, b, l of nbin x 2nx
 * (row-major) and r of nbin; nbin = 0 removes them (at most 16).  The rows come last: row
 * nb + nx N + npath nun + q, bounds (-inf, 0] in ocp_bounds.  Row q has one Jacobian entry per
 * variable with a or l non-zero, X_0 columns before X_N columns (slots after the path rows'
 * entries); a squared term on component k adds 2 a y_q to the (k, k) Hessian entry of node 0
 * or node N, and (k, k) becomes structural in every node's block (the node blocks share one
 * template; the entry is zero at the other nodes).  Every evaluation, product and the KKT
 * assembly include them (one small kernel after the model's and the path rows' on the same
 * stream).  Trapezoidal scheme only (OCP_EMODEL with Euler, here or in ocp_set_scheme); not in
 * node ranges or the batched form (OCP_EMODEL).  Rebuilds the pattern.  Errors: OCP_EINVAL (bad
 * count, NULL or non-finite arrays, a row without variables). */
ocp_status ocp_set_boundary_inequalities(ocp_t* h, int nbin, const double* a, const double* b, const double* l,
                                         const double* r);

/* Free final time (Goddard; paper appendix "tf in R, variable"): enable != 0 appends tf to the
 * unknowns (n grows by one, tf = x[n-1]) and the grid becomes t_j = j tf / N; T of ocp_create
 * is then unused.  Every defect row gains its tf entry -(f_k(z_j) + f_k(z_{j+1})) / (2N) as its
 * last (largest-column) entry; the Hessian gains the tf row (row n-1, after every other row)
 * with the entries -(1/(2N)) sum_k ybar_{j,k} df_k/dz_{j,v} on the state columns of every
 * node (node-major), then on the control columns (no (tf, tf) entry: c and F are linear in
 * tf).  J^T w and H v get their tf component as a deterministic sum over the nodes.
 * Rebuilds the pattern (n, nnz_J, nnz_H change).  Other models: OCP_EMODEL. */
ocp_status ocp_set_free_final_time(ocp_t* h, int enable);

/* Final rows on part of the state (Goddard: m(tf) = mf): rows nx..nx+count-1 are X_{N,comps[i]}
 * with bounds values[i]; comps ascending state indices (host arrays).  count == 0 removes the
 * final rows; count == nx is ocp_set_boundary's full final state.  Rebuilds the pattern.
 * Errors: OCP_EINVAL (bad indices), OCP_EMODEL (models other than Goddard: use
 * ocp_set_boundary). */
ocp_status ocp_set_final_components(ocp_t* h, int count, const int32_t* comps, const double* values);

/* Boundary cost (paper Sec. 3: the Bolza term g(X_0, X_N) of the objective), for every model:
 *     F += g(z) = sum_v [ a[v] (z_v - b[v])^2 + l[v] z_v ],   z = (X_0, X_N)
 * (terminal penalties, start-end couplings).  Host arrays a, b, l of 2 nx (v < nx is X_{0,v},
 * nx + v is X_{N,v}); all three NULL remove it.  The gradient gains dg/dz at X_0 and X_N; the
 * Hessian gains sigma 2 a[v] on the (k, k) entry of node 0 or node N, and (k, k) becomes
 * structural in every node's block (zero at the other nodes).  Every evaluation, hprod and the
 * KKT assembly include it (one small kernel after the others on the same stream).  With the
 * Euler scheme the X_N terms must be linear (node N has no Hessian block): OCP_EMODEL here or
 * in ocp_set_scheme otherwise.  Not in node ranges, the batched form or the objective-only
 * kernels of the differentiation form (OCP_EMODEL).  Rebuilds the pattern.  Errors: OCP_EINVAL
 * (some but not all arrays NULL, non-finite values). */
ocp_status ocp_set_boundary_cost(ocp_t* h, const double* a, const double* b, const double* l);

/* Terminal (Mayer) cost added to the objective: F += sum_k mayer_k X_{N,k} (host array of nx;
 * NULL removes it).  Goddard "r(tf) -> max" is mayer = (-1, 0, 0).  Other models: OCP_EMODEL. */
ocp_status ocp_set_terminal_cost(ocp_t* h, const double* mayer);

/* Variable bounds reported by ocp_bounds (host arrays of nx / nu, NULL = unbounded; tflo/tfhi
 * bound the free final time).  They do not enter any evaluation. */
ocp_status ocp_set_variable_bounds(ocp_t* h, const double* xlo, const double* xhi, const double* ulo,
                                   const double* uhi, double tflo, double tfhi);

/* Start point (the generated model's `init`, Sec. 5: one value per state and per control
 * component, repeated at every node): writes x (DEVICE array of n) with X_{j,k} = xs[k],
 * U_{j,i} = us[i] and, with a free final time, tf.  xs, us: host arrays of nx and nu (NULL:
 * zeros).  Asynchronous on `stream`.  Errors: OCP_EINVAL (NULL or misaligned x). */
ocp_status ocp_start_point(ocp_t* h, const double* xs, const double* us, double tf, double* x, void* stream);

/* Sizes: n variables, m constraints, Jacobian and (lower) Hessian nonzeros.  Host outputs. */
ocp_status ocp_dims(const ocp_t* h, int64_t* n, int64_t* m, int64_t* nnzj, int64_t* nnzh);

/* Bounds (HOST arrays): lvar/uvar = the variable bounds of ocp_set_variable_bounds (default
 * -inf/+inf; the free final time last), lcon = ucon = [x0; final values; 0 for every defect].
 * Any pointer may be NULL. */
ocp_status ocp_bounds(const ocp_t* h, double* lvar, double* uvar, double* lcon, double* ucon);

/* Objective F(x) (Sec. 5 trapezoidal cost) written to the device scalar f. */
ocp_status eval_obj(ocp_t* h, const double* x, double* f, void* stream);
/* Constraint vector c(x), length m (Sec. 5 boundary rows and trapezoidal defects). */
ocp_status eval_cons(ocp_t* h, const double* x, double* c, void* stream);
/* Gradient of F, length n. */
ocp_status eval_grad(ocp_t* h, const double* x, double* g, void* stream);

/* Jacobian of c: structure (int32 device arrays of length nnzj) and values (FP64, same order).
 * Row (k,j) holds, by increasing column, the entries on X_j, X_{j+1}, U_j, U_{j+1}. */
ocp_status jac_coo_structure(const ocp_t* h, int32_t* rows, int32_t* cols, void* stream);
ocp_status jac_coo_values(ocp_t* h, const double* x, double* vals, void* stream);

/* Lagrangian Hessian, lower triangle (row >= col): structure (length nnzh) and values for
 * multipliers y (length m, boundary rows first) and objective weight sigma.  H is block-
 * diagonal by node; the X rows of all nodes come first, then the U rows. */
ocp_status hess_coo_structure(const ocp_t* h, int32_t* rows, int32_t* cols, void* stream);
ocp_status hess_coo_values(ocp_t* h, const double* x, const double* y, double sigma, double* vals,
                           void* stream);

/* The Jacobian's per-variable scatter map: the COO of jac_coo_structure in column order (CSC
 * of the COO value array; the paper's Sec. 5 Jacobian of the generated constraints, viewed by
 * unknowns).  For column c, the entries t in colptr[c] .. colptr[c+1]-1 have row
 * rows[t] and value jvals[slots[t]], rows ascending.  colptr: int32 device array of n + 1;
 * rows, slots: int32 device arrays of nnz_J.  Built from the pattern compiler's per-variable
 * templates (for each unknown of a node, the rows and entry positions that reference it), one
 * thread per column, no sort.  Synchronizes `stream` (it uses temporary device memory).
 * Errors: OCP_EINVAL (NULL arrays), OCP_ENOMEM/OCP_ECUDA. */
ocp_status ocp_jac_scatter_map(ocp_t* h, int32_t* colptr, int32_t* rows, int32_t* slots, void* stream);

/* J^T w from STORED Jacobian values (the paper defines no products: this is the gather a
 * solver holding J values needs; jvals from jac_coo_values or ocp_eval_all, length nnz_J;
 * w of length m; Jtw of length n, device arrays): the gather over the scatter map, each
 * column's entries added in row order (deterministic); the free final time's column by one
 * CTA's fixed-order reduction.  The handle keeps the map (about 8 bytes per J entry, built on
 * the first call, synchronizing `stream` then; rebuilt after a pattern change).  jtprod
 * computes the same product without stored values (node-local, from x). */
ocp_status ocp_jtprod_coo(ocp_t* h, const double* jvals, const double* w, double* Jtw, void* stream);

/* Matrix-free products at x:  Jv (v: n -> m),  J^T v (v: m -> n),  H v (v: n -> n, full
 * symmetric H for multipliers y and weight sigma) of the Sec. 5 Jacobian and Lagrangian
 * Hessian (not formed: each node's derivatives are recomputed from x).  Output arrays must not
 * alias inputs. */
ocp_status jprod(ocp_t* h, const double* x, const double* v, double* Jv, void* stream);
ocp_status jtprod(ocp_t* h, const double* x, const double* v, double* Jtv, void* stream);
ocp_status hprod(ocp_t* h, const double* x, const double* y, double sigma, const double* v,
                 double* Hv, void* stream);

/* Everything one interior-point iteration needs, in one fused launch: f (device scalar), c,
 * g, Jacobian values and Hessian values.  Any output pointer may be NULL (not computed). */
ocp_status ocp_eval_all(ocp_t* h, const double* x, const double* y, double sigma, double* f,
                        double* c, double* g, double* jvals, double* hvals, void* stream);

/* The whole per-iteration evaluation in one pass over the nodes: everything of ocp_eval_all
 * plus the products Jv = J vn, Jtv = J^T vm and Hv = H(y, sigma) vn at the same x, sharing the
 * per-node derivative work and the loads of x and y (one launch for the node models; the heat
 * model runs two: its evaluation, then its three products in one).  vn has length n, vm length
 * m.  All arguments are
 * required.  Values are bit-identical to the separate calls. */
ocp_status ocp_eval_step(ocp_t* h, const double* x, const double* y, double sigma, const double* vn,
                         const double* vm, double* f, double* c, double* g, double* jvals,
                         double* hvals, double* Jv, double* Jtv, double* Hv, void* stream);

/* ocp_eval_step with every array in HOST memory (x, y, vn, vm read; f, c, g, jvals, hvals, Jv,
 * Jtv, Hv written, same lengths and layouts as ocp_eval_step; f is one double).  The handle
 * keeps two sets of device copies of all arrays (allocated on the first call and when the
 * dimensions change, about 16 (5n + 4m + nnz_J + nnz_H) bytes in all, freed by ocp_destroy) and
 * alternates between them: the inputs are copied in on an internal stream (once the call
 * before the previous one has copied its outputs out of that set), the step runs on `stream`,
 * the outputs are copied out on a second internal stream, and `stream` waits for that copy.
 * So consecutive calls on one stream overlap one call's input copy with the previous call's
 * output copy, and a call's outputs are complete when `stream` reaches its end (synchronize it
 * before reading them).  The input copy waits only for the handle's earlier calls, not for
 * other work on `stream`: the host inputs must be ready when the call is made, and must not
 * change before the call's work on `stream` is complete.  Host arrays should be page-locked (pinned)
 * for asynchronous copies; pageable memory works but the copies then block the calling
 * thread.  Results are bit-identical to ocp_eval_step.  Calls on one handle must be ordered on
 * one stream (they share the device copies).  All pointers are required and 8-byte aligned
 * (OCP_EINVAL otherwise). */
ocp_status ocp_eval_step_host(ocp_t* h, const double* x, const double* y, double sigma, const double* vn,
                              const double* vm, double* f, double* c, double* g, double* jvals,
                              double* hvals, double* Jv, double* Jtv, double* Hv, void* stream);

/* ocp_eval_step_host without the last wait: `stream` does NOT wait for this call's output copy,
 * so the next call's step can run while these outputs are still being copied to the host (the
 * handle's two sets of device copies keep the calls apart).  The outputs are complete once
 * ocp_host_step_wait(h, stream) has been called after the last such call and `stream` has
 * reached that point; until then they must not be read, and an output array must not be handed
 * to a call that is not ordered after this one by that wait or by the handle (calls on one
 * handle write their outputs in call order).  Inputs, ordering and errors as
 * ocp_eval_step_host; results bit-identical to ocp_eval_step. */
ocp_status ocp_eval_step_host_async(ocp_t* h, const double* x, const double* y, double sigma,
                                    const double* vn, const double* vm, double* f, double* c, double* g,
                                    double* jvals, double* hvals, double* Jv, double* Jtv, double* Hv,
                                    void* stream);

/* Make `stream` wait for the output copies of every earlier ocp_eval_step_host(_async) call on
 * this handle (nothing to wait for: returns OCP_OK).  OCP_EINVAL for a NULL handle. */
ocp_status ocp_host_step_wait(ocp_t* h, void* stream);

/* KKT matrix of the interior-point step (paper Sec. 6: the solver assembles the KKT system in
 * device buffers from the derivative values), lower triangle, COO sorted by (row, col):
 *     K = [ H + diag(sigma_x + delta_w)                ]    size (n + m) x (n + m)
 *         [ J                          -delta_c I      ]
 * with H and J the values of hess_coo_values and jac_coo_values (same x, y, sigma).  Every
 * row ends with its diagonal entry (added to the (1,1) block where H has none).
 * ocp_kkt_dims: the number of entries (host; OCP_EDIM when it does not fit int32).
 * ocp_kkt_structure: rows and cols (int32 device arrays of length nnzk).
 * ocp_kkt_values: kvals (device, length nnzk) from hvals (nnz_H) and jvals (nnz_J); sigma_x
 *   (device, length n) may be NULL (zero); delta_w, delta_c are the regularisation scalars. */
ocp_status ocp_kkt_dims(const ocp_t* h, int64_t* nnzk);
ocp_status ocp_kkt_structure(ocp_t* h, int32_t* rows, int32_t* cols, void* stream);
ocp_status ocp_kkt_values(ocp_t* h, const double* hvals, const double* jvals, const double* sigma_x,
                          double delta_w, double delta_c, double* kvals, void* stream);

/* Parameter derivative for the Van der Pol model (mu = params[0]):
 *   dmu = (dc/dmu)^T w   (device scalar), together with J^T w into Jtw (both required).
 * Other models: OCP_EMODEL (ocp_vjp_params covers every model with dynamics parameters). */
ocp_status ocp_vjp_param(ocp_t* h, const double* x, const double* w, double* Jtw, double* dmu,
                         void* stream);

/* eval_cons and ocp_vjp_param with params[0] (Van der Pol mu) read from the device scalar p0
 * for this call only (NULL: the handle's current value or binding): one call each for the
 * forward and backward of the differentiation form, c(x; mu) and (J^T w, (dc/dmu)^T w), with
 * mu a device tensor.  Other models: OCP_EMODEL when p0 is given (ocp_vjp_param_p: always). */
ocp_status ocp_eval_cons_p(ocp_t* h, const double* x, const double* p0, double* c, void* stream);
ocp_status ocp_vjp_param_p(ocp_t* h, const double* x, const double* w, const double* p0, double* Jtw,
                           double* dmu, void* stream);

/* Derivatives in every dynamics parameter (paper Sec. 3: the dynamics f(x, u; p) enter the
 * constraints only through the defect rows, Sec. 5 trapezoidal defects, so
 *   dc_{k,j}/dp = -h (df_k/dp(z_j) + df_k/dp(z_{j+1})) / 2 ).
 * The parameters with a derivative, in the order of ocp_dynamics.params:
 *   Van der Pol (mu); cart-pole (m_c, m_p, l, g); Goddard (Cd, beta, Tmax, b); quadrotor (g).
 * The double integrator has none and the heat model's parameter (its cell count) is structural.
 * ocp_param_count: *np = the number of those parameters for the handle's model (0, 1 or 4).
 * ocp_set_params: replace all of them (np = that count, host values, finite) without
 *   rebuilding the pattern; OCP_EDIM for another count, OCP_EMODEL when the count is 0.
 * ocp_eval_cons_params: c(x; p) with p read from device memory (np doubles) for this call only
 *   (NULL: the handle's values, or the Van der Pol binding of ocp_bind_param0).
 * ocp_vjp_params: J^T w into Jtw (length n) and dp = (dc/dp)^T w (device, np doubles, each a
 *   fixed-order sum over the nodes: deterministic), with p as in ocp_eval_cons_params.
 * Trapezoidal scheme only for ocp_vjp_params (OCP_EMODEL under forward Euler); models with
 * np = 0 return OCP_EMODEL when p or dp is given.  All pointers 8-byte aligned; the call
 * is asynchronous on `stream` and reads p when its kernels run. */
ocp_status ocp_param_count(const ocp_t* h, int* np);
/* ocp_bind_params: later calls on this handle read all np dynamics parameters from device
 * memory p_dev (NULL unbinds; the memory must stay valid while bound).  Van der Pol: every call
 * (as ocp_bind_param0).  The other models, trapezoidal scheme: the constraints (eval_cons,
 * ocp_eval_cons_params), J v, J^T w (with ocp_vjp_params) and H v; their other calls return
 * OCP_EMODEL while bound (under forward Euler: the constraints only). */
ocp_status ocp_bind_params(ocp_t* h, const double* p_dev);
ocp_status ocp_set_params(ocp_t* h, const double* p, int np);
ocp_status ocp_eval_cons_params(ocp_t* h, const double* x, const double* p, double* c, void* stream);
ocp_status ocp_vjp_params(ocp_t* h, const double* x, const double* w, const double* p, double* Jtw, double* dp,
                          void* stream);

/* Set the value of params[0] (e.g. Van der Pol mu) without rebuilding the pattern. */
ocp_status ocp_set_param0(ocp_t* h, double value);

/* Differentiation support (the autograd form; Van der Pol parameter mu = params[0]).
 * ocp_bind_param0: later calls on this handle read mu from the device scalar p0_dev (NULL
 *   unbinds and returns to the host value); the pointer must stay valid while bound.
 * ocp_jprod_param: Jv = J v + (dc/dmu) s, with s a device scalar (NULL: plain jprod).
 * ocp_hprod_param: Hv = (sigma Hess F + sum_r y_r Hess c_r) v + s sum_r y_r d2 c_r/dmu dx, and
 *   dmu = (sum_r y_r d2 c_r / dx dmu) . v (device scalar, NULL: not computed; needs s).
 *   s == NULL: plain hprod.  These are the second-order terms of the constraint adjoint.
 * ocp_eval_grad_scaled: g = s grad F(x), s a device scalar (the upstream gradient).
 * ocp_obj_hvp: Hv = s Hess F(x) v, and dot = grad F(x) . v (device scalar, may be NULL).
 * Models without a parameter derivative return OCP_EMODEL when s or p0_dev is given. */
ocp_status ocp_bind_param0(ocp_t* h, const double* p0_dev);
ocp_status ocp_jprod_param(ocp_t* h, const double* x, const double* v, const double* s, double* Jv, void* stream);
ocp_status ocp_hprod_param(ocp_t* h, const double* x, const double* y, double sigma, const double* v,
                           const double* s, double* Hv, double* dmu, void* stream);
ocp_status ocp_eval_grad_scaled(ocp_t* h, const double* x, const double* s, double* g, void* stream);
ocp_status ocp_obj_hvp(ocp_t* h, const double* x, const double* s, const double* v, double* Hv, double* dot,
                       void* stream);

/* Evaluate only the nodes [node_begin, node_end) (and the defect rows j in that range) of
 * eval_all, writing into the full-size output arrays.  Used to split one problem into
 * contiguous node shards (each shard reads a one-node halo of x and y).  f receives this
 * shard's partial objective.  Boundary rows are written by the shards that own node 0 / N. */
ocp_status ocp_eval_all_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x,
                              const double* y, double sigma, double* f, double* c, double* g,
                              double* jvals, double* hvals, void* stream);

/* The fused step (ocp_eval_step) on the nodes [node_begin, node_end) only: one contiguous
 * node shard of a problem split over several devices (the paper's Discussion, Sec. 8, names
 * multi-GPU execution as a future extension; every node's terms are independent given its
 * neighbours, Sec. 3).  The
 * arrays are the full-size arrays of ocp_eval_step in the global layout; the call writes the
 * outputs the shard owns: c, J values and Jv on the defect rows j in [node_begin,
 * min(node_end, N)) (and the boundary rows of node 0 / node N if the shard holds them), g,
 * H values, J^T w and Hv on its nodes, and f = the shard's partial objective (the sum over
 * its nodes of w_j f0(z_j)).  It reads x and vn on the nodes node_begin..min(node_end, N) (a
 * one-node halo on the right) and y and vm on the defect rows node_begin-1..node_end-1 (the
 * row to its left), plus the boundary rows it writes.  The objective of the whole problem is
 * the sum of the shards' partials (added in rank order for a deterministic result).
 * Node models (Van der Pol, cart-pole, double integrator, quadrotor), trapezoidal scheme,
 * path inequalities allowed; boundary inequalities, a boundary cost, the Goddard and heat
 * models and the Euler scheme return OCP_EMODEL; an empty or out-of-range node range OCP_EDIM. */
ocp_status ocp_eval_step_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x,
                               const double* y, double sigma, const double* vn, const double* vm,
                               double* f, double* c, double* g, double* jvals, double* hvals,
                               double* Jv, double* Jtv, double* Hv, void* stream);

/* ocp_vjp_param on the nodes [node_begin, node_end) only: J^T w on those nodes' entries of Jtw
 * and dmu = their share of (dc/dmu)^T w (the shards' shares add up to the whole product).
 * Reads x on the nodes of the range and w on the defect rows node_begin-1..node_end-1 and the
 * boundary rows of the nodes it holds.  Van der Pol only; the same restrictions and errors as
 * ocp_eval_step_range. */
ocp_status ocp_vjp_param_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x,
                               const double* w, double* Jtw, double* dmu, void* stream);

/* ocp_vjp_params on the nodes [node_begin, node_end) only: J^T w on those nodes' entries of Jtw
 * and dp = their shares of (dc/dp)^T w (np doubles; the shards' shares add up to the whole
 * product), with p as in ocp_vjp_params (device parameters, NULL: the handle's).  The node
 * models with parameters (Van der Pol, cart-pole, quadrotor); otherwise the restrictions and
 * errors of ocp_eval_step_range, and OCP_EMODEL for a model without parameters. */
ocp_status ocp_vjp_params_range(ocp_t* h, int64_t node_begin, int64_t node_end, const double* x, const double* w,
                                const double* p, double* Jtw, double* dp, void* stream);

/* out = parts[0] + parts[1] + ... + parts[count-1], added in index order (device arrays; one
 * thread): the rank-ordered combination of the shards' partial sums of ocp_eval_step_range,
 * ocp_vjp_param_range and ocp_vjp_params_range, which gives every rank the same bits.  Errors: OCP_EINVAL, OCP_ECUDA
 * (ocp_last_error(NULL)). */
ocp_status ocp_sum_ordered(const double* parts, int count, double* out, void* stream);

/* Layout of the COO values (host query): nb boundary rows; row_count[k] (nx entries) values per
 * defect row of component k, whose N rows are consecutive from the slot of component k-1's last
 * row (the boundary rows' nb values first); hx and hu values per node in the Hessian's X block
 * (node-major, first) and U block. */
ocp_status ocp_value_layout(const ocp_t* h, int64_t* nb, int32_t* row_count, int32_t* hx, int32_t* hu);

/* Objective F(x) without any device allocation, for callers that cannot call cudaMalloc at
 * evaluation time: a real-time control loop that must not allocate after start-up (cudaMalloc
 * can synchronize the device and its latency is unbounded), or a framework whose allocator
 * owns all device memory.  The paper has no counterpart: its evaluator owns its buffers.
 * Arguments: the problem description of ocp_create (host pointers, copied) instead of a handle;
 * x (length (nx+nu)(N+1)) and f (one double) are device pointers, as in eval_obj; the call is
 * asynchronous on `stream`.  The reduction scratch is a file-scope device array of 65536
 * tiles (about 512 KB on every device that loads the library, held until the process exits);
 * a horizon needing more tiles (N+1 above 65536 x 255 nodes for Van der Pol and the double
 * integrator, x 127 for the cart-pole and the quadrotor, x 31 for the heat model; the
 * constant reference only) returns OCP_EDIM without
 * launching.  The first call on a device looks up the array's device address with that device
 * current (and caches it for the life of the process); make that first call before any stream
 * capture.  CUDA loads the library's kernels lazily by default, so the first call of each model
 * on a device also makes the driver load them, which allocates device memory inside the
 * driver: a caller that must not allocate after start-up makes one warm-up call per model and
 * device at start-up (or sets CUDA_MODULE_LOADING=EAGER).  After cudaDeviceReset the cached
 * address is stale: do not call this entry point in a process that has reset a device it used
 * it on.  Every call on a device shares the
 * array and the last call's contents stay in it: calls that overlap on the GPU race.  Errors
 * as ocp_create and eval_obj, reported by ocp_last_error(NULL).  Calls neither cudaMalloc nor
 * cudaFree. */
ocp_status ocp_eval_obj_noalloc(const ocp_dynamics* dyn, const ocp_cost* cost, int nx, int nu, int64_t N,
                                double T, const double* x, double* f, void* stream);

/* Host-side fault injection, for testing the error paths of callers and of the library (the
 * paper has no counterpart).  spec: "alloc:K" makes the K-th device allocation of the library
 * from now on fail (the call reports OCP_ENOMEM), "upload:K" the K-th host-to-device upload of
 * its tables (OCP_ECUDA), "dims" the next pattern build (OCP_EDIM, as for a problem too large
 * for the int32 ABI); "" disarms.  The failure is made on the host before any CUDA call; each
 * specification fires once.  The environment variable OCP_FAULT with the same syntax arms a
 * fault at the library's first allocation or upload.  The failing call's message ends with
 * "(injected by OCP_FAULT)".  A handle being created is released; a setter that fails after it
 * has started to rebuild the pattern leaves the handle unusable: every later call on it but
 * ocp_destroy and ocp_last_error returns OCP_EINVAL.  Errors: OCP_EINVAL for a bad spec. */
ocp_status ocp_set_fault(const char* spec);

/* Message of the last failure on this handle (NULL: of the last failed create). */
const char* ocp_last_error(const ocp_t* h);

/* Batched form (many problems of one model, possibly different N, cost weights and boundary
 * values, in ONE persistent launch).  Provided for the Van der Pol, cart-pole, double-integrator
 * and quadrotor models (trapezoidal scheme, without path or boundary inequalities or a boundary
 * cost); others return OCP_EMODEL.  The handles must stay alive while the batch is used.
 * Variables, constraints, Jacobian and Hessian values of instance i start at the prefix
 * offsets given by ocp_batch_offsets (host arrays of length count+1 for x/g, y/c, jac values,
 * hess values), each instance laid out exactly as for its own handle: its slices are
 * bit-identical to the plain evaluator's; its objective goes to f[i] (device, length count).
 * Any output may be NULL (not stored); y is required with Hessian values.
 * Launch configuration: threads per CTA (64, 128, 256), nodes per thread (1 or 2: 32 or 64
 * nodes per warp), CTAs per SM of the persistent grid (0: as many as fit).  The quadrotor's
 * staged Jacobian rows allow at most 128 nodes per CTA (threads x nodes per thread); a larger
 * configuration returns OCP_EINVAL and the autotuner skips it.
 * ocp_batch_autotune times every configuration on the caller's data (synchronizes the
 * stream) and keeps the fastest; best_ms (host, may be NULL) receives its time.  With the
 * environment variable OCP_AUTOTUNE_CACHE naming a file, the result is appended to it, keyed
 * by the batch's shape (model, instance count, total and largest horizon, requested outputs)
 * and the GPU (SM count, compute capability); a later autotune of a batch of the same shape
 * takes the stored configuration and time without timing anything.
 * ocp_batch_graph_capture records one ocp_batch_eval_all launch with these arguments in a
 * CUDA graph (stream must be a created stream, not the legacy default one);
 * ocp_batch_graph_launch replays it.  Changing the configuration drops the graph. */
ocp_status ocp_batch_create(ocp_t* const* items, int count, ocp_batch_t** out);
void ocp_batch_destroy(ocp_batch_t* b);
ocp_status ocp_batch_offsets(const ocp_batch_t* b, int64_t* xoff, int64_t* coff, int64_t* joff,
                             int64_t* hoff);
ocp_status ocp_batch_set_config(ocp_batch_t* b, int nodes_per_thread, int threads, int ctas_per_sm);
ocp_status ocp_batch_get_config(const ocp_batch_t* b, int* nodes_per_thread, int* threads, int* ctas_per_sm);
ocp_status ocp_batch_eval_all(ocp_batch_t* b, const double* x, const double* y, double sigma,
                              double* f, double* c, double* g, double* jvals, double* hvals, void* stream);
ocp_status ocp_batch_autotune(ocp_batch_t* b, const double* x, const double* y, double sigma,
                              double* f, double* c, double* g, double* jvals, double* hvals,
                              void* stream, double* best_ms);
ocp_status ocp_batch_graph_capture(ocp_batch_t* b, const double* x, const double* y, double sigma,
                                   double* f, double* c, double* g, double* jvals, double* hvals,
                                   void* stream);
ocp_status ocp_batch_graph_launch(ocp_batch_t* b, void* stream);
const char* ocp_batch_last_error(const ocp_batch_t* b);

#ifdef __cplusplus
}
#endif
#endif /* OCP_GB300_H */
