// ocp_eval_step_host: the fused step of ocp_eval_step with every input and output in host
// memory.  The library keeps two sets of device mirrors of the arrays (allocated on the first
// call and whenever the problem's dimensions change) and alternates between them: call k
// copies its four inputs into set k mod 2 on its host-to-device stream (after the copy-out of
// call k-2, which used that set, has finished), runs ocp_eval_step on the caller's stream,
// copies the eight outputs out on its device-to-host stream, and makes the caller's stream
// wait for that copy-out.  Consecutive calls on one stream therefore overlap the input copy of
// call k+1 with the output copy of call k (the host link carries both directions at once),
// while each call's outputs are complete when the caller's stream reaches its end.  Each array
// moves in one copy: a pipeline over node ranges within one call (inputs of one range in
// flight while the previous one is evaluated and the one before it copied out) measured
// 1.73-2.02 ms per step at Van der Pol N = 1e6 with 2 to 16 ranges, against 1.64 ms for whole
// arrays (the extra copies and waits cost more than the partial overlap they bought).
// ocp_eval_step_host_async leaves out the caller's wait for the copy-out, so the next call's step
// runs while this call's outputs are still crossing the host link; ocp_host_step_wait joins
// the copies later.
#include <cstring>

#include "ocp_internal.h"

namespace ocpg {

struct HostStep {
  int64_t n = 0, m = 0, nnzj = 0, nnzh = 0;
  double* buf[2] = {};          // one allocation per set of mirrors
  double* arr[2][12] = {};      // x, y, vn, vm, f, c, g, jvals, hvals, Jv, Jtv, Hv
  int next = 0;                 // the set the next call uses
  cudaStream_t sh = nullptr, sd = nullptr;  // host-to-device and device-to-host copy streams
  cudaEvent_t in[2] = {}, comp[2] = {}, done[2] = {};
};

void host_step_free(ocp* h) {
  HostStep* s = h ? h->hstep : nullptr;
  if (!s) return;
  // copies of earlier calls may still read the mirrors or write the caller's host arrays
  if (s->sd) cudaStreamSynchronize(s->sd);
  if (s->sh) cudaStreamSynchronize(s->sh);
  for (int b = 0; b < 2; ++b) {
    cudaFree(s->buf[b]);
    for (cudaEvent_t e : {s->in[b], s->comp[b], s->done[b]})
      if (e) cudaEventDestroy(e);
  }
  if (s->sh) cudaStreamDestroy(s->sh);
  if (s->sd) cudaStreamDestroy(s->sd);
  delete s;
  h->hstep = nullptr;
}

// Lengths of the twelve arrays of the step, in the order of HostStep::arr.
static void step_sizes(const Pattern& P, int64_t (&sz)[12]) {
  const int64_t v[12] = {P.n, P.m, P.n, P.m, 1, P.m, P.n, P.nnzj, P.nnzh, P.m, P.n, P.n};
  for (int i = 0; i < 12; ++i) sz[i] = v[i];
}

// Streams, events and both sets of mirrors for the handle's current dimensions.
static ocp_status host_step_ready(ocp* h) {
  const Pattern& P = h->pat;
  HostStep* s = h->hstep;
  if (s && s->buf[0] && s->buf[1] && s->n == P.n && s->m == P.m && s->nnzj == P.nnzj && s->nnzh == P.nnzh)
    return OCP_OK;
  if (!s) {
    s = new HostStep();
    h->hstep = s;
    cudaError_t e = cudaStreamCreateWithFlags(&s->sh, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->sd, cudaStreamNonBlocking);
    for (int b = 0; b < 2; ++b)
      for (cudaEvent_t* ev : {&s->in[b], &s->comp[b], &s->done[b]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      host_step_free(h);
      return cuda_err(h, e, "host step streams and events");
    }
  } else {
    // earlier calls may still be copying from the old mirrors
    cudaError_t e = cudaStreamSynchronize(s->sd);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->sh);
    if (e != cudaSuccess) return cuda_err(h, e, "host step: wait before resizing");
  }
  for (int b = 0; b < 2; ++b) {
    cudaFree(s->buf[b]);
    s->buf[b] = nullptr;
  }
  s->n = s->m = s->nnzj = s->nnzh = 0;
  int64_t sz[12], total = 0;
  step_sizes(P, sz);
  auto up = [](int64_t k) { return (k + 31) / 32 * 32; };  // each mirror on a 256-byte boundary
  for (int64_t k : sz) total += up(k);
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = ocpg::dev_malloc(&s->buf[b], sizeof(double) * (size_t)total);
    if (e != cudaSuccess) {
      s->buf[b] = nullptr;
      return cuda_err(h, e, "cudaMalloc(host step mirrors)");
    }
    double* p = s->buf[b];
    for (int i = 0; i < 12; ++i) {
      s->arr[b][i] = p;
      p += up(sz[i]);
    }
  }
  s->n = P.n; s->m = P.m; s->nnzj = P.nnzj; s->nnzh = P.nnzh;
  return OCP_OK;
}

}  // namespace ocpg

using namespace ocpg;

// One host step; with `join` the caller's stream waits for the copy-out of this call.
static ocp_status host_step_run(ocp_t* h, const double* x, const double* y, double sigma, const double* vn,
                                const double* vm, double* f, double* cv, double* g, double* jvals,
                                double* hvals, double* Jv, double* Jtv, double* Hv, void* stream, bool join) {
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  const double* in[4] = {x, y, vn, vm};
  double* out[8] = {f, cv, g, jvals, hvals, Jv, Jtv, Hv};
  const char* names[12] = {"x", "y", "vn", "vm", "f", "c", "g", "jvals", "hvals", "Jv", "Jtv", "Hv"};
  for (int i = 0; i < 12; ++i) {
    const void* p = i < 4 ? (const void*)in[i] : (const void*)out[i - 4];
    if (!p) return set_err(h, OCP_EINVAL, std::string(names[i]) + " is NULL");
    if (reinterpret_cast<uintptr_t>(p) % 8) return set_err(h, OCP_EINVAL, std::string(names[i]) + " is not 8-byte aligned");
  }
  ocp_status st = host_step_ready(h);
  if (st != OCP_OK) return st;
  HostStep* S = h->hstep;
  const int b = S->next;
  double* const* A = S->arr[b];
  int64_t sz[12];
  step_sizes(h->pat, sz);
  cudaStream_t s0 = (cudaStream_t)stream;
  // inputs into this call's set, once the call that used it last has copied its outputs out
  cudaError_t e = cudaStreamWaitEvent(S->sh, S->done[b], 0);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(A[i], in[i], sizeof(double) * (size_t)sz[i], cudaMemcpyHostToDevice, S->sh);
  if (e == cudaSuccess) e = cudaEventRecord(S->in[b], S->sh);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, S->in[b], 0);
  if (e != cudaSuccess) return cuda_err(h, e, "host step: inputs");
  st = ocp_eval_step(h, A[0], A[1], sigma, A[2], A[3], A[4], A[5], A[6], A[7], A[8], A[9], A[10], A[11], s0);
  if (st != OCP_OK) return st;
  e = cudaEventRecord(S->comp[b], s0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(S->sd, S->comp[b], 0);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(out[i], A[4 + i], sizeof(double) * (size_t)sz[4 + i], cudaMemcpyDeviceToHost, S->sd);
  if (e == cudaSuccess) e = cudaEventRecord(S->done[b], S->sd);
  if (e == cudaSuccess && join) e = cudaStreamWaitEvent(s0, S->done[b], 0);
  if (e != cudaSuccess) return cuda_err(h, e, "host step: outputs");
  S->next = b ^ 1;
  return OCP_OK;
}

extern "C" ocp_status ocp_eval_step_host(ocp_t* h, const double* x, const double* y, double sigma,
                                         const double* vn, const double* vm, double* f, double* cv, double* g,
                                         double* jvals, double* hvals, double* Jv, double* Jtv, double* Hv,
                                         void* stream) {
  OCP_RANGE();
  return host_step_run(h, x, y, sigma, vn, vm, f, cv, g, jvals, hvals, Jv, Jtv, Hv, stream, true);
}

extern "C" ocp_status ocp_eval_step_host_async(ocp_t* h, const double* x, const double* y, double sigma,
                                               const double* vn, const double* vm, double* f, double* cv,
                                               double* g, double* jvals, double* hvals, double* Jv, double* Jtv,
                                               double* Hv, void* stream) {
  OCP_RANGE();
  return host_step_run(h, x, y, sigma, vn, vm, f, cv, g, jvals, hvals, Jv, Jtv, Hv, stream, false);
}

extern "C" ocp_status ocp_host_step_wait(ocp_t* h, void* stream) {
  OCP_RANGE();
  if (!h) return OCP_EINVAL;
  if (h->unusable) return unusable_err(h);
  HostStep* S = h->hstep;
  if (!S) return OCP_OK;
  // the copy-out stream is serial, so its last recorded event covers every earlier copy; an
  // event never recorded counts as complete
  cudaError_t e = cudaStreamWaitEvent((cudaStream_t)stream, S->done[S->next ^ 1], 0);
  if (e != cudaSuccess) return cuda_err(h, e, "host step: wait");
  return OCP_OK;
}
