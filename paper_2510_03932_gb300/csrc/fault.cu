// Host-side fault injection for testing the library's error paths (no GPU fault is involved).
//
// Every device allocation and every host-to-device table upload of the library goes through
// dev_malloc / dev_upload.  A fault specification, from the environment variable OCP_FAULT
// (read once, at the first allocation or upload) or from ocp_set_fault, makes one of them fail
// on the host, before any CUDA call is made:
//   alloc:K   the K-th dev_malloc from now returns cudaErrorMemoryAllocation (status OCP_ENOMEM)
//   upload:K  the K-th dev_upload from now returns cudaErrorInvalidValue (status OCP_ECUDA)
//   dims      the next pattern build reports that the problem does not fit the int32 ABI (OCP_EDIM)
// Each specification fires once and then disarms.  The status and message of the failing call
// name the injected fault; the handle or batch being built is released as on a real failure.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "ocp_internal.h"

namespace ocpg {
namespace {

enum FaultKind { F_NONE = 0, F_ALLOC = 1, F_UPLOAD = 2, F_DIMS = 3 };
std::mutex g_mu;
int g_kind = F_NONE;
long g_left = 0;
bool g_env_read = false;
thread_local bool g_injected = false;

bool parse(const char* spec, int& kind, long& k) {
  kind = F_NONE;
  k = 0;
  if (!spec || !*spec) return true;
  if (std::strcmp(spec, "dims") == 0) { kind = F_DIMS; k = 1; return true; }
  const char* colon = std::strchr(spec, ':');
  if (!colon) return false;
  const std::string what(spec, colon - spec);
  char* end = nullptr;
  const long n = std::strtol(colon + 1, &end, 10);
  if (!end || *end || n < 1) return false;
  if (what == "alloc") kind = F_ALLOC;
  else if (what == "upload") kind = F_UPLOAD;
  else return false;
  k = n;
  return true;
}

void read_env_locked() {
  if (g_env_read) return;
  g_env_read = true;
  int kind;
  long k;
  if (parse(std::getenv("OCP_FAULT"), kind, k)) { g_kind = kind; g_left = k; }
}

// True when this call is the one the armed fault of `kind` targets (and disarms it).
bool fire(int kind) {
  std::lock_guard<std::mutex> g(g_mu);
  read_env_locked();
  if (g_kind != kind) return false;
  if (--g_left > 0) return false;
  g_kind = F_NONE;
  g_injected = true;
  return true;
}

}  // namespace

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  if (fire(F_ALLOC)) { *p = nullptr; return cudaErrorMemoryAllocation; }
  return cudaMalloc(p, bytes);
}

cudaError_t dev_upload(void* dst, const void* src, size_t bytes) {
  if (fire(F_UPLOAD)) return cudaErrorInvalidValue;
  return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}

bool fault_dims() { return fire(F_DIMS); }

bool take_injected() {
  const bool v = g_injected;
  g_injected = false;
  return v;
}

}  // namespace ocpg

extern "C" ocp_status ocp_set_fault(const char* spec) {
  OCP_RANGE();
  int kind;
  long k;
  if (!ocpg::parse(spec, kind, k))
    return ocpg::set_err(nullptr, OCP_EINVAL, "ocp_set_fault: expected alloc:K, upload:K, dims or an empty string");
  std::lock_guard<std::mutex> g(ocpg::g_mu);
  ocpg::g_env_read = true;  // an explicit setting replaces the environment's
  ocpg::g_kind = kind;
  ocpg::g_left = k;
  ocpg::g_injected = false;
  return OCP_OK;
}
