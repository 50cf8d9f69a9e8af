// Pauli-sum energies for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: they run under a device-memory budget
// that a host framework has already reserved in full, or inside a loop that
// must never enter the allocator. tnmps_expect_pauli_sum_dev needs a
// caller-supplied workspace; this variant instead uses a scratch array that
// the library owns: a file-scope __device__ array of a fixed size, present on
// every GPU that loads the library until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address. The first call on each device, with that device current, asks
// the runtime for the real address (cudaGetSymbolAddress) and caches it;
// that call should therefore come before any stream capture. Every call
// shares the one array and leaves the previous call's contents in it, so the
// term plan is uploaded again on every call and nothing may rely on earlier
// contents; calls whose GPU work overlaps (other streams, other contexts)
// race on the array.
#include <mutex>

#include "tnmps_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[TNMPS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

tnmps_status expect_noalloc_impl(tnmps_ctx *c, const TermPlan &p, uint64_t gen,
                                 double *energy_dev, double *per_term_dev) {
  void *ws = nullptr;
  cudaError_t e = scratch_for_current_device(&ws);
  if (e != cudaSuccess) {
    c->last_error = std::string("no-alloc scratch address: ") + cudaGetErrorString(e);
    return TNMPS_ERR_CUDA;
  }
  const size_t need = expect_ws_bytes(c, p, 1);
  if (need > (size_t)TNMPS_NOALLOC_SCRATCH_BYTES) {
    c->last_error = "term set needs " + std::to_string(need) +
                    " bytes of scratch for one state; the no-alloc scratch holds " +
                    std::to_string((size_t)TNMPS_NOALLOC_SCRATCH_BYTES) + " bytes";
    return TNMPS_ERR_NOMEM;
  }
  // the shared array may hold another context's plan: always upload ours
  c->plan_terms = nullptr;
  c->plan_ws = nullptr;
  c->plan_gen = gen;
  e = expect_run(c, p, (char *)ws, (size_t)TNMPS_NOALLOC_SCRATCH_BYTES, 0, energy_dev,
                 per_term_dev, nullptr, nullptr);
  if (e != cudaSuccess) {
    c->last_error = std::string("no-alloc expectation: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TNMPS_ERR_NOMEM : TNMPS_ERR_CUDA;
  }
  return TNMPS_OK;
}
