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
// the runtime for the real address (cudaGetSymbolAddress) and caches it
// together with the CUDA context it belongs to; a call made in another
// context (after a cudaDeviceReset, or from a non-primary context) looks the
// address up again. The first call should therefore come before any stream
// capture.
//
// Every call shares the one array, which keeps the last call's contents. The
// term plan (trie, coefficients, geometry) at the start of the array is
// uploaded only when the array last held another context's or another term
// set's plan: that upload copies from host memory and synchronises the
// context's stream; a repeated call with the same context and term set only
// enqueues kernels. Calls whose GPU work overlaps (other streams, other
// contexts, other host threads) race on the array.
#include <cuda.h>

#include <mutex>

#include "tnmps_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[TNMPS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);

struct DeviceScratch {
  void *ptr = nullptr;          // device address of g_noalloc_scratch
  CUcontext ctx = nullptr;      // context the address belongs to
  uint64_t plan_ctx = 0;        // tnmps context (uid) whose plan the array holds
  uint64_t plan_gen = 0;        // ... and its term set's generation (0: none)
};

std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

CUcontext current_context() {
  static CtxGetCurrentFn fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  CUcontext ctx = nullptr;
  if (fn) fn(&ctx);
  return ctx;
}

// device index and cached scratch address for the current device (g_mu held)
cudaError_t scratch_for_current_device(int *dev_out, void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  DeviceScratch &d = g_dev[dev];
  const CUcontext ctx = current_context();
  if (!d.ptr || d.ctx != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    d = DeviceScratch{};
    d.ptr = p;
    d.ctx = ctx;
  }
  *dev_out = dev;
  *out = d.ptr;
  return cudaSuccess;
}

}  // namespace

tnmps_status expect_noalloc_impl(tnmps_ctx *c, const TermPlan &p, uint64_t gen,
                                 double *energy_dev, double *per_term_dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  void *ws = nullptr;
  int dev = 0;
  cudaError_t e = scratch_for_current_device(&dev, &ws);
  if (e != cudaSuccess) {
    c->last_error = std::string("no-alloc scratch address: ") + cudaGetErrorString(e);
    return TNMPS_ERR_CUDA;
  }
  // result regions only where the caller gives no output (energy_dev is required)
  const size_t need = expect_ws_bytes(c, p, 1, per_term_dev == nullptr, energy_dev == nullptr);
  if (need > (size_t)TNMPS_NOALLOC_SCRATCH_BYTES) {
    c->last_error = "term set needs " + std::to_string(need) +
                    " bytes of scratch for one state; the no-alloc scratch holds " +
                    std::to_string((size_t)TNMPS_NOALLOC_SCRATCH_BYTES) + " bytes";
    return TNMPS_ERR_NOMEM;
  }
  // the array holds this context's plan for this term set only if the last
  // call that wrote it was ours with the same terms
  DeviceScratch &d = g_dev[dev];
  const bool resident = d.plan_ctx == c->uid && d.plan_gen == gen;
  c->plan_terms = resident ? (const void *)&p : nullptr;
  c->plan_ws = resident ? ws : nullptr;
  c->plan_gen = gen;
  d.plan_ctx = 0;  // unknown until this call's upload has been enqueued
  d.plan_gen = 0;
  e = expect_run(c, p, (char *)ws, (size_t)TNMPS_NOALLOC_SCRATCH_BYTES, 0, energy_dev,
                 per_term_dev, nullptr, nullptr);
  // the workspace path's cache must not point at the shared array
  c->plan_terms = nullptr;
  c->plan_ws = nullptr;
  if (e != cudaSuccess) {
    c->last_error = std::string("no-alloc expectation: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TNMPS_ERR_NOMEM : TNMPS_ERR_CUDA;
  }
  d.plan_ctx = c->uid;
  d.plan_gen = gen;
  return TNMPS_OK;
}
