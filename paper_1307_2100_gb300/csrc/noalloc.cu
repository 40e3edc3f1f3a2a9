// noalloc.cu -- tc_contract_dot_noalloc: the scalar (Class 1) contraction
// without a caller-supplied workspace.
//
// Some callers cannot allocate device memory at the point where they run a
// contraction: runtimes that hand all device memory to their own pool up
// front, plug-ins that are only given input and output pointers, and
// latency-critical loops that cannot afford the device synchronisation that
// cudaMalloc and cudaFree may imply.  The scalar contraction needs scratch
// space for its per-block partial sums; this entry point keeps that scratch
// in a fixed array compiled into the library instead of asking for a
// workspace.  It launches the same two DOT kernels as tc_contract (one
// partial per CTA, then their ordered sum), only with the partials in that
// array.
//
// The array is file-scope device memory: every GPU that loads the library
// holds it (TC_NOALLOC_SCRATCH_BYTES) until the process exits.  All calls
// share it, so two calls that overlap on the GPU (different streams, or
// concurrent work on one device) race and give wrong results; calls ordered
// on one stream are fine.  The array keeps the last call's partial sums;
// nothing in it has to start at zero, because each call writes every slot it
// later reads.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress while
// that device is current and keeps it for the life of the process (a
// cudaDeviceReset of that device invalidates the kept address).
#include <cuda_runtime.h>

#include <mutex>

#include "tc_internal.h"

namespace tc {
namespace {

constexpr size_t kScratchBytes = TC_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
tc_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return TC_ERR_CUDA;
  if (dev >= kMaxDevices) return TC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return TC_ERR_CUDA;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return TC_OK;
}

}  // namespace
}  // namespace tc

using namespace tc;

extern "C" tc_status tc_contract_dot_noalloc(tc_plan_t plan, double alpha, const void* A,
                                             const void* B, double beta, void* C, void* stream) {
  if (!plan) return TC_ERR_INVALID_ARG;
  const Plan* P = reinterpret_cast<const Plan*>(plan);
  const GemmArgs& g = P->args;
  const uint64_t outs = (uint64_t)g.M * (uint64_t)g.N * (uint64_t)g.nbatch;
  if (P->kernel != K_DOT || outs != 1 || P->copy_which) return TC_ERR_UNSUPPORTED;
  if (P->empty_out) return TC_OK;
  if (!C) return TC_ERR_INVALID_ARG;
  // The DOT kernel writes a fixed number of partial sums (608 doubles, 4.9 KB),
  // whatever the contraction's size, so every scalar plan fits today; this
  // guard keeps the limit enforced should that number ever grow.
  if ((size_t)dot_partials(g, P->tile) * sizeof(double) > kScratchBytes) return TC_ERR_WORKSPACE;
  if (P->empty_k || alpha == 0.0)
    return launch_scale(P->gc, C, beta, P->dtype, P->c_elems_span, stream);
  if (!A || !B) return TC_ERR_INVALID_ARG;
  void* scratch = nullptr;
  tc_status st = scratch_address(&scratch);
  if (st != TC_OK) return st;
  GemmArgs a = g;
  a.A = P->swapped ? B : A;
  a.B = P->swapped ? A : B;
  a.C = C;
  a.alpha = alpha;
  a.beta = beta;
  a.ws = nullptr;
  return launch_dot_scalar(a, P->dtype, static_cast<double*>(scratch), stream);
}
