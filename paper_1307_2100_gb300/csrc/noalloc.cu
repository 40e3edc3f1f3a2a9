// noalloc.cu -- tc_contract_dot_noalloc: the scalar (Class 1) contraction
// without a caller-supplied workspace.
//
// Some callers cannot allocate device memory at the point where they run a
// contraction: code that executes while a CUDA graph is being captured (where
// cudaMalloc is not allowed), runtimes that hand all device memory to their
// own pool up front, or plug-ins that are only given input and output
// pointers.  The scalar contraction needs scratch space for its per-block
// partial sums; this entry point keeps that scratch in a fixed array compiled
// into the library instead of asking for a workspace.
//
// The array is file-scope device memory: every GPU that loads the library
// holds it (TC_NOALLOC_SCRATCH_BYTES) until the process exits.  All calls
// share it, so two calls that overlap on the GPU (different streams, or the
// same stream in concurrent graphs) race and give wrong results; calls
// ordered on one stream are fine.  The array keeps the last call's partial
// sums; nothing in it has to start at zero, because each call writes every
// slot it later reads.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress while
// that device is current and keeps it; make that first call before any
// stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "groups.cuh"
#include "tc_internal.h"

namespace tc {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 152 * 4;                 // partial sums per call
constexpr size_t kScratchBytes = TC_NOALLOC_SCRATCH_BYTES;
static_assert(kNaBlocks * sizeof(double) <= kScratchBytes, "scratch too small");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Each CTA sums a grid-strided share of k in FP64 into one slot of `part`.
template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_na_partial(const __grid_constant__ GemmArgs p,
                                                           double* part) {
  __shared__ double red[kNaThreads / 32];
  const T* __restrict__ X = static_cast<const T*>(p.A);
  const T* __restrict__ Y = static_cast<const T*>(p.B);
  const uint32_t K = (uint32_t)p.K;
  double acc = 0.0;
  const uint32_t stride = gridDim.x * kNaThreads;
  for (uint32_t k = blockIdx.x * kNaThreads + threadIdx.x; k < K; k += stride) {
    int64_t ox, oy;
    goff2(p.gk, 0, 1, k, ox, oy);
    acc = fma((double)X[ox], (double)Y[oy], acc);
  }
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// One CTA adds the partial sums in slot order and applies alpha and beta.
template <typename T>
__global__ void k_na_final(const __grid_constant__ GemmArgs p, const double* part, int nparts) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    T* dst = static_cast<T*>(p.C);
    double v = p.alpha * t;
    if (p.beta != 0.0) v += p.beta * (double)*dst;
    *dst = (T)v;
  }
}

// Device address of the scratch array on the current device (looked up once).
tc_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TC_ERR_CUDA;
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
  if ((size_t)kNaBlocks * sizeof(double) > kScratchBytes) return TC_ERR_WORKSPACE;
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
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* part = static_cast<double*>(scratch);
  if (P->dtype == TC_F64) {
    k_na_partial<double><<<kNaBlocks, kNaThreads, 0, s>>>(a, part);
    k_na_final<double><<<1, 256, 0, s>>>(a, part, kNaBlocks);
  } else {
    k_na_partial<float><<<kNaBlocks, kNaThreads, 0, s>>>(a, part);
    k_na_final<float><<<1, 256, 0, s>>>(a, part, kNaBlocks);
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
