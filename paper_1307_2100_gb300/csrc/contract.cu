// contract.cu -- tc_contract: run a plan's kernels on the caller's stream.
#include <cuda_runtime.h>

#include "sm100.cuh"
#include "tc_internal.h"

using namespace tc;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" tc_status tc_contract(tc_plan_t plan, double alpha, const void* A, const void* B,
                                 double beta, void* C, void* workspace, size_t ws_bytes,
                                 void* stream) {
  if (!plan) return TC_ERR_INVALID_ARG;
  const Plan* P = reinterpret_cast<const Plan*>(plan);
  if (P->empty_out) return TC_OK;
  if (!C) return TC_ERR_INVALID_ARG;
  if (P->workspace > 0 && (!workspace || ws_bytes < P->workspace)) return TC_ERR_WORKSPACE;
  const bool packed = P->kernel == K_GEMM_FP8 ||
                      (P->kernel == K_GEMM_TC && (P->tile == kTilePacked || P->tile == kTilePackedWide ||
                                                  P->tile == kTilePackedPair));
  if (packed && (reinterpret_cast<uintptr_t>(workspace) & 15) != 0)
    return TC_ERR_INVALID_ARG;  // the packed operands are moved by 16-byte bulk copies
  if (P->empty_k || alpha == 0.0)
    return launch_scale(P->gc, C, beta, P->dtype, P->c_elems_span, stream);
  if (!A || !B) return TC_ERR_INVALID_ARG;

  GemmArgs a = P->args;
  a.A = P->swapped ? B : A;
  a.B = P->swapped ? A : B;
  a.C = C;
  a.alpha = alpha;
  a.beta = beta;
  char* ws = static_cast<char*>(workspace);
  const uint64_t outs = (uint64_t)a.M * (uint64_t)a.N * (uint64_t)a.nbatch;
  if (P->kernel == K_DOT && outs == 1) {
    a.ws = ws;
    ws += align256((size_t)dot_partials(a, P->tile) * 8);
  }
  tc_status st;
  if (P->copy_which) {
    PermArgs pa = P->perm;
    pa.in = P->copy_which == 1 ? a.A : a.B;
    pa.out = ws;
    if ((st = launch_perm(pa, P->dtype, stream)) != TC_OK) return st;
    if (P->copy_which == 1) a.A = ws; else a.B = ws;
    ws += align256((size_t)P->copy_elems * elem_size(P->dtype));
  }
  if (P->kernel == K_GEMM_SIMT && a.ksplit > 1) a.ws = ws;  // split-K partial tiles
  switch (P->kernel) {
    case K_GEMM_SIMT: return launch_gemm_simt(a, P->dtype, P->tile, stream);
    case K_GEMM_TC:
      return (P->tile == kTilePacked || P->tile == kTilePackedWide ||
              P->tile == kTilePackedPair)
                 ? launch_gemm_tc_packed(a, P->math, P->dtype, P->tile, ws, stream)
                                    : launch_gemm_tc(a, P->math, stream);
    case K_GEMM_FP8: return launch_gemm_fp8(a, P->tile, ws, stream);
    case K_GEMV: return launch_gemv(a, P->dtype, P->tile, stream);
    case K_DOT: return launch_dot(a, P->dtype, P->tile, stream);
    case K_GER: return launch_ger(a, P->dtype, stream);
    default: return TC_ERR_UNSUPPORTED;
  }
}

namespace tc {
// One warp waits (bounded) on a barrier that never completes.
__global__ void k_selftest_wait(uint64_t timeout_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort, timeout_ns);
}
}  // namespace tc

extern "C" tc_status tc_selftest_wait_timeout(int64_t timeout_ns, void* stream) {
  if (timeout_ns <= 0 || timeout_ns > 10000000000ll) return TC_ERR_INVALID_ARG;
  k_selftest_wait<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((uint64_t)timeout_ns);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

extern "C" tc_status tc_device_status(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h0 = 0, h1 = 0, h2 = 0, h3 = 0, h4 = 0;
  if (read_clear_status(&h0, s) != cudaSuccess || tc_gemm_read_status(&h1, s) != TC_OK ||
      tc_fp8_read_status(&h2, s) != TC_OK || tc_pk_read_status(&h3, s) != TC_OK ||
      peak_read_status(&h4, s) != TC_OK || cudaStreamSynchronize(s) != cudaSuccess)
    return TC_ERR_CUDA;
  return (h0 || h1 || h2 || h3 || h4) ? TC_ERR_TIMEOUT : TC_OK;
}
