// k_peak.cu -- peak-rate probes: how many floating-point operations per second
// one GB300 executes in each arithmetic the contraction kernels use, measured
// in the same process as the kernels they are the roofline of.  No memory
// traffic: operands live in registers (CUDA-core probes) or in a shared-memory
// tile that every MMA re-reads (tensor-core probes).
//
//   TC_PEAK_DFMA     FP64 fused multiply-adds on the CUDA cores (the FP64 GEMM,
//                    GEMV and DOT kernels' arithmetic)
//   TC_PEAK_DMMA     FP64 mma.sync m8n8k4 (the FP64 tensor path, for reference)
//   TC_PEAK_FFMA     FP32 fused multiply-adds (the FP32 CUDA-core kernels)
//   TC_PEAK_BF16     tcgen05.mma kind::f16, BF16, M = 128, N = 128, K = 16 (the
//                    split-BF16 GEMMs' instruction shape)
//   TC_PEAK_BF16_N256  the same with N = 256
//   TC_PEAK_FP8      tcgen05.mma kind::mxf8f6f4 block-scaled E4M3, M = 128,
//                    N = 128, K = 32 (the FP8 GEMM's instruction shape)
#include <cuda_runtime.h>

#include "sm100.cuh"
#include "tc_internal.h"

namespace tc {
namespace {

constexpr int kSms = 152;
constexpr uint64_t kTimeoutNs = 2000000000ull;
static __device__ double g_sink[4];

// ---------------------------------------------------------------- CUDA cores
template <typename T>
__global__ void __launch_bounds__(256) k_peak_fma(int64_t iters, T seed) {
  T x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = seed + (T)(threadIdx.x + c);
  const T a = (T)0.999999, b = (T)1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  if (s == (T)-12345.0) g_sink[0] = (double)s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_dmma(int64_t iters) {
  double d[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) d[c][0] = d[c][1] = 0.0;
  const double a = 1e-3 * (threadIdx.x & 7), b = 1e-3 * (threadIdx.x >> 3);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
          : "+d"(d[c][0]), "+d"(d[c][1])
          : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += d[c][0] + d[c][1];
  if (s == -12345.0) g_sink[1] = s;
}

// --------------------------------------------------------------- tensor cores
// One CTA per SM, 128 threads.  Thread 0 issues `iters` MMAs on operand tiles
// in shared memory (zeros) into tensor memory, then one commit; the CTA waits
// for it with a bounded wait.
// The launch asks for kPeakSmem bytes of dynamic shared memory so that one
// CTA fits on an SM (two would share one SM's tensor core).
constexpr int kPeakSmem = 160 * 1024;

template <int KIND>
__global__ void __launch_bounds__(128, 1) k_peak_tc(int64_t iters) {
  extern __shared__ __align__(1024) uint8_t ops[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 16384 / 16; i += 128)
    reinterpret_cast<uint4*>(ops)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 0) tmem_alloc(&tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (KIND == 2) {  // scale cells: 2^0 for every row and column (byte 127)
    uint32_t r[4] = {0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu, 0x7F7F7F7Fu};
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    tmem_st4(tl + 256, r);
    tmem_st4(tl + 260, r);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    const uint32_t sa = smem_u32(ops), sb = sa + 8192;
    for (int64_t i = 0; i < iters; ++i) {
      const uint32_t acc = i > 1 ? 1u : 0u;
      if (KIND == 0) {  // BF16, 128 x 128 x 16, two accumulators
        mma_bf16(tmem + (uint32_t)(i & 1) * 128, smem_desc(sa, 2048, 128),
                 smem_desc(sb, 2048, 128), idesc_bf16(128, 128), acc);
      } else if (KIND == 1) {  // BF16, 128 x 256 x 16
        mma_bf16(tmem + (uint32_t)(i & 1) * 256, smem_desc(sa, 2048, 128),
                 smem_desc(sb, 4096, 128), idesc_bf16(128, 256), acc);
      } else {  // block-scaled E4M3, 128 x 128 x 32
        mma_mx_e4m3(tmem + (uint32_t)(i & 1) * 128, smem_desc(sa, 2048, 128),
                    smem_desc(sb, 2048, 128), idesc_mx_e4m3(128, 128, 0, 0), tmem + 256,
                    tmem + 260, acc);
      }
    }
    mma_commit(&bar);
  }
  __syncwarp();
  if (tid == 0) mbar_wait(&bar, 0, &abort_flag, kTimeoutNs);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

tc_status peak_read_status(int* h, void* stream) {
  return read_clear_status(h, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TC_OK
                                                                                : TC_ERR_CUDA;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_peak_probe(int32_t kind, int64_t iters, double* flops, void* stream) {
  if (iters < 1 || !flops) return TC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int fma_grid = kSms * 8;  // 8 CTAs of 256 threads per SM
  switch (kind) {
    case TC_PEAK_DFMA:
      k_peak_fma<double><<<fma_grid, 256, 0, s>>>(iters, 1.0);
      *flops = 2.0 * 8 * (double)iters * fma_grid * 256;
      break;
    case TC_PEAK_FFMA:
      k_peak_fma<float><<<fma_grid, 256, 0, s>>>(iters, 1.0f);
      *flops = 2.0 * 8 * (double)iters * fma_grid * 256;
      break;
    case TC_PEAK_DMMA:
      k_peak_dmma<<<fma_grid, 256, 0, s>>>(iters);
      *flops = 2.0 * 8 * 8 * 4 * 4 * (double)iters * (fma_grid * 256 / 32);
      break;
    case TC_PEAK_BF16:
      if (cudaFuncSetAttribute(k_peak_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kPeakSmem) != cudaSuccess)
        return TC_ERR_CUDA;
      k_peak_tc<0><<<kSms, 128, kPeakSmem, s>>>(iters);
      *flops = 2.0 * 128 * 128 * 16 * (double)iters * kSms;
      break;
    case TC_PEAK_BF16_N256:
      if (cudaFuncSetAttribute(k_peak_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kPeakSmem) != cudaSuccess)
        return TC_ERR_CUDA;
      k_peak_tc<1><<<kSms, 128, kPeakSmem, s>>>(iters);
      *flops = 2.0 * 128 * 256 * 16 * (double)iters * kSms;
      break;
    case TC_PEAK_FP8:
      if (cudaFuncSetAttribute(k_peak_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kPeakSmem) != cudaSuccess)
        return TC_ERR_CUDA;
      k_peak_tc<2><<<kSms, 128, kPeakSmem, s>>>(iters);
      *flops = 2.0 * 128 * 128 * 32 * (double)iters * kSms;
      break;
    default:
      return TC_ERR_INVALID_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
