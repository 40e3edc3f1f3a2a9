// storage.cuh -- element types of stored tensors and their arithmetic types.
//
// A, B and C are stored as FP64, FP32, BF16 or FP16 (tc_dtype).  The CUDA-core
// kernels compute in FP64 for FP64 data and in FP32 otherwise: a BF16 or FP16
// element is widened exactly on load, and a result is rounded to nearest
// (ties to even) when it is stored.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace tc {

template <typename S>
struct Cmp {
  using T = S;
};
template <>
struct Cmp<__nv_bfloat16> {
  using T = float;
};
template <>
struct Cmp<__half> {
  using T = float;
};

__device__ __forceinline__ double ld_c(double x) { return x; }
__device__ __forceinline__ float ld_c(float x) { return x; }
__device__ __forceinline__ float ld_c(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float ld_c(__half x) { return __half2float(x); }

// Round a value to the storage type (to nearest, ties to even).
template <typename S>
__device__ __forceinline__ S st_c(double v);
template <>
__device__ __forceinline__ double st_c<double>(double v) { return v; }
template <>
__device__ __forceinline__ float st_c<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 st_c<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
template <>
__device__ __forceinline__ __half st_c<__half>(double v) { return __double2half(v); }

template <typename S>
__device__ __forceinline__ S st_cf(float v);
template <>
__device__ __forceinline__ double st_cf<double>(float v) { return (double)v; }
template <>
__device__ __forceinline__ float st_cf<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 st_cf<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half st_cf<__half>(float v) { return __float2half_rn(v); }

// Store a compute-type value (FP64 or FP32) to storage type S.
template <typename S>
__device__ __forceinline__ S st_any(double v) { return st_c<S>(v); }
template <typename S>
__device__ __forceinline__ S st_any(float v) { return st_cf<S>(v); }

}  // namespace tc
