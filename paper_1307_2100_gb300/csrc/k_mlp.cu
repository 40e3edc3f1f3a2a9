// k_mlp.cu -- the mapping selector's network, trained and run by the
// library's own kernels.
//
// A 3-layer perceptron predicts, from a contraction descriptor's feature
// vector, the log2 runtime of every candidate mapping:
//   H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),  Y = H2 W3^T + b3.
// Parameters live as an FP32 master copy (updated by Adam) and an FP16
// working copy (used by the forward and backward passes, i.e. the network
// that is deployed is the FP16 one).  The loss is the masked mean squared
// error over the candidates that can run the descriptor.  All kernels are
// plain CUDA-core kernels (the network is 20k parameters); each sum runs in a
// fixed order, so training is deterministic.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "tc_internal.h"

namespace tc {
namespace mlp {

struct Net {
  int32_t n_in, n_hidden, n_out, max_batch;
  int64_t n_params;
  int64_t off[6];      // W1, b1, W2, b2, W3, b3 offsets in the flat vector
  float* master;       // FP32 parameters
  __half* work;        // FP16 working copy
  float* m;            // Adam moments
  float* v;
  float* z1;           // pre-activations [max_batch, hidden]
  float* z2;
  float* y;            // [max_batch, n_out]
  float* dy;
  float* dz2;
  float* dz1;
  float* loss;         // device scalar
};

constexpr int kT = 256;

// out[b, o] = act(sum_i in[b, i] * W[o, i] + bias[o]); relu applied to `in`
// when relu_in (the previous layer's pre-activation is stored).
__global__ void k_fwd(const float* __restrict__ in, int relu_in, const __half* __restrict__ W,
                      const __half* __restrict__ bias, float* __restrict__ out, int B, int nin,
                      int nout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * nout) return;
  const int b = idx / nout, o = idx % nout;
  float s = __half2float(bias[o]);
  const float* x = in + (size_t)b * nin;
  const __half* w = W + (size_t)o * nin;
  for (int i = 0; i < nin; ++i) {
    float xv = x[i];
    if (relu_in) xv = fmaxf(xv, 0.0f);
    s = fmaf(xv, __half2float(w[i]), s);
  }
  out[idx] = s;
}

// dy = 2 * mask * (y - t) / sum(mask); loss = sum(mask * (y - t)^2) / sum(mask).
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t,
                       const float* __restrict__ mask, float* __restrict__ dy,
                       float* __restrict__ loss, int n) {
  __shared__ double red[2][kT];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n; i += kT) {
    const double r = (double)y[i] - (double)t[i];
    s += (double)mask[i] * r * r;
    c += (double)mask[i];
  }
  red[0][threadIdx.x] = s;
  red[1][threadIdx.x] = c;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  const double cnt = red[1][0] > 0 ? red[1][0] : 1.0;
  if (threadIdx.x == 0) *loss = (float)(red[0][0] / cnt);
  for (int i = threadIdx.x; i < n; i += kT)
    dy[i] = (float)(2.0 * (double)mask[i] * ((double)y[i] - (double)t[i]) / cnt);
}

// dW[o, i] = sum_b dz[b, o] * act(in[b, i]);  db[o] = sum_b dz[b, o].
__global__ void k_wgrad(const float* __restrict__ dz, const float* __restrict__ in, int relu_in,
                        float* __restrict__ dW, float* __restrict__ db, int B, int nin, int nout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nout * nin) {
    const int o = idx / nin, i = idx % nin;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) {
      float xv = in[(size_t)b * nin + i];
      if (relu_in) xv = fmaxf(xv, 0.0f);
      s = fmaf(dz[(size_t)b * nout + o], xv, s);
    }
    dW[idx] = s;
  } else if (idx < nout * nin + nout) {
    const int o = idx - nout * nin;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dz[(size_t)b * nout + o];
    db[o] = s;
  }
}

// dz_in[b, i] = (sum_o dz[b, o] * W[o, i]) * (z_in[b, i] > 0).
__global__ void k_dgrad(const float* __restrict__ dz, const __half* __restrict__ W,
                        const float* __restrict__ z_in, float* __restrict__ dz_in, int B, int nin,
                        int nout) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * nin) return;
  const int b = idx / nin, i = idx % nin;
  float s = 0.0f;
  for (int o = 0; o < nout; ++o) s = fmaf(dz[(size_t)b * nout + o], __half2float(W[(size_t)o * nin + i]), s);
  dz_in[idx] = z_in[idx] > 0.0f ? s : 0.0f;
}

// Adam (bias-corrected) on the FP32 master copy, then the FP16 working copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __half* __restrict__ w, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  w[i] = __float2half_rn(pi);
}

__global__ void k_to_half(const float* __restrict__ p, __half* __restrict__ w, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) w[i] = __float2half_rn(p[i]);
}

__global__ void k_to_float(const __half* __restrict__ w, float* __restrict__ p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = __half2float(w[i]);
}

inline int blocks(int64_t n) { return (int)((n + kT - 1) / kT); }

void free_net(Net* N) {
  if (!N) return;
  cudaFree(N->master);
  cudaFree(N->work);
  cudaFree(N->m);
  cudaFree(N->v);
  cudaFree(N->z1);
  cudaFree(N->z2);
  cudaFree(N->y);
  cudaFree(N->dy);
  cudaFree(N->dz2);
  cudaFree(N->dz1);
  cudaFree(N->loss);
  delete N;
}

// Forward pass of the working copy; fills z1, z2, y.
tc_status forward(Net* N, const float* X, int B, cudaStream_t s) {
  const int F = N->n_in, H = N->n_hidden, C = N->n_out;
  const __half* w = N->work;
  k_fwd<<<blocks((int64_t)B * H), kT, 0, s>>>(X, 0, w + N->off[0], w + N->off[1], N->z1, B, F, H);
  k_fwd<<<blocks((int64_t)B * H), kT, 0, s>>>(N->z1, 1, w + N->off[2], w + N->off[3], N->z2, B, H,
                                              H);
  k_fwd<<<blocks((int64_t)B * C), kT, 0, s>>>(N->z2, 1, w + N->off[4], w + N->off[5], N->y, B, H,
                                              C);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

}  // namespace mlp
}  // namespace tc

using namespace tc;
using namespace tc::mlp;

extern "C" tc_status tc_mlp_create(tc_mlp_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                                   int32_t max_batch) {
  if (!out || n_in <= 0 || n_hidden <= 0 || n_out <= 0 || max_batch <= 0) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  Net* N = new (std::nothrow) Net();
  if (!N) return TC_ERR_INVALID_ARG;
  std::memset(N, 0, sizeof(*N));
  N->n_in = n_in;
  N->n_hidden = n_hidden;
  N->n_out = n_out;
  N->max_batch = max_batch;
  const int64_t sz[6] = {(int64_t)n_hidden * n_in, n_hidden, (int64_t)n_hidden * n_hidden,
                         n_hidden, (int64_t)n_out * n_hidden, n_out};
  int64_t k = 0;
  for (int i = 0; i < 6; ++i) {
    N->off[i] = k;
    k += sz[i];
  }
  N->n_params = k;
  const size_t P = (size_t)k, BH = (size_t)max_batch * n_hidden, BC = (size_t)max_batch * n_out;
  bool ok = cudaMalloc(&N->master, P * 4) == cudaSuccess &&
            cudaMalloc(&N->work, P * 2) == cudaSuccess && cudaMalloc(&N->m, P * 4) == cudaSuccess &&
            cudaMalloc(&N->v, P * 4) == cudaSuccess && cudaMalloc(&N->z1, BH * 4) == cudaSuccess &&
            cudaMalloc(&N->z2, BH * 4) == cudaSuccess && cudaMalloc(&N->y, BC * 4) == cudaSuccess &&
            cudaMalloc(&N->dy, BC * 4) == cudaSuccess && cudaMalloc(&N->dz2, BH * 4) == cudaSuccess &&
            cudaMalloc(&N->dz1, BH * 4) == cudaSuccess && cudaMalloc(&N->loss, 4) == cudaSuccess;
  if (ok) ok = cudaMemset(N->master, 0, P * 4) == cudaSuccess &&
               cudaMemset(N->work, 0, P * 2) == cudaSuccess &&
               cudaMemset(N->m, 0, P * 4) == cudaSuccess && cudaMemset(N->v, 0, P * 4) == cudaSuccess;
  if (!ok) {
    free_net(N);
    return TC_ERR_CUDA;
  }
  *out = reinterpret_cast<tc_mlp_t>(N);
  return TC_OK;
}

extern "C" tc_status tc_mlp_destroy(tc_mlp_t net) {
  free_net(reinterpret_cast<Net*>(net));
  return TC_OK;
}

extern "C" tc_status tc_mlp_num_params(tc_mlp_t net, int64_t* n) {
  if (!net || !n) return TC_ERR_INVALID_ARG;
  *n = reinterpret_cast<Net*>(net)->n_params;
  return TC_OK;
}

extern "C" tc_status tc_mlp_set_params(tc_mlp_t net, const float* host, int64_t n) {
  Net* N = reinterpret_cast<Net*>(net);
  if (!N || !host || n != N->n_params) return TC_ERR_INVALID_ARG;
  if (cudaMemcpy(N->master, host, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return TC_ERR_CUDA;
  k_to_half<<<blocks(n), kT>>>(N->master, N->work, n);
  if (cudaMemset(N->m, 0, (size_t)n * 4) != cudaSuccess ||
      cudaMemset(N->v, 0, (size_t)n * 4) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return TC_ERR_CUDA;
  return TC_OK;
}

extern "C" tc_status tc_mlp_get_params(tc_mlp_t net, float* host, int64_t n, int32_t working) {
  Net* N = reinterpret_cast<Net*>(net);
  if (!N || !host || n != N->n_params) return TC_ERR_INVALID_ARG;
  if (!working)
    return cudaMemcpy(host, N->master, (size_t)n * 4, cudaMemcpyDeviceToHost) == cudaSuccess
               ? TC_OK
               : TC_ERR_CUDA;
  std::vector<__half> h((size_t)n);
  if (cudaMemcpy(h.data(), N->work, (size_t)n * 2, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TC_ERR_CUDA;
  for (int64_t i = 0; i < n; ++i) host[i] = __half2float(h[(size_t)i]);
  return TC_OK;
}

extern "C" tc_status tc_mlp_forward(tc_mlp_t net, const float* X, float* Y, int32_t batch,
                                    void* stream) {
  Net* N = reinterpret_cast<Net*>(net);
  if (!N || !X || !Y || batch <= 0 || batch > N->max_batch) return TC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tc_status st = forward(N, X, batch, s);
  if (st != TC_OK) return st;
  if (cudaMemcpyAsync(Y, N->y, (size_t)batch * N->n_out * 4, cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return TC_ERR_CUDA;
  return TC_OK;
}

extern "C" tc_status tc_mlp_loss_grad(tc_mlp_t net, const float* X, const float* T,
                                      const float* mask, int32_t batch, float* loss, float* grad,
                                      void* stream) {
  Net* N = reinterpret_cast<Net*>(net);
  if (!N || !X || !T || !mask || !loss || !grad || batch <= 0 || batch > N->max_batch)
    return TC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int F = N->n_in, H = N->n_hidden, C = N->n_out, B = batch;
  tc_status st = forward(N, X, B, s);
  if (st != TC_OK) return st;
  const __half* w = N->work;
  k_loss<<<1, kT, 0, s>>>(N->y, T, mask, N->dy, loss, B * C);
  // layer 3
  k_wgrad<<<blocks((int64_t)C * H + C), kT, 0, s>>>(N->dy, N->z2, 1, grad + N->off[4],
                                                    grad + N->off[5], B, H, C);
  k_dgrad<<<blocks((int64_t)B * H), kT, 0, s>>>(N->dy, w + N->off[4], N->z2, N->dz2, B, H, C);
  // layer 2
  k_wgrad<<<blocks((int64_t)H * H + H), kT, 0, s>>>(N->dz2, N->z1, 1, grad + N->off[2],
                                                    grad + N->off[3], B, H, H);
  k_dgrad<<<blocks((int64_t)B * H), kT, 0, s>>>(N->dz2, w + N->off[2], N->z1, N->dz1, B, H, H);
  // layer 1
  k_wgrad<<<blocks((int64_t)H * F + H), kT, 0, s>>>(N->dz1, X, 0, grad + N->off[0],
                                                    grad + N->off[1], B, F, H);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

extern "C" tc_status tc_mlp_adam_step(tc_mlp_t net, const float* grad, float lr, float beta1,
                                      float beta2, float eps, int32_t t, void* stream) {
  Net* N = reinterpret_cast<Net*>(net);
  if (!N || !grad || t <= 0) return TC_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
  k_adam<<<blocks(N->n_params), kT, 0, static_cast<cudaStream_t>(stream)>>>(
      N->master, grad, N->m, N->v, N->work, N->n_params, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
