// batch.cu -- many contractions in one submission (tc_batch_plan /
// tc_contract_batched).
//
// Each contraction of a batch is routed by its GEMM view:
//   * tensor-core route: one GEMM (no batch group) with M and N both at least
//     `tc_min_mn` (64 by default):
//     one batched pack pass splits the operands of every such contraction into
//     BF16 terms in the batch's own device memory (one CTA per operand tile and
//     128 K), then their 128x128 tiles join one work list, longest K first,
//     processed by the persistent packed tcgen05 kernel (one CTA per SM);
//     tiles with more K than half an SM's share are split into K ranges whose
//     partial sums a reduction kernel adds;
//   * SIMT route: the low-arithmetic-intensity contractions (Class 1 and 2 and
//     skinny Class 3 ones; the paper's BLAS-1/2 cases of Sec. 3.2.1-3.2.2) and
//     plans of the slicing mapping (a batch group of GEMMs),
//     where a 128x128 tile would waste most of its work: batched CUDA-core
//     kernels compute partial sums over K segments into the batch's own
//     workspace -- 32x32 output tiles with operand blocks staged in shared
//     memory where min(M, N) >= 16, a thread per output otherwise (a warp per
//     output below 256 outputs) -- and a last kernel adds the segments of each
//     output in order (deterministic) and applies alpha and beta; outputs of
//     one segment are stored by the partial kernels themselves.  Long K is
//     split so that even a single-output contraction spreads over many SMs.
// The (up to six) kernels go on the caller's stream, the CUDA-core ones on a
// stream of the batch's own forked from and joined back to it when both routes
// have work; nothing is allocated or copied per call, so tc_contract_batched
// may be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "groups.cuh"
#include "tc_internal.h"

namespace tc {
namespace bat {

constexpr int kThreads = 256;
constexpr int kChunk = 512;     // K offsets staged in shared memory at a time
constexpr int kRun = 8;         // thread mode: products per FP32 run

struct TcWork {
  int32_t item, tile, split;  // split: the K range of the item's tile
};

// One entry of the SIMT partial-sum kernel.
struct SimtWork {
  int32_t item;    // index into the batch's items
  int32_t mode;    // 0: a thread per output (256 consecutive outputs), 1: a warp per output (8)
  int64_t out0;    // first output of the entry
  int64_t k0, k1;  // K segment [k0, k1)
  int64_t slot;    // partial-sum slot of the first output (thread mode: + thread index)
  int32_t nseg;    // segments of this item (slots of one output are nseg apart)
  int32_t pad_;
};

// One entry of the SIMT tile kernel: a kTile x kTile tile of outputs of an
// item over a K segment.
struct SimtTileWork {
  int32_t item;
  int32_t nseg;    // segments of this item
  int64_t tile;    // (m-tile fastest, n-tile, batch)
  int64_t k0, k1;  // K segment [k0, k1)
  int64_t slot;    // partial-sum slot of the item's output 0, segment 0
  int64_t seg;     // this entry's segment
};

constexpr int kTile = 32;      // tile kernel: outputs per tile side
constexpr int kTileK = 16;     // K per shared-memory block
constexpr int kTileRun = 2;    // blocks summed in FP32 before a compensated add
constexpr int kTileThreads = 128;
constexpr int kTileMin = 16;   // items with min(M, N) at least this take the tile kernel
constexpr int kTcTile = 128;   // output tile side of the packed tensor-core kernel

// One entry of the SIMT final kernel: 256 consecutive outputs of an item.
struct SimtFinal {
  int32_t item, nseg;
  int64_t out0, slot0;  // slot of output out0, segment 0
};

struct Batch {
  int32_t n;
  int32_t math;
  double flops, min_bytes;
  int32_t n_tc_items, n_simt_items;
  int64_t n_tc_work, n_simt_work, n_simt_tiles, n_simt_final, n_pack;
  GemmArgs* d_items;
  TcWork* d_tc_work;
  SimtWork* d_simt_work;
  SimtTileWork* d_simt_tile;
  SimtFinal* d_simt_final;
  double* d_partials;
  PkItem* d_pk;          // per item: the packed GEMM of tensor-core items
  int32_t* d_pack;       // pack entries (item, operand, row tile, 128-K chunk)
  uint8_t* d_pkws;       // packed operands of every tensor-core item
  float2* d_pkpart;      // split-K partial sums of tensor-core items
  int32_t* d_red;        // split-K reduction entries (item, tile)
  int64_t n_red;
  cudaStream_t side;     // the CUDA-core route's stream when both routes have work
  cudaEvent_t fork, join;
};

// Neumaier's compensated summation of FP32 terms (here: the sums of short
// runs of FP32 fused multiply-adds).
struct Neumaier {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    if (fabsf(s) >= fabsf(x)) c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
    else c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (m, n, batch) of output o = m + M (n + N b): 32-bit divisions while the
// outputs of the item fit in 32 bits.
__device__ __forceinline__ void split_output(uint64_t o, uint64_t M, uint64_t N, uint64_t outs,
                                             uint32_t& m, uint32_t& n, uint32_t& b) {
  if (outs <= 0xffffffffull) {
    const uint32_t o32 = (uint32_t)o, M32 = (uint32_t)M, N32 = (uint32_t)N;
    const uint32_t r = o32 / M32;
    m = o32 - r * M32;
    n = r % N32;
    b = r / N32;
  } else {
    const uint64_t r = o / M;
    m = (uint32_t)(o - r * M);
    n = (uint32_t)(r % N);
    b = (uint32_t)(r / N);
  }
}

// C = alpha * v + beta * C of one output, in FP64 (C is not read when beta == 0).
__device__ __forceinline__ void store_output(float* dst, double v, double alpha, double beta) {
  double x = alpha * v;
  if (beta != 0.0) x += beta * (double)*dst;
  *dst = (float)x;
}

// Partial sums of one K segment.  Operand pointers come from the device
// pointer arrays (exchanged for items whose plan swapped the operands).  The
// K offsets of both operands are staged in shared memory as pairs, kChunk at a
// time.  Thread mode: a thread per output, runs of kRun products summed by
// FP32 fused multiply-adds (loads of a run issued together), the run sums
// added with Neumaier compensation.  Warp mode: up to 8 outputs of an item
// per block, a warp per output with lanes along K (each lane's run is its
// share of a chunk), lanes combined in FP64; the offset table of a chunk
// serves all of them.
__global__ void __launch_bounds__(kThreads, 6) k_simt_partial(
    const GemmArgs* __restrict__ items, const SimtWork* __restrict__ work, int64_t nwork,
    const void* const* Ap, const void* const* Bp, void* const* Cp, const double* alpha,
    const double* beta, double* __restrict__ partials) {
  __shared__ GemmArgs sa;
  __shared__ longlong2 oXY[kChunk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int cur = -1;
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const SimtWork wk = work[w];
    __syncthreads();
    if (wk.item != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(items + wk.item);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
      for (int i = tid; i < (int)(sizeof(GemmArgs) / 4); i += kThreads) dst[i] = src[i];
      cur = wk.item;
      __syncthreads();
    }
    const GemmArgs& p = sa;
    const float* X = static_cast<const float*>(p.swapped ? Bp[wk.item] : Ap[wk.item]);
    const float* Y = static_cast<const float*>(p.swapped ? Ap[wk.item] : Bp[wk.item]);
    const uint64_t M = (uint64_t)p.M, N = (uint64_t)p.N;
    const uint64_t outs = M * N * (uint64_t)p.nbatch;
    // output of this thread (thread mode) or of this warp (warp mode)
    const uint64_t o = (uint64_t)wk.out0 + (wk.mode == 0 ? tid : warp);
    int64_t xo = 0, yo = 0, co = 0;
    const bool valid = o < outs;
    if (valid) {
      uint32_t m, n, b;
      split_output(o, M, N, outs, m, n, b);
      int64_t bX, bY, bC, oXm, oCm, oYn, oCn;
      goff3(p.gb, b, bX, bY, bC);
      goff2(p.gm, 0, 2, m, oXm, oCm);
      goff2(p.gn, 1, 2, n, oYn, oCn);
      xo = bX + oXm;
      yo = bY + oYn;
      co = bC + oCm + oCn;
    }
    Neumaier acc;
    for (int64_t c0 = wk.k0; c0 < wk.k1; c0 += kChunk) {
      const int kn = (int)min((int64_t)kChunk, wk.k1 - c0);
      __syncthreads();
      for (int i = tid; i < kn; i += kThreads) {
        int64_t ox, oy;
        goff2(p.gk, 0, 1, (uint32_t)(c0 + i), ox, oy);
        oXY[i] = make_longlong2(ox, oy);
      }
      __syncthreads();
      if (!valid) continue;
      if (wk.mode == 0) {
        int i = 0;
        for (; i + kRun <= kn; i += kRun) {
          float xv[kRun], yv[kRun];
#pragma unroll
          for (int u = 0; u < kRun; ++u) {
            const longlong2 q = oXY[i + u];
            xv[u] = X[xo + q.x];
            yv[u] = Y[yo + q.y];
          }
          float run = 0.0f;
#pragma unroll
          for (int u = 0; u < kRun; ++u) run = fmaf(xv[u], yv[u], run);
          acc.add(run);
        }
        float run = 0.0f;
        for (; i < kn; ++i) {
          const longlong2 q = oXY[i];
          run = fmaf(X[xo + q.x], Y[yo + q.y], run);
        }
        acc.add(run);
      } else {
        float run = 0.0f;
#pragma unroll 4
        for (int i = lane; i < kn; i += 32) {
          const longlong2 q = oXY[i];
          run = fmaf(X[xo + q.x], Y[yo + q.y], run);
        }
        acc.add(run);
      }
    }
    // one segment: the output itself; else its partial-sum slot
    double v = acc.value();
    if (wk.mode != 0) v = warp_sum(v);
    if (valid && (wk.mode == 0 || lane == 0)) {
      if (wk.nseg == 1)
        store_output(static_cast<float*>(Cp[wk.item]) + co, v, alpha[wk.item], beta[wk.item]);
      else
        partials[wk.slot + (int64_t)(wk.mode == 0 ? tid : warp) * wk.nseg] = v;
    }
  }
}

// Partial sums of a 32 x 32 tile of outputs over one K segment, 128 threads
// (small enough to run beside the tensor-core kernel on an SM): operand
// blocks of 16 K are gathered into shared memory in the order of each
// operand's contiguous index (the next block prefetched into registers),
// each thread accumulates a 2 x 4 register tile (two adjacent rows read as
// float2, four adjacent columns as float4) in FP32 over two blocks and adds
// those sums into Neumaier-compensated (s, c) pairs: at most 32 FP32
// roundings per run plus the compensated sum.  Outputs of one segment are
// stored to C; otherwise partials go to the per-output segment slots.
__global__ void __launch_bounds__(kTileThreads, 6) k_simt_tile(
    const GemmArgs* __restrict__ items, const SimtTileWork* __restrict__ work, int64_t nwork,
    const void* const* Ap, const void* const* Bp, void* const* Cp, const double* alpha,
    const double* beta, double* __restrict__ partials) {
  __shared__ GemmArgs sa;
  __shared__ int64_t oX[kChunk], oY[kChunk];
  __shared__ int64_t offXm[kTile], offYn[kTile], offCm[kTile], offCn[kTile];
  __shared__ __align__(16) float Xs[kTileK][kTile + 2];
  __shared__ __align__(16) float Ys[kTileK][kTile + 4];
  constexpr int R = kTile * kTileK / kTileThreads;  // elements of each operand per thread
  const int tid = threadIdx.x;
  const int tx = tid % 8, ty = tid / 8;  // columns 4 tx .. 4 tx + 3, rows 2 ty, 2 ty + 1
  int cur = -1;
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const SimtTileWork wk = work[w];
    __syncthreads();
    if (wk.item != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(items + wk.item);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
      for (int i = tid; i < (int)(sizeof(GemmArgs) / 4); i += kTileThreads) dst[i] = src[i];
      cur = wk.item;
      __syncthreads();
    }
    const GemmArgs& p = sa;
    const float* X = static_cast<const float*>(p.swapped ? Bp[wk.item] : Ap[wk.item]);
    const float* Y = static_cast<const float*>(p.swapped ? Ap[wk.item] : Bp[wk.item]);
    const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N;
    const uint32_t tiles_m = (M + kTile - 1) / kTile, tiles_n = (N + kTile - 1) / kTile;
    const uint32_t tm = (uint32_t)(wk.tile % tiles_m);
    const uint64_t rest = (uint64_t)wk.tile / tiles_m;
    const uint32_t tn = (uint32_t)(rest % tiles_n), b = (uint32_t)(rest / tiles_n);
    int64_t bX, bY, bC;
    goff3(p.gb, b, bX, bY, bC);
    if (tid < kTile) {
      const uint32_t m = tm * kTile + tid;
      int64_t ox = -1, oc = 0;
      if (m < M) { goff2(p.gm, 0, 2, m, ox, oc); ox += bX; }
      offXm[tid] = ox;
      offCm[tid] = bC + oc;
    } else if (tid < 2 * kTile) {
      const uint32_t n = tn * kTile + (tid - kTile);
      int64_t oy = -1, oc = 0;
      if (n < N) { goff2(p.gn, 1, 2, n, oy, oc); oy += bY; }
      offYn[tid - kTile] = oy;
      offCn[tid - kTile] = oc;
    }
    float s[2][4], c[2][4], a0[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) s[i][j] = c[i][j] = a0[i][j] = 0.0f;
    const bool x_mn = p.a_contig == CONTIG_MN, y_mn = p.b_contig == CONTIG_MN;
    // element r of this thread: row / column and k in the block
    auto xrow = [&](int r) { const int e = tid + r * kTileThreads; return x_mn ? e % kTile : e / kTileK; };
    auto xkk = [&](int r) { const int e = tid + r * kTileThreads; return x_mn ? e / kTile : e % kTileK; };
    auto ycol = [&](int r) { const int e = tid + r * kTileThreads; return y_mn ? e % kTile : e / kTileK; };
    auto ykk = [&](int r) { const int e = tid + r * kTileThreads; return y_mn ? e / kTile : e % kTileK; };
    int64_t xo[R], yo[R];
    float rx[R], ry[R];
    __syncthreads();  // row and column offsets written
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xo[r] = offXm[xrow(r)];
      yo[r] = offYn[ycol(r)];
    }
    int kn = 0;
    auto fetch = [&](int kb) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int kx = kb + xkk(r), ky = kb + ykk(r);
        rx[r] = (xo[r] >= 0 && kx < kn) ? X[xo[r] + oX[kx]] : 0.0f;
        ry[r] = (yo[r] >= 0 && ky < kn) ? Y[yo[r] + oY[ky]] : 0.0f;
      }
    };
    auto fold = [&]() {  // Neumaier: (s, c) += run sums
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float x = a0[i][j], t = __fadd_rn(s[i][j], x);
          if (fabsf(s[i][j]) >= fabsf(x))
            c[i][j] = __fadd_rn(c[i][j], __fadd_rn(__fsub_rn(s[i][j], t), x));
          else
            c[i][j] = __fadd_rn(c[i][j], __fadd_rn(__fsub_rn(x, t), s[i][j]));
          s[i][j] = t;
          a0[i][j] = 0.0f;
        }
    };
    int nblk = 0;  // blocks in the current run
    for (int64_t c0 = wk.k0; c0 < wk.k1; c0 += kChunk) {
      kn = (int)min((int64_t)kChunk, wk.k1 - c0);
      __syncthreads();  // previous chunk's blocks are done with the tables
      for (int i = tid; i < kn; i += kTileThreads) {
        int64_t ox, oy;
        goff2(p.gk, 0, 1, (uint32_t)(c0 + i), ox, oy);
        oX[i] = ox;
        oY[i] = oy;
      }
      __syncthreads();  // tables written
      fetch(0);
      for (int kb = 0; kb < kn; kb += kTileK) {
        __syncthreads();  // previous block's Xs, Ys read
#pragma unroll
        for (int r = 0; r < R; ++r) {
          Xs[xkk(r)][xrow(r)] = rx[r];
          Ys[ykk(r)][ycol(r)] = ry[r];
        }
        __syncthreads();
        if (kb + kTileK < kn) fetch(kb + kTileK);
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
          const float2 xv = *reinterpret_cast<const float2*>(&Xs[kk][2 * ty]);
          const float4 yv = *reinterpret_cast<const float4*>(&Ys[kk][4 * tx]);
          const float xa[2] = {xv.x, xv.y}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a0[i][j] = fmaf(xa[i], ya[j], a0[i][j]);
        }
        if (++nblk == kTileRun) {
          fold();
          nblk = 0;
        }
      }
    }
    fold();
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t m = tm * kTile + 2 * ty + i, n = tn * kTile + 4 * tx + j;
        if (m >= M || n >= N) continue;
        const double v = (double)s[i][j] + (double)c[i][j];
        if (wk.nseg == 1) {  // one segment: the output itself
          store_output(static_cast<float*>(Cp[wk.item]) + offCm[2 * ty + i] + offCn[4 * tx + j], v,
                       alpha[wk.item], beta[wk.item]);
        } else {
          const uint64_t o = (uint64_t)m + (uint64_t)M * ((uint64_t)n + (uint64_t)N * b);
          partials[wk.slot + (int64_t)o * wk.nseg + wk.seg] = v;
        }
      }
  }
}

// C = alpha * (sum of an output's segments, in order) + beta * C.
__global__ void __launch_bounds__(kThreads) k_simt_final(
    const GemmArgs* __restrict__ items, const SimtFinal* __restrict__ fin, int64_t nfin,
    void* const* Cp, const double* alpha, const double* beta,
    const double* __restrict__ partials) {
  for (int64_t w = blockIdx.x; w < nfin; w += gridDim.x) {
    const SimtFinal f = fin[w];
    const GemmArgs& p = items[f.item];
    const uint64_t M = (uint64_t)p.M, N = (uint64_t)p.N;
    const uint64_t outs = M * N * (uint64_t)p.nbatch;
    const uint64_t o = (uint64_t)f.out0 + threadIdx.x;
    if (o >= outs) continue;
    const double* ps = partials + f.slot0 + (int64_t)threadIdx.x * f.nseg;
    double s = 0.0;
    for (int i = 0; i < f.nseg; ++i) s += ps[i];
    uint32_t m, n, b;
    split_output(o, M, N, outs, m, n, b);
    int64_t bX, bY, bC, oXm, oCm, oYn, oCn;
    goff3(p.gb, b, bX, bY, bC);
    goff2(p.gm, 0, 2, m, oXm, oCm);
    goff2(p.gn, 1, 2, n, oYn, oCn);
    store_output(static_cast<float*>(Cp[f.item]) + bC + oCm + oCn, s, alpha[f.item],
                 beta[f.item]);
  }
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * v.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  return e;
}

void free_batch(Batch* B) {
  if (!B) return;
  cudaFree(B->d_items);
  cudaFree(B->d_tc_work);
  cudaFree(B->d_simt_work);
  cudaFree(B->d_simt_tile);
  cudaFree(B->d_simt_final);
  cudaFree(B->d_partials);
  cudaFree(B->d_pk);
  cudaFree(B->d_pack);
  cudaFree(B->d_pkws);
  cudaFree(B->d_pkpart);
  cudaFree(B->d_red);
  if (B->join) cudaEventDestroy(B->join);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->side) cudaStreamDestroy(B->side);
  delete B;
}

int g_tc_min_mn = 64;

}  // namespace bat
}  // namespace tc

using namespace tc;
using namespace tc::bat;

extern "C" tc_status tc_batch_set_route(int32_t tc_min_mn) {
  if (tc_min_mn < 1) return TC_ERR_INVALID_ARG;
  g_tc_min_mn = tc_min_mn;
  return TC_OK;
}

extern "C" tc_status tc_batch_plan(tc_batch_t* out, const tc_plan_t* plans, int32_t n) {
  return tc_batch_plan_routes(out, plans, nullptr, n);
}

extern "C" tc_status tc_batch_plan_routes(tc_batch_t* out, const tc_plan_t* plans,
                                          const int32_t* routes, int32_t n) {
  if (!out || (!plans && n > 0) || n < 0) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<GemmArgs> items((size_t)n);
  std::vector<PkItem> pk((size_t)n);
  std::vector<size_t> pk_off((size_t)n, 0);   // packed operands of item i in the workspace
  std::vector<int32_t> pack;                   // (item, operand, row tile, 128-K chunk)
  size_t pk_bytes = 0;
  std::vector<std::pair<uint64_t, TcWork>> tcw;  // (cost, entry)
  std::vector<int32_t> tc_items;               // tensor-core items, in order
  int64_t tc_blocks = 0;                       // their tiles' 32-K blocks
  std::vector<int32_t> red;                    // split-K reductions (item, tile)
  size_t part_bytes = 0;
  std::vector<size_t> part_off((size_t)n, 0);
  std::vector<SimtWork> sw;
  std::vector<SimtTileWork> stw;
  std::vector<SimtFinal> sf;
  int64_t slots = 0;
  int32_t math = -1;
  double flops = 0, bytes = 0;
  int32_t ntc = 0, nsimt = 0;
  for (int32_t i = 0; i < n; ++i) {
    const Plan* P = reinterpret_cast<const Plan*>(plans[i]);
    if (!P) return TC_ERR_INVALID_ARG;
    if (P->dtype != TC_F32 || P->math < TC_MATH_BF16 || P->math > TC_MATH_BF16X6)
      return TC_ERR_UNSUPPORTED;
    if (math >= 0 && P->math != math) return TC_ERR_UNSUPPORTED;
    if (P->copy_which || P->empty_out || P->empty_k) return TC_ERR_UNSUPPORTED;
    math = P->math;
    GemmArgs a = P->args;
    a.swapped = P->swapped ? 1 : 0;
    a.chunk_kb = tc_chunk_kb(math, 0);
    if (a.chunk_kb % pk_stage_blocks(math) != 0) return TC_ERR_UNSUPPORTED;
    a.raster = 0;
    items[i] = a;
    flops += P->info.flops;
    bytes += P->info.min_bytes;
    const int32_t route = routes ? routes[i] : -1;
    if (route < -1 || route > 3) return TC_ERR_INVALID_ARG;
    if (route == 1 && a.nbatch != 1) return TC_ERR_UNSUPPORTED;
    const bool to_tc =
        route == 1 || (route == -1 && a.M >= g_tc_min_mn && a.N >= g_tc_min_mn && a.nbatch == 1);
    if (to_tc) {
      ++ntc;
      const PkLayout L = pk_layout(a, math);
      pk_off[i] = pk_bytes;
      pk_bytes += L.bytes;
      PkItem& it = pk[i];
      std::memset(&it, 0, sizeof(it));
      it.gm = a.gm;
      it.gn = a.gn;
      it.M = a.M;
      it.N = a.N;
      it.tiles_m = (int32_t)L.tiles_m;
      it.tiles_n = (int32_t)L.tiles_n;
      it.nkb = (int32_t)L.nkb;
      it.chunk_kb = a.chunk_kb;
      it.raster = 0;
      it.ksplit = 1;
      it.part = nullptr;
      it.qa = reinterpret_cast<const uint8_t*>(L.off_qa);   // offsets until allocation
      it.qb = reinterpret_cast<const uint8_t*>(L.off_qb);
      const int32_t npk = (int32_t)((L.nkb + 3) / 4);
      for (int32_t o = 0; o < 2; ++o)
        for (int32_t t = 0; t < (o ? L.tiles_n : L.tiles_m); ++t)
          for (int32_t kc = 0; kc < npk; ++kc) {
            pack.push_back(i);
            pack.push_back(o);
            pack.push_back(t);
            pack.push_back(kc);
          }
      tc_items.push_back(i);
      tc_blocks += (int64_t)L.tiles_m * L.tiles_n * L.nkb;
    } else {
      ++nsimt;
      const int64_t outs = a.M * a.N * a.nbatch;
      const int64_t K = a.K;
      // 32x32 tiles (route 2, or the rule for min(M, N) >= kTileMin); split K
      // when there are few
      const bool tiled = route == 2 || (route != 3 && std::min(a.M, a.N) >= kTileMin);
      if (tiled) {
        const int64_t tiles = ((a.M + kTile - 1) / kTile) * ((a.N + kTile - 1) / kTile) * a.nbatch;
        int64_t nseg = std::max<int64_t>(1, std::min<int64_t>((K + 511) / 512, 1216 / tiles));
        const int64_t KS = (K + nseg - 1) / nseg;
        nseg = (K + KS - 1) / KS;
        for (int64_t sg = 0; sg < nseg; ++sg)
          for (int64_t t = 0; t < tiles; ++t)
            stw.push_back(SimtTileWork{i, (int32_t)nseg, t, sg * KS, std::min(K, (sg + 1) * KS),
                                       slots, sg});
        if (nseg > 1) {  // one segment: the tiles write C themselves
          for (int64_t o0 = 0; o0 < outs; o0 += kThreads)
            sf.push_back(SimtFinal{i, (int32_t)nseg, o0, slots + o0 * nseg});
          slots += outs * nseg;
        }
      } else if (outs < kThreads) {  // a warp per output, 8 outputs per block, K segments
        const int64_t KS = std::max<int64_t>(2048, (K + 255) / 256);
        const int32_t nseg = (int32_t)((K + KS - 1) / KS);
        for (int64_t o = 0; o < outs; o += kThreads / 32)
          for (int32_t s = 0; s < nseg; ++s)
            sw.push_back(SimtWork{i, 1, o, s * KS, std::min(K, (s + 1) * KS),
                                  slots + o * nseg + s, nseg, 0});
        if (nseg > 1) {
          for (int64_t o0 = 0; o0 < outs; o0 += kThreads)
            sf.push_back(SimtFinal{i, nseg, o0, slots + o0 * nseg});
          slots += outs * nseg;
        }
      } else {  // a thread per output; split K when there are few output blocks
        const int64_t blocks = (outs + kThreads - 1) / kThreads;
        int64_t nseg = std::max<int64_t>(1, std::min<int64_t>((K + 255) / 256, 1216 / blocks));
        const int64_t KS = (K + nseg - 1) / nseg;
        nseg = (K + KS - 1) / KS;
        for (int64_t bl = 0; bl < blocks; ++bl) {
          for (int64_t s = 0; s < nseg; ++s)
            sw.push_back(SimtWork{i, 0, bl * kThreads, s * KS, std::min(K, (s + 1) * KS),
                                  slots + bl * kThreads * nseg + s, (int32_t)nseg, 0});
          if (nseg > 1)
            sf.push_back(SimtFinal{i, (int32_t)nseg, bl * kThreads, slots + bl * kThreads * nseg});
        }
        if (nseg > 1) slots += blocks * kThreads * nseg;
      }
    }
  }
  // Tensor-core work entries.  A tile whose K blocks exceed half of one SM's
  // share of the route's blocks is split into K ranges (each >= 16 blocks,
  // at most 64), so that no single long-K tile holds the launch up; the
  // ranges write FP32 (s, r) partial sums that a last kernel adds in order.
  const int64_t half_share = std::max<int64_t>(16, tc_blocks / (2 * 152));
  for (int32_t i : tc_items) {
    PkItem& it = pk[i];
    const int64_t t = (int64_t)it.tiles_m * it.tiles_n;
    int64_t ks = std::min<int64_t>({(it.nkb + half_share - 1) / half_share, it.nkb / 16, 64});
    const size_t pb = (size_t)t * kTcTile * kTcTile * sizeof(float2);
    if (ks > 1 && part_bytes + (size_t)ks * pb > ((size_t)256 << 20)) ks = 1;  // bounded partials
    if (ks < 1) ks = 1;
    it.ksplit = (int32_t)ks;
    if (ks > 1) {
      part_off[i] = part_bytes;
      part_bytes += (size_t)ks * pb;
      for (int64_t k = 0; k < t; ++k) {
        red.push_back(i);
        red.push_back((int32_t)k);
      }
    }
    for (int64_t sp = 0; sp < ks; ++sp) {
      const int64_t k0 = sp * it.nkb / ks, k1 = (sp + 1) * it.nkb / ks;
      const uint64_t cost = (uint64_t)(k1 - k0) + 2;
      for (int64_t k = 0; k < t; ++k) tcw.push_back({cost, TcWork{i, (int32_t)k, (int32_t)sp}});
    }
  }
  std::stable_sort(tcw.begin(), tcw.end(),
                   [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<TcWork> tw(tcw.size());
  for (size_t k = 0; k < tcw.size(); ++k) tw[k] = tcw[k].second;

  Batch* B = new (std::nothrow) Batch();
  if (!B) return TC_ERR_INVALID_ARG;
  std::memset(B, 0, sizeof(*B));
  B->n = n;
  B->math = math;
  B->flops = flops;
  B->min_bytes = bytes;
  B->n_tc_items = ntc;
  B->n_simt_items = nsimt;
  B->n_tc_work = (int64_t)tw.size();
  B->n_simt_work = (int64_t)sw.size();
  B->n_simt_tiles = (int64_t)stw.size();
  B->n_simt_final = (int64_t)sf.size();
  B->n_pack = (int64_t)(pack.size() / 4);
  if (pk_bytes > 0 && cudaMalloc(reinterpret_cast<void**>(&B->d_pkws), pk_bytes) != cudaSuccess) {
    free_batch(B);
    return TC_ERR_CUDA;
  }
  if (part_bytes > 0 &&
      cudaMalloc(reinterpret_cast<void**>(&B->d_pkpart), part_bytes) != cudaSuccess) {
    free_batch(B);
    return TC_ERR_CUDA;
  }
  for (int32_t i = 0; i < n; ++i)
    if (pk[i].nkb > 0) {  // tensor-core items: offsets -> device addresses
      pk[i].qa = B->d_pkws + pk_off[i] + reinterpret_cast<size_t>(pk[i].qa);
      pk[i].qb = B->d_pkws + pk_off[i] + reinterpret_cast<size_t>(pk[i].qb);
      if (pk[i].ksplit > 1)
        pk[i].part = B->d_pkpart + part_off[i] / sizeof(float2);
    }
  B->n_red = (int64_t)(red.size() / 2);
  if (upload(&B->d_items, items) != cudaSuccess || upload(&B->d_tc_work, tw) != cudaSuccess ||
      upload(&B->d_pk, pk) != cudaSuccess || upload(&B->d_pack, pack) != cudaSuccess ||
      upload(&B->d_simt_work, sw) != cudaSuccess || upload(&B->d_simt_tile, stw) != cudaSuccess ||
      upload(&B->d_simt_final, sf) != cudaSuccess || upload(&B->d_red, red) != cudaSuccess ||
      (slots > 0 && cudaMalloc(reinterpret_cast<void**>(&B->d_partials),
                               sizeof(double) * (size_t)slots) != cudaSuccess)) {
    free_batch(B);
    return TC_ERR_CUDA;
  }
  // both routes: the CUDA-core kernels run on a stream of the batch's own,
  // forked from and joined back to the caller's stream, beside the tensor-core
  // kernels (which leave most of each SM's threads idle)
  if (B->n_tc_work > 0 && B->n_simt_work + B->n_simt_tiles > 0 &&
      (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming) != cudaSuccess)) {
    free_batch(B);
    return TC_ERR_CUDA;
  }
  *out = reinterpret_cast<tc_batch_t>(B);
  return TC_OK;
}

extern "C" tc_status tc_batch_get_info(tc_batch_t batch, tc_batch_info* info) {
  if (!batch || !info) return TC_ERR_INVALID_ARG;
  const Batch* B = reinterpret_cast<const Batch*>(batch);
  info->n_items = B->n;
  info->math = B->math;
  info->n_tiles = B->n_tc_work;
  info->flops = B->flops;
  info->min_bytes = B->min_bytes;
  info->n_tc_items = B->n_tc_items;
  info->n_simt_items = B->n_simt_items;
  info->n_simt_work = B->n_simt_work;
  info->n_simt_tiles = B->n_simt_tiles;
  info->n_tc_split = B->n_red;
  return TC_OK;
}

extern "C" tc_status tc_contract_batched(tc_batch_t batch, const void* const* A,
                                         const void* const* B, void* const* C,
                                         const double* alpha, const double* beta, void* stream) {
  if (!batch) return TC_ERR_INVALID_ARG;
  const Batch* Bt = reinterpret_cast<const Batch*>(batch);
  if (Bt->n == 0) return TC_OK;
  if (!A || !B || !C || !alpha || !beta) return TC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStream_t ss = s;  // the CUDA-core route's stream
  if (Bt->side) {
    if (cudaEventRecord(Bt->fork, s) != cudaSuccess ||
        cudaStreamWaitEvent(Bt->side, Bt->fork, 0) != cudaSuccess)
      return TC_ERR_CUDA;
    ss = Bt->side;
  }
  if (Bt->n_tc_work > 0) {
    PkBatch pb;
    pb.items = Bt->d_items;
    pb.pk = Bt->d_pk;
    pb.pack_work = Bt->d_pack;
    pb.n_pack = Bt->n_pack;
    pb.work = reinterpret_cast<const int32_t*>(Bt->d_tc_work);
    pb.n_work = Bt->n_tc_work;
    pb.red = Bt->d_red;
    pb.n_red = Bt->n_red;
    tc_status st = launch_gemm_tc_packed_batch(pb, A, B, C, alpha, beta, Bt->math, stream);
    if (st != TC_OK) return st;
  }
  if (Bt->n_simt_work > 0) {
    const int g1 = (int)std::min<int64_t>(Bt->n_simt_work, 152 * 8);
    k_simt_partial<<<g1, kThreads, 0, ss>>>(Bt->d_items, Bt->d_simt_work, Bt->n_simt_work, A, B,
                                            C, alpha, beta, Bt->d_partials);
  }
  if (Bt->n_simt_tiles > 0) {
    const int g1 = (int)std::min<int64_t>(Bt->n_simt_tiles, 152 * 12);
    k_simt_tile<<<g1, kTileThreads, 0, ss>>>(Bt->d_items, Bt->d_simt_tile, Bt->n_simt_tiles, A, B,
                                         C, alpha, beta, Bt->d_partials);
  }
  if (Bt->n_simt_final > 0) {
    const int g2 = (int)std::min<int64_t>(Bt->n_simt_final, 152 * 8);
    k_simt_final<<<g2, kThreads, 0, ss>>>(Bt->d_items, Bt->d_simt_final, Bt->n_simt_final, C,
                                         alpha, beta, Bt->d_partials);
  }
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (Bt->side && (cudaEventRecord(Bt->join, Bt->side) != cudaSuccess ||
                   cudaStreamWaitEvent(s, Bt->join, 0) != cudaSuccess))
    return TC_ERR_CUDA;
  return TC_OK;
}

extern "C" tc_status tc_batch_destroy(tc_batch_t batch) {
  free_batch(reinterpret_cast<Batch*>(batch));
  return TC_OK;
}
