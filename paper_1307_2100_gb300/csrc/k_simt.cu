// k_simt.cu -- CUDA-core kernels: the plain FP64 (and FP32) GEMM over gathered
// index groups, GEMV, DOT, the permute kernel of the explicit COPY baseline,
// and C = beta * C.
//
// Every kernel addresses its operands through index groups (tc_internal.h):
// a group index is split column-major into its labels and each label adds
// idx * stride.  This is how one kernel serves every slicing of Sec. 2.4:
// the tile loaders gather the rows and columns of A and B wherever their
// strides put them, so no slice is ever copied (Sec. 3.1 F1 is avoided).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "groups.cuh"
#include "storage.cuh"
#include "tc_internal.h"

namespace tc {

// ---------------------------------------------------------------------------
// GEMM on the CUDA cores (storage type S, arithmetic in T: FP64 for FP64
// data, FP32 otherwise).  CTA tile TM x TN, K step TK, each thread a 4x4
// register tile (rows ty + i*TM/4, columns tx + j*TN/4).  Tiles are taken in
// the order (m-tile fastest, n-tile, batch).  The next K block is fetched into
// registers while the current one is multiplied.  With p.ksplit > 1 (FP64,
// fewer tiles than SMs) the work entries are (K range, tile), K ranges
// slowest; each writes its partial tile [TM][TN] to the workspace and
// k_simt_reduce adds the ranges in order.
// ---------------------------------------------------------------------------
template <typename S, int TM, int TN, int TK>
__global__ void __launch_bounds__((TM / 4) * (TN / 4))
    k_gemm_simt(const __grid_constant__ GemmArgs p) {
  using T = typename Cmp<S>::T;
  constexpr int NT = (TM / 4) * (TN / 4);
  constexpr int LA = (TM * TK + NT - 1) / NT;  // A elements loaded per thread
  constexpr int LB = (TN * TK + NT - 1) / NT;
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  __shared__ int64_t offAm[TM], offCm[TM], offBn[TN], offCn[TN];
  __shared__ int64_t offAk[2][TK], offBk[2][TK];

  const S* __restrict__ A = static_cast<const S*>(p.A);
  const S* __restrict__ B = static_cast<const S*>(p.B);
  S* __restrict__ C = static_cast<S*>(p.C);
  const int tid = threadIdx.x;
  const int tx = tid % (TN / 4), ty = tid / (TN / 4);
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
  const uint32_t tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN;
  const uint64_t total = (uint64_t)tiles_m * tiles_n * (uint64_t)p.nbatch;
  const int ksplit = max(p.ksplit, 1);
  const uint32_t nkb_all = (K + TK - 1) / TK;

  for (uint64_t wk = blockIdx.x; wk < total * (uint64_t)ksplit; wk += gridDim.x) {
    const uint64_t tile = wk % total;
    const uint32_t split = (uint32_t)(wk / total);
    // K blocks [kb0, kb1) of this range (balanced, none empty)
    const uint32_t kb0 = (uint32_t)((uint64_t)split * nkb_all / ksplit);
    const uint32_t kb1 = (uint32_t)((uint64_t)(split + 1) * nkb_all / ksplit);
    const uint32_t tm = (uint32_t)(tile % tiles_m);
    const uint64_t rest = tile / tiles_m;
    const uint32_t tn = (uint32_t)(rest % tiles_n);
    const uint32_t b = (uint32_t)(rest / tiles_n);
    int64_t bA, bB, bC;
    goff3(p.gb, b, bA, bB, bC);

    __syncthreads();  // previous tile's epilogue is done with the offset tables
    for (int i = tid; i < TM; i += NT) {
      uint32_t m = tm * TM + i;
      int64_t oa = -1, oc = 0;
      if (m < M) goff2(p.gm, 0, 2, m, oa, oc);
      offAm[i] = oa;
      offCm[i] = oc;
    }
    for (int i = tid; i < TN; i += NT) {
      uint32_t n = tn * TN + i;
      int64_t ob = -1, oc = 0;
      if (n < N) goff2(p.gn, 1, 2, n, ob, oc);
      offBn[i] = ob;
      offCn[i] = oc;
    }
    auto k_offsets = [&](int buf, uint32_t k0) {
      for (int i = tid; i < TK; i += NT) {
        uint32_t k = k0 + i;
        int64_t oa = -1, ob = -1;
        if (k < K) goff2(p.gk, 0, 1, k, oa, ob);
        offAk[buf][i] = oa;
        offBk[buf][i] = ob;
      }
    };
    k_offsets(0, kb0 * TK);
    __syncthreads();

    T ra[LA], rb[LB];
    auto fetch = [&](int buf) {
#pragma unroll
      for (int r = 0; r < LA; ++r) {
        int e = tid + r * NT;
        int ml, kl;
        if (p.a_contig == CONTIG_MN) { ml = e % TM; kl = e / TM; }
        else { kl = e % TK; ml = e / TK; }
        T v = T(0);
        if (kl < TK && ml < TM) {
          int64_t om = offAm[ml], ok = offAk[buf][kl];
          if (om >= 0 && ok >= 0) v = ld_c(A[bA + om + ok]);
        }
        ra[r] = v;
      }
#pragma unroll
      for (int r = 0; r < LB; ++r) {
        int e = tid + r * NT;
        int nl, kl;
        if (p.b_contig == CONTIG_MN) { nl = e % TN; kl = e / TN; }
        else { kl = e % TK; nl = e / TK; }
        T v = T(0);
        if (kl < TK && nl < TN) {
          int64_t on = offBn[nl], ok = offBk[buf][kl];
          if (on >= 0 && ok >= 0) v = ld_c(B[bB + on + ok]);
        }
        rb[r] = v;
      }
    };
    auto stash = [&]() {
#pragma unroll
      for (int r = 0; r < LA; ++r) {
        int e = tid + r * NT;
        int ml, kl;
        if (p.a_contig == CONTIG_MN) { ml = e % TM; kl = e / TM; }
        else { kl = e % TK; ml = e / TK; }
        if (kl < TK && ml < TM) As[kl][ml] = ra[r];
      }
#pragma unroll
      for (int r = 0; r < LB; ++r) {
        int e = tid + r * NT;
        int nl, kl;
        if (p.b_contig == CONTIG_MN) { nl = e % TN; kl = e / TN; }
        else { kl = e % TK; nl = e / TK; }
        if (kl < TK && nl < TN) Bs[kl][nl] = rb[r];
      }
    };

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    if (kb0 < kb1) fetch(0);
    for (uint32_t kb = kb0; kb < kb1; ++kb) {
      const int buf = (kb - kb0) & 1;
      __syncthreads();  // everyone is done reading As/Bs of the previous block
      stash();
      if (kb + 1 < kb1) k_offsets(buf ^ 1, (kb + 1) * TK);
      __syncthreads();
      if (kb + 1 < kb1) fetch(buf ^ 1);
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        T a[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + i * (TM / 4)];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + j * (TN / 4)];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
      }
    }

    if (ksplit > 1) {  // partial tile of this K range
      T* part = static_cast<T*>(p.ws) + (split * total + tile) * (uint64_t)(TM * TN);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          part[(ty + i * (TM / 4)) * TN + tx + j * (TN / 4)] = acc[i][j];
      continue;
    }
    const T alpha = (T)p.alpha, beta = (T)p.beta;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ml = ty + i * (TM / 4);
      if (offAm[ml] < 0) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nl = tx + j * (TN / 4);
        if (offBn[nl] < 0) continue;
        S* dst = C + bC + offCm[ml] + offCn[nl];
        T v = alpha * acc[i][j];
        if (p.beta != 0.0) v = fma(beta, ld_c(*dst), v);
        *dst = st_any<S>(v);
      }
    }
  }
}

struct SimtTile { int tm, tn; };
// Tile configurations 0-3.  16 x 16 tiles (16 threads: half-filled warps)
// are a candidate of the FP64 selector for small GEMMs; the planner's default
// is 64 x 64 or 32 x 32.
static const SimtTile kSimtTiles[] = {{64, 64}, {32, 32}, {128, 64}, {16, 16}};
int num_tiles_simt(tc_dtype) { return 4; }

static int grid_for(uint64_t total) {
  return (int)std::min<uint64_t>(total, (uint64_t)1 << 30);
}

// Split-K: C = alpha * (sum of the K ranges' partial tiles, in order) + beta * C.
template <typename S, int TM, int TN>
__global__ void __launch_bounds__(256) k_simt_reduce(const __grid_constant__ GemmArgs p) {
  using T = typename Cmp<S>::T;
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N;
  const uint32_t tiles_m = (M + TM - 1) / TM, tiles_n = (N + TN - 1) / TN;
  const uint64_t total = (uint64_t)tiles_m * tiles_n * (uint64_t)p.nbatch;
  const uint64_t elems = total * (uint64_t)(TM * TN);
  const T* part = static_cast<const T*>(p.ws);
  S* C = static_cast<S*>(p.C);
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < elems;
       e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t tile = e / (TM * TN);
    const int ml = (int)((e / TN) % TM), nl = (int)(e % TN);
    const uint32_t tm = (uint32_t)(tile % tiles_m);
    const uint64_t rest = tile / tiles_m;
    const uint32_t tn = (uint32_t)(rest % tiles_n), b = (uint32_t)(rest / tiles_n);
    const uint32_t m = tm * TM + ml, n = tn * TN + nl;
    if (m >= M || n >= N) continue;
    T t = T(0);
    for (int sp = 0; sp < p.ksplit; ++sp) t += part[(uint64_t)sp * elems + e];
    int64_t bA, bB, bC;
    goff3(p.gb, b, bA, bB, bC);
    S* dst = C + bC + goff(p.gm, 2, m) + goff(p.gn, 2, n);
    T v = (T)p.alpha * t;
    if (p.beta != 0.0) v = fma((T)p.beta, ld_c(*dst), v);
    *dst = st_any<S>(v);
  }
}

// FP64 split-K: with fewer 64 x 64 tiles than SMs and a long K, at most two
// (K range, tile) entries per SM (two CTAs of 256 threads fit one SM), so that
// they run in one wave, each of at least 512 K (32 blocks of 16).
int simt_ksplit(const GemmArgs& a, tc_dtype dt, int tile) {
  if (dt != TC_F64 || tile != 0) return 1;
  const int64_t tiles = ((a.M + 63) / 64) * ((a.N + 63) / 64) * std::max<int64_t>(a.nbatch, 1);
  const int64_t nkb = (a.K + 15) / 16;
  if (tiles <= 0 || tiles >= 152) return 1;
  const int64_t want = (2 * 152) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, nkb / 32, 64}));
}

size_t simt_part_bytes(const GemmArgs& a, tc_dtype dt, int tile) {
  const int sp = simt_ksplit(a, dt, tile);
  if (sp <= 1) return 0;
  const int64_t tiles = ((a.M + 63) / 64) * ((a.N + 63) / 64) * std::max<int64_t>(a.nbatch, 1);
  return (size_t)sp * (size_t)tiles * 64 * 64 * sizeof(double);
}

template <typename T>  // the storage type
static tc_status gemm_simt_t(const GemmArgs& a, int tile, cudaStream_t s) {
  const SimtTile t = kSimtTiles[tile];
  const uint64_t total = (uint64_t)((a.M + t.tm - 1) / t.tm) * (uint64_t)((a.N + t.tn - 1) / t.tn) *
                         (uint64_t)a.nbatch;
  if (total == 0) return TC_OK;
  const int ksplit = std::max(a.ksplit, 1);
  if (ksplit > 1 && (!a.ws || t.tm != 64 || t.tn != 64)) return TC_ERR_WORKSPACE;
  const int grid = grid_for(total * (uint64_t)ksplit);
  if (t.tm == 64 && t.tn == 64)
    k_gemm_simt<T, 64, 64, 16><<<grid, 256, 0, s>>>(a);
  else if (t.tm == 32 && t.tn == 32)
    k_gemm_simt<T, 32, 32, 16><<<grid, 64, 0, s>>>(a);
  else if (t.tm == 16 && t.tn == 16)
    k_gemm_simt<T, 16, 16, 16><<<grid, 16, 0, s>>>(a);
  else
    k_gemm_simt<T, 128, 64, 16><<<grid, 512, 0, s>>>(a);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (ksplit > 1) {
    const uint64_t elems = total * 64 * 64;
    k_simt_reduce<T, 64, 64><<<grid_for(std::min<uint64_t>((elems + 255) / 256, 152 * 16)), 256,
                               0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

tc_status launch_gemm_simt(const GemmArgs& a, tc_dtype dt, int tile, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dt) {
    case TC_F64: return gemm_simt_t<double>(a, tile, s);
    case TC_F32: return gemm_simt_t<float>(a, tile, s);
    case TC_BF16: return gemm_simt_t<__nv_bfloat16>(a, tile, s);
    case TC_F16: return gemm_simt_t<__half>(a, tile, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

// Accumulators of the GEMV/DOT kernels.  FP64 data accumulate in FP64; FP32
// data accumulate with Neumaier's compensated summation (sum + running error,
// both FP32), so long K does not lose FP32-class accuracy.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float a, float b) {
    const float x = __fmul_rn(a, b);
    const float t = __fadd_rn(s, x);
    if (fabsf(s) >= fabsf(x)) c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
    else c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------------------
// GEMV (Sec. 3.2.2): y[m, n, b] = alpha * sum_k X[m, k, b] * Y[k, n, b] + beta*y.
// When X is contiguous along m (non-transposed GEMV) each thread owns one m and
// walks k, consecutive threads reading consecutive addresses; when X is
// contiguous along k (transposed GEMV) each warp owns one output and its lanes
// walk k, reduced with warp shuffles.  The k offsets of X and Y are staged in
// shared memory in chunks.
// ---------------------------------------------------------------------------
constexpr int kGemvThreads = 256;
constexpr int kGemvChunk = 512;

template <typename S>
__global__ void __launch_bounds__(kGemvThreads) k_gemv_m(const __grid_constant__ GemmArgs p) {
  using T = typename Cmp<S>::T;
  __shared__ int64_t oX[kGemvChunk], oY[kGemvChunk];
  const S* __restrict__ X = static_cast<const S*>(p.A);
  const S* __restrict__ Y = static_cast<const S*>(p.B);
  S* __restrict__ Cp = static_cast<S*>(p.C);
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
  const uint64_t mblocks = (M + kGemvThreads - 1) / kGemvThreads;
  const uint64_t total = mblocks * (uint64_t)N * (uint64_t)p.nbatch;
  for (uint64_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
    const uint32_t m = (uint32_t)(blk % mblocks) * kGemvThreads + threadIdx.x;
    const uint64_t nb = blk / mblocks;  // (n, b) pair
    const uint32_t n = (uint32_t)(nb % N), b = (uint32_t)(nb / N);
    int64_t bX, bY, bC, oYn, oCn, oXm = 0, oCm = 0;
    goff3(p.gb, b, bX, bY, bC);
    goff2(p.gn, 1, 2, n, oYn, oCn);
    if (m < M) goff2(p.gm, 0, 2, m, oXm, oCm);
    const S* xrow = X + bX + oXm;
    const S* yv = Y + bY + oYn;
    Acc<T> acc;
    for (uint32_t k0 = 0; k0 < K; k0 += kGemvChunk) {
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < kGemvChunk; i += kGemvThreads) {
        uint32_t k = k0 + i;
        int64_t ox = 0, oy = 0;
        if (k < K) goff2(p.gk, 0, 1, k, ox, oy);
        oX[i] = ox;
        oY[i] = oy;
      }
      __syncthreads();
      const uint32_t kn = min((uint32_t)kGemvChunk, K - k0);
      if (m < M) {
        uint32_t i = 0;
        for (; i + 8 <= kn; i += 8) {
          T xv[8], yy[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) xv[u] = ld_c(xrow[oX[i + u]]);
#pragma unroll
          for (int u = 0; u < 8; ++u) yy[u] = ld_c(yv[oY[i + u]]);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc.add(xv[u], yy[u]);
        }
        for (; i < kn; ++i) acc.add(ld_c(xrow[oX[i]]), ld_c(yv[oY[i]]));
      }
    }
    if (m < M) {
      S* dst = Cp + bC + oCm + oCn;
      double v = p.alpha * acc.value();
      if (p.beta != 0.0) v += p.beta * (double)ld_c(*dst);
      *dst = st_c<S>(v);
    }
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per output (m, n, b); lanes stride over k.  Used by the transposed
// GEMV and by the DOT mapping (Sec. 3.2.1: one inner product per output).
template <typename S>
__global__ void __launch_bounds__(256) k_dot_rows(const __grid_constant__ GemmArgs p) {
  using T = typename Cmp<S>::T;
  const S* __restrict__ X = static_cast<const S*>(p.A);
  const S* __restrict__ Y = static_cast<const S*>(p.B);
  S* __restrict__ Cp = static_cast<S*>(p.C);
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
  const uint64_t total = (uint64_t)M * N * (uint64_t)p.nbatch;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t w = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); w < total;
       w += warps) {
    const uint32_t m = (uint32_t)(w % M);
    const uint64_t r = w / M;
    const uint32_t n = (uint32_t)(r % N), b = (uint32_t)(r / N);
    int64_t bX, bY, bC, oXm, oCm, oYn, oCn;
    goff3(p.gb, b, bX, bY, bC);
    goff2(p.gm, 0, 2, m, oXm, oCm);
    goff2(p.gn, 1, 2, n, oYn, oCn);
    const S* xr = X + bX + oXm;
    const S* yr = Y + bY + oYn;
    Acc<T> acc;
    for (uint32_t k = lane; k < K; k += 32) {
      int64_t ox, oy;
      goff2(p.gk, 0, 1, k, ox, oy);
      acc.add(ld_c(xr[ox]), ld_c(yr[oy]));
    }
    const double tot = warp_sum(acc.value());
    if (lane == 0) {
      S* dst = Cp + bC + oCm + oCn;
      double v = p.alpha * tot;
      if (p.beta != 0.0) v += p.beta * (double)ld_c(*dst);
      *dst = st_c<S>(v);
    }
  }
}

int num_tiles_gemv() { return 1; }

template <typename T>
static tc_status gemv_t(const GemmArgs& a, cudaStream_t s) {
  const uint64_t outs = (uint64_t)a.N * (uint64_t)a.nbatch;
  if (a.M == 0 || outs == 0) return TC_OK;
  if (a.a_contig == CONTIG_K) {
    const uint64_t warps = (uint64_t)a.M * outs;
    const int grid = grid_for((warps + 7) / 8);
    k_dot_rows<T><<<grid, 256, 0, s>>>(a);
  } else {
    const uint64_t blocks = (uint64_t)((a.M + kGemvThreads - 1) / kGemvThreads) * outs;
    k_gemv_m<T><<<grid_for(blocks), kGemvThreads, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_gemv(const GemmArgs& a, tc_dtype dt, int, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dt) {
    case TC_F64: return gemv_t<double>(a, s);
    case TC_F32: return gemv_t<float>(a, s);
    case TC_BF16: return gemv_t<__nv_bfloat16>(a, s);
    case TC_F16: return gemv_t<__half>(a, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------
// GER: rank-K update for K <= TC_GER_MAX_K (the sum-of-GERs slicing of Sec. 2.2
// done in one pass).  A CTA owns 256 rows of C and a chunk of its columns:
// each thread loads its row's K values of the first operand into registers
// once, then for every 32 columns of the chunk the CTA stages their K values
// of the second operand in shared memory and each thread writes its 32
// outputs (consecutive threads on consecutive rows, the planner's choice of
// C's stride-1 index).  KB, the register width, is K rounded up to 4, 8, 16
// or 32 (zero-padded).
// ---------------------------------------------------------------------------
constexpr int kGerThreads = 256, kGerN = 32;

template <typename S, int KB>
__global__ void __launch_bounds__(kGerThreads) k_ger(const __grid_constant__ GemmArgs p,
                                                     uint32_t tiles_per_chunk) {
  using T = typename Cmp<S>::T;
  __shared__ T sB[KB][kGerN];
  __shared__ int64_t sC[kGerN];
  const S* __restrict__ X = static_cast<const S*>(p.A);
  const S* __restrict__ Y = static_cast<const S*>(p.B);
  S* __restrict__ Cp = static_cast<S*>(p.C);
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
  const uint32_t mb = (M + kGerThreads - 1) / kGerThreads, nt = (N + kGerN - 1) / kGerN;
  const uint32_t nchunks = (nt + tiles_per_chunk - 1) / tiles_per_chunk;
  const T alpha = (T)p.alpha, beta = (T)p.beta;
  const int tid = threadIdx.x;
  for (uint64_t w = blockIdx.x; w < (uint64_t)mb * nchunks * (uint64_t)p.nbatch;
       w += gridDim.x) {
    const uint32_t bm = (uint32_t)(w % mb);
    const uint64_t r = w / mb;
    const uint32_t ch = (uint32_t)(r % nchunks), b = (uint32_t)(r / nchunks);
    int64_t bX, bY, bC;
    goff3(p.gb, b, bX, bY, bC);
    const uint32_t m = bm * kGerThreads + tid;
    const bool row_ok = m < M;
    int64_t oxm = 0, ocm = 0;
    if (row_ok) goff2(p.gm, 0, 2, m, oxm, ocm);
    T a[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k)
      a[k] = (row_ok && k < (int)K) ? ld_c(X[bX + oxm + goff(p.gk, 0, (uint32_t)k)]) : T(0);
    S* Crow = Cp + bC + ocm;
    const uint32_t t_end = min(nt, (ch + 1) * tiles_per_chunk);
    for (uint32_t bn = ch * tiles_per_chunk; bn < t_end; ++bn) {
      __syncthreads();  // the previous columns' shared values are no longer read
      for (int i = tid; i < KB * kGerN; i += kGerThreads) {
        const int k = i / kGerN, j = i % kGerN;
        const uint32_t n = bn * kGerN + j;
        T v = T(0);
        if (k < (int)K && n < N) v = ld_c(Y[bY + goff(p.gn, 1, n) + goff(p.gk, 1, (uint32_t)k)]);
        sB[k][j] = v;
      }
      if (tid < kGerN) {
        const uint32_t n = bn * kGerN + tid;
        sC[tid] = n < N ? goff(p.gn, 2, n) : -1;
      }
      __syncthreads();
      if (!row_ok) continue;
#pragma unroll 4
      for (int j = 0; j < kGerN; ++j) {
        const int64_t cj = sC[j];
        if (cj < 0) break;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < KB; ++k) acc = fma(a[k], sB[k][j], acc);
        // alpha and beta in the storage precision (FP64 is the slow pipe on
        // this GPU: FP32 outputs stay in FP32)
        T v = alpha * acc;
        if (beta != T(0)) v = fma(beta, ld_c(Crow[cj]), v);
        Crow[cj] = st_any<S>(v);
      }
    }
  }
}

template <typename T>  // the storage type
static tc_status ger_t(const GemmArgs& a, cudaStream_t s) {
  const uint64_t mb = (uint64_t)((a.M + kGerThreads - 1) / kGerThreads) * (uint64_t)a.nbatch;
  const uint64_t nt = (uint64_t)((a.N + kGerN - 1) / kGerN);
  if (mb == 0 || nt == 0) return TC_OK;
  // enough CTAs for 8 per SM, each over as many column tiles as that leaves
  const uint64_t want_chunks = std::max<uint64_t>(1, (152 * 8 + mb - 1) / mb);
  const uint32_t tpc = (uint32_t)std::max<uint64_t>(1, (nt + want_chunks - 1) / want_chunks);
  const uint64_t ctas = mb * ((nt + tpc - 1) / tpc);
  const int grid = (int)std::min<uint64_t>(ctas, 152 * 16);
  if (a.K <= 4) k_ger<T, 4><<<grid, kGerThreads, 0, s>>>(a, tpc);
  else if (a.K <= 8) k_ger<T, 8><<<grid, kGerThreads, 0, s>>>(a, tpc);
  else if (a.K <= 16) k_ger<T, 16><<<grid, kGerThreads, 0, s>>>(a, tpc);
  else if (a.K <= TC_GER_MAX_K) k_ger<T, TC_GER_MAX_K><<<grid, kGerThreads, 0, s>>>(a, tpc);
  else return TC_ERR_UNSUPPORTED;
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_ger(const GemmArgs& a, tc_dtype dt, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dt) {
    case TC_F64: return ger_t<double>(a, s);
    case TC_F32: return ger_t<float>(a, s);
    case TC_BF16: return ger_t<__nv_bfloat16>(a, s);
    case TC_F16: return ger_t<__half>(a, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------
// DOT.  Many outputs: one warp each (k_dot_rows).  A single output (Class 1,
// Sec. 3.2.1: all indices contracted, a scalar result): every CTA sums a
// grid-strided share of k into one partial in the workspace, then one CTA adds
// the partials in index order (deterministic) and applies alpha and beta.
// ---------------------------------------------------------------------------
constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 152 * 4;

int dot_partials(const GemmArgs&, int) { return kDotBlocks; }

// `part` receives one FP64 partial per CTA: the plan's workspace, or the
// library's built-in scratch array for tc_contract_dot_noalloc.
template <typename S>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const __grid_constant__ GemmArgs p,
                                                             double* __restrict__ part) {
  __shared__ double red[kDotThreads / 32];
  const S* __restrict__ X = static_cast<const S*>(p.A);
  const S* __restrict__ Y = static_cast<const S*>(p.B);
  const uint32_t K = (uint32_t)p.K;
  double acc = 0.0;
  const uint32_t stride = gridDim.x * kDotThreads;
  for (uint32_t k = blockIdx.x * kDotThreads + threadIdx.x; k < K; k += stride) {
    int64_t ox, oy;
    goff2(p.gk, 0, 1, k, ox, oy);
    acc = fma((double)ld_c(X[ox]), (double)ld_c(Y[oy]), acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

template <typename S>
__global__ void k_dot_final(const __grid_constant__ GemmArgs p, const double* __restrict__ part,
                            int nparts) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    S* dst = static_cast<S*>(p.C);
    double v = p.alpha * t;
    if (p.beta != 0.0) v += p.beta * (double)ld_c(*dst);
    *dst = st_c<S>(v);
  }
}

template <typename T>
static void dot_scalar_t(const GemmArgs& a, double* part, cudaStream_t s) {
  k_dot_partial<T><<<kDotBlocks, kDotThreads, 0, s>>>(a, part);
  k_dot_final<T><<<1, 256, 0, s>>>(a, part, kDotBlocks);
}

tc_status launch_dot_scalar(const GemmArgs& a, tc_dtype dt, double* part, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dt) {
    case TC_F64: dot_scalar_t<double>(a, part, s); break;
    case TC_F32: dot_scalar_t<float>(a, part, s); break;
    case TC_BF16: dot_scalar_t<__nv_bfloat16>(a, part, s); break;
    case TC_F16: dot_scalar_t<__half>(a, part, s); break;
    default: return TC_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

template <typename T>
static tc_status dot_t(const GemmArgs& a, cudaStream_t s) {
  const uint64_t outs = (uint64_t)a.M * a.N * (uint64_t)a.nbatch;
  if (outs == 0) return TC_OK;
  if (outs == 1) {
    if (!a.ws) return TC_ERR_WORKSPACE;
    dot_scalar_t<T>(a, static_cast<double*>(a.ws), s);
  } else {
    k_dot_rows<T><<<grid_for((outs + 7) / 8), 256, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_dot(const GemmArgs& a, tc_dtype dt, int, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dt) {
    case TC_F64: return dot_t<double>(a, s);
    case TC_F32: return dot_t<float>(a, s);
    case TC_BF16: return dot_t<__nv_bfloat16>(a, s);
    case TC_F16: return dot_t<__half>(a, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------
// Permute (the COPY of Sec. 3.1 F1, kept as the explicit baseline).  The
// output is dense in the group's label order.  When the input's fastest label
// is not the output's first label the copy is a tiled transpose: a 32x32 tile
// over (output-first label, input-fastest label) goes through shared memory
// so that both the reads and the writes are coalesced.
// ---------------------------------------------------------------------------
// Wide: the tensor has 2^31 or more elements, so its flat index is split in
// 64 bits (a 32-bit split would wrap and leave elements unwritten).
template <typename T, bool Wide>
__global__ void __launch_bounds__(256) k_perm_direct(const __grid_constant__ PermArgs p) {
  const T* __restrict__ in = static_cast<const T*>(p.in);
  T* __restrict__ out = static_cast<T*>(p.out);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < (uint64_t)p.total;
       q += stride) {
    int64_t oi, oo;
    if (Wide) {
      oi = goff_wide(p.g, 0, q);
      oo = goff_wide(p.g, 2, q);
    } else {
      goff2(p.g, 0, 2, (uint32_t)q, oi, oo);
    }
    out[oo] = in[oi];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_perm_tiled(const __grid_constant__ PermArgs p, int li,
                                                    uint64_t rest_total) {
  __shared__ T tile[32][33];
  const T* __restrict__ in = static_cast<const T*>(p.in);
  T* __restrict__ out = static_cast<T*>(p.out);
  const uint32_t e0 = (uint32_t)p.g.ext[0], e1 = (uint32_t)p.g.ext[li];
  const uint32_t t0n = (e0 + 31) / 32, t1n = (e1 + 31) / 32;
  const uint64_t ntiles = (uint64_t)t0n * t1n * rest_total;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t t0 = (uint32_t)(t % t0n);
    const uint64_t r1 = t / t0n;
    const uint32_t t1 = (uint32_t)(r1 % t1n);
    uint64_t rest = r1 / t1n;  // once per 32x32 tile: 64-bit division is cheap here
    int64_t bi = 0, bo = 0;
    for (int i = 1; i < p.g.n; ++i) {  // the other labels, column-major
      if (i == li) continue;
      const uint64_t e = (uint64_t)p.g.ext[i];
      const uint64_t q = rest / e, r = rest - q * e;
      bi += (int64_t)r * p.g.st[0][i];
      bo += (int64_t)r * p.g.st[2][i];
      rest = q;
    }
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; r += 8) {
      uint32_t a1 = t1 * 32 + tx, a0 = t0 * 32 + ty + r;  // read: lanes along label li
      if (a1 < e1 && a0 < e0)
        tile[ty + r][tx] = in[bi + (int64_t)a1 * p.g.st[0][li] + (int64_t)a0 * p.g.st[0][0]];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; r += 8) {
      uint32_t a0 = t0 * 32 + tx, a1 = t1 * 32 + ty + r;  // write: lanes along label 0
      if (a0 < e0 && a1 < e1)
        out[bo + (int64_t)a0 * p.g.st[2][0] + (int64_t)a1 * p.g.st[2][li]] = tile[tx][ty + r];
    }
  }
}

template <typename T>
static tc_status perm_t(const PermArgs& a, cudaStream_t s) {
  if (a.total == 0) return TC_OK;
  int li = 0;
  for (int i = 1; i < a.g.n; ++i)
    if (a.g.st[0][i] < a.g.st[0][li]) li = i;
  if (li == 0 || a.g.st[0][li] != 1) {
    const int grid = grid_for(std::min<uint64_t>((a.total + 255) / 256, 152 * 64));
    if (a.total >= ((int64_t)1 << 31))
      k_perm_direct<T, true><<<grid, 256, 0, s>>>(a);
    else
      k_perm_direct<T, false><<<grid, 256, 0, s>>>(a);
  } else {
    uint64_t rest = 1;
    for (int i = 1; i < a.g.n; ++i)
      if (i != li) rest *= (uint64_t)a.g.ext[i];
    const uint64_t ntiles = ((a.g.ext[0] + 31) / 32) * ((a.g.ext[li] + 31) / 32) * rest;
    k_perm_tiled<T><<<grid_for(std::min<uint64_t>(ntiles, 152 * 64)), 256, 0, s>>>(a, li, rest);
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_perm(const PermArgs& a, tc_dtype dt, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (elem_size(dt)) {  // a permute moves bits: one instantiation per size
    case 8: return perm_t<uint64_t>(a, s);
    case 4: return perm_t<uint32_t>(a, s);
    case 2: return perm_t<uint16_t>(a, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

// C = beta * C over C's own labels (empty contraction or alpha == 0).
// Wide: C has 2^31 or more elements (index split in 64 bits, as in k_perm_direct).
template <typename S, bool Wide>
__global__ void k_scale(const __grid_constant__ Group g, S* C, double beta, uint64_t total) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < total; q += stride) {
    S* dst = C + (Wide ? goff_wide(g, 2, q) : goff(g, 2, (uint32_t)q));
    *dst = st_c<S>(beta == 0.0 ? 0.0 : beta * (double)ld_c(*dst));
  }
}

template <typename S>
static void scale_t(const Group& gc, void* C, double beta, int64_t total, bool wide, int grid,
                    cudaStream_t s) {
  S* c = static_cast<S*>(C);
  if (wide) k_scale<S, true><<<grid, 256, 0, s>>>(gc, c, beta, (uint64_t)total);
  else k_scale<S, false><<<grid, 256, 0, s>>>(gc, c, beta, (uint64_t)total);
}

tc_status launch_scale(const Group& gc, void* C, double beta, tc_dtype dt, int64_t total,
                       void* stream) {
  if (total <= 0) return TC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = grid_for(std::min<uint64_t>((total + 255) / 256, 152 * 32));
  const bool wide = total >= ((int64_t)1 << 31);
  switch (dt) {
    case TC_F64: scale_t<double>(gc, C, beta, total, wide, grid, s); break;
    case TC_F32: scale_t<float>(gc, C, beta, total, wide, grid, s); break;
    case TC_BF16: scale_t<__nv_bfloat16>(gc, C, beta, total, wide, grid, s); break;
    case TC_F16: scale_t<__half>(gc, C, beta, total, wide, grid, s); break;
    default: return TC_ERR_UNSUPPORTED;
  }
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

}  // namespace tc
