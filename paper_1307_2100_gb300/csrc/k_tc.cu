// k_tc.cu -- the tensor-core GEMM over gathered index groups (sm_103a, tcgen05),
// for one contraction or a batch of contractions in one persistent launch.
//
// C[m, n, b] = alpha * sum_k A[m, k, b] * B[k, n, b] + beta * C[m, n, b] for
// FP32 tensors of any layout, computed as a sum of BF16 products:
//   BF16    a0 b0                                (1 term per operand)
//   BF16x3  a0 b0 + a0 b1 + a1 b0                 (2 terms)
//   BF16x6  + a0 b2 + a1 b1 + a2 b0               (3 terms)
// with x = x0 + x1 + x2 the split of an FP32 value into BF16 terms, each the
// round-to-nearest-even BF16 value of the remaining residual.
//
// Accuracy.  The tensor cores add each 16-product block into the FP32
// accumulator without rounding to nearest (the error grows with the number of
// additions, not with its square root), so the main product a0 b0 and the
// small correction products go to separate accumulators, and the main
// accumulator is emptied every K-chunk (256 K by default): the chunks are
// summed in compensated FP32 (TwoSum; the high word in tensor memory, the low
// word in registers) and the final sum hi + lo + corrections is formed in FP64.
//
// One CTA per SM, persistent over a work list of 128 x 128 output tiles.
// Warp roles (416 threads):
//   warps 0-3   producers: read FP32 elements of A and B through the index
//               groups (any strides: the permutation of a Class 3.1 operand is
//               absorbed here, so no copy pass touches HBM), split them into
//               BF16 terms in registers, store the terms to shared memory in the
//               canonical K-major layout of the tensor cores;
//   warps 4-11  epilogue: two warps per tensor-memory lane quadrant, 64 columns
//               each; drain K-chunks, finish with alpha/beta and a strided store;
//   warp 12     tensor-memory allocation and the single thread issuing
//               tcgen05.mma.
// Tensor memory (512 columns x 128 lanes): [0,128) and [128,256) the double
// buffered main accumulator, [256,384) the correction accumulator, [384,512)
// the high word of the compensated chunk sum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "groups.cuh"
#include "sm100.cuh"
#include "tc_internal.h"

namespace tc {

namespace tcg {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kProducers = 128;
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = 4 + kEpiWarps;
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t COL_MAIN = 0, COL_CORR = 256, COL_HI = 384;
constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait

struct Work {
  int32_t item, tile;
};

struct Launch {
  GemmArgs single;             // one contraction (items == nullptr)
  const GemmArgs* items;       // batch: per-item arguments (device)
  const Work* work;            // batch: (item, tile) entries (device)
  int64_t nwork;
  const void* const* Ap;       // batch: device arrays of per-item pointers and scalars
  const void* const* Bp;
  void* const* Cp;
  const double* alpha;
  const double* beta;
};

template <int NT>
struct Cfg {
  static constexpr int S = NT == 1 ? 6 : NT == 2 ? 3 : 2;         // pipeline stages
  static constexpr uint32_t A_TERM = BM * BK * 2;                  // bytes per A term
  static constexpr uint32_t B_TERM = BN * BK * 2;
  static constexpr uint32_t STAGE = NT * (A_TERM + B_TERM);
  static constexpr uint32_t OFF_KOFF = S * STAGE;                   // int64 koffA[S][BK], koffB[S][BK]
  static constexpr uint32_t OFF_KVEC = OFF_KOFF + S * BK * 2 * 8;  // uint8 kvecA[S][8], kvecB[S][8]
  static constexpr uint32_t OFF_ROWS = OFF_KVEC + S * 16 + 64;      // rowA[BM], rowB[BN], rowC[BM], colC[BN]
  static constexpr uint32_t OFF_ARGS = OFF_ROWS + (2 * BM + 2 * BN) * 8;
  static constexpr uint32_t OFF_BAR = OFF_ARGS + ((sizeof(GemmArgs) + 15) / 16) * 16;
  static constexpr uint32_t NBAR = 2 * S + 5;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 32 + 1024;          // + alignment slack
};

// Products (term of A, term of B) of each form; product 0 is the main one.
__constant__ int8_t kProdA[6] = {0, 0, 1, 0, 1, 2};
__constant__ int8_t kProdB[6] = {0, 1, 0, 2, 1, 0};
__host__ __device__ constexpr int nprod(int nt) { return nt == 1 ? 1 : nt == 2 ? 3 : 6; }

// Producer: one operand tile (ROWS x 64 K) of one K block.  Every load of the
// tile is issued before any is converted, so a thread keeps 64 loads in
// flight.  Lanes run along rows when the operand is contiguous along its
// M/N index (each k is then one coalesced row segment); otherwise lanes take
// (row-in-8, 8-wide K chunk) units, read as two 16-byte vectors when the
// chunk is contiguous and aligned.
template <int NT, int ROWS>
__device__ __forceinline__ void produce(const float* __restrict__ X, const int64_t* rowoff,
                                        const int64_t* koff, const uint8_t* kvec, bool contig_mn,
                                        bool rowvec, uint32_t sbuf, int ptid) {
  constexpr int PER = ROWS * (BK / 8) / kProducers;  // units per thread
  constexpr uint32_t TERM = ROWS * BK * 2;
  constexpr uint32_t LBO = (ROWS / 8) * 128;
  float v[PER][8];
  if (contig_mn && rowvec) {
    // four consecutive rows per 16-byte load: thread -> (row quad, chunk pair)
    const int quad = ptid & (ROWS / 4 - 1);
    const int cp = ptid / (ROWS / 4);          // 0 .. 128 / (ROWS / 4) - 1
    constexpr int NCP = kProducers / (ROWS / 4);
    const int64_t ro = rowoff[quad * 4];
#pragma unroll
    for (int h = 0; h < PER / 4; ++h) {
      const int chunk = cp + h * NCP;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t ko = koff[chunk * 8 + j];
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ko >= 0) x = __ldg(reinterpret_cast<const float4*>(X + ro + ko));
        v[h * 4 + 0][j] = x.x;
        v[h * 4 + 1][j] = x.y;
        v[h * 4 + 2][j] = x.z;
        v[h * 4 + 3][j] = x.w;
      }
    }
#pragma unroll
    for (int h = 0; h < PER / 4; ++h) {
      const int chunk = cp + h * NCP;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int row = quad * 4 + q4;
        const uint32_t dst = sbuf + chunk * LBO + (row >> 3) * 128 + (row & 7) * 16;
        float* vv = v[h * 4 + q4];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          uint32_t w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            w[q] = pack_bf16x2(vv[2 * q], vv[2 * q + 1]);
            if (t + 1 < NT) {
              vv[2 * q] = __fsub_rn(vv[2 * q], bf16_lo(w[q]));
              vv[2 * q + 1] = __fsub_rn(vv[2 * q + 1], bf16_hi(w[q]));
            }
          }
          st_shared_v4(dst + t * TERM, w[0], w[1], w[2], w[3]);
        }
      }
    }
    return;
  }
  if (contig_mn) {
    const int row = ptid % ROWS;
    const int64_t ro = rowoff[row];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int chunk = (ptid + r * kProducers) / ROWS;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t ko = koff[chunk * 8 + j];
        v[r][j] = (ro >= 0 && ko >= 0) ? __ldg(X + ro + ko) : 0.0f;
      }
    }
  } else {
    const int chunk = (ptid >> 3) & 7;
    const int64_t k0 = koff[chunk * 8];
    const bool vec = (kvec[chunk] & 1) != 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int u = ptid + r * kProducers;
      const int64_t ro = rowoff[(u & 7) + 8 * (u >> 6)];
      const float* src = X + ro + k0;
      if (vec && ro >= 0 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
        const float4 x0 = __ldg(reinterpret_cast<const float4*>(src));
        const float4 x1 = __ldg(reinterpret_cast<const float4*>(src) + 1);
        v[r][0] = x0.x; v[r][1] = x0.y; v[r][2] = x0.z; v[r][3] = x0.w;
        v[r][4] = x1.x; v[r][5] = x1.y; v[r][6] = x1.z; v[r][7] = x1.w;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t ko = koff[chunk * 8 + j];
          v[r][j] = (ro >= 0 && ko >= 0) ? __ldg(X + ro + ko) : 0.0f;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int u = ptid + r * kProducers;
    int row, chunk;
    if (contig_mn) {
      row = u % ROWS;
      chunk = u / ROWS;
    } else {
      row = (u & 7) + 8 * (u >> 6);
      chunk = (u >> 3) & 7;
    }
    const uint32_t dst = sbuf + chunk * LBO + (row >> 3) * 128 + (row & 7) * 16;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        w[q] = pack_bf16x2(v[r][2 * q], v[r][2 * q + 1]);
        if (t + 1 < NT) {  // exact FP32 residuals
          v[r][2 * q] = __fsub_rn(v[r][2 * q], bf16_lo(w[q]));
          v[r][2 * q + 1] = __fsub_rn(v[r][2 * q + 1], bf16_hi(w[q]));
        }
      }
      st_shared_v4(dst + t * TERM, w[0], w[1], w[2], w[3]);
    }
  }
}

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  bool ok = (*abort == 0) && mbar_wait(bar, parity, abort, kTimeoutNs);
  return __all_sync(0xffffffffu, ok);
}

// s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
  return s;
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ Launch L) {
  using G = Cfg<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  int64_t* koffA = reinterpret_cast<int64_t*>(smem + G::OFF_KOFF);
  int64_t* koffB = koffA + S * BK;
  uint8_t* kvecA = smem + G::OFF_KVEC;
  uint8_t* kvecB = kvecA + S * 8;
  int64_t* rowA = reinterpret_cast<int64_t*>(smem + G::OFF_ROWS);
  int64_t* rowB = rowA + BM;
  int64_t* rowC = rowB + BN;
  int64_t* colC = rowC + BM;
  int* rowvec = reinterpret_cast<int*>(smem + G::OFF_MISC + 8);  // [A, B]
  GemmArgs* sargs = reinterpret_cast<GemmArgs*>(smem + G::OFF_ARGS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = bars + 2 * S + 2;
  uint64_t* done = bars + 2 * S + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- once per CTA: barriers, tensor memory
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], kProducers);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], kEpiWarps * 32);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  uint32_t g_kb = 0;     // K blocks processed by this CTA (stage ring position)
  uint32_t g_chunk = 0;  // K chunks processed by this CTA (accumulator ring position)
  int cur_item = -2;

  for (int64_t w = blockIdx.x; w < L.nwork; w += gridDim.x) {
    // ---- the tile's arguments
    int item = -1;
    uint32_t tile = (uint32_t)w;
    if (L.items) {
      const Work wk = L.work[w];
      item = wk.item;
      tile = (uint32_t)wk.tile;
    }
    if (item != cur_item) {
      const uint32_t* src = item >= 0 ? reinterpret_cast<const uint32_t*>(L.items + item)
                                      : reinterpret_cast<const uint32_t*>(&L.single);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sargs);
      for (int i = tid; i < (int)(sizeof(GemmArgs) / 4); i += kThreads) dst[i] = src[i];
      __syncthreads();
      if (item >= 0 && tid == 0) {
        const bool sw = sargs->swapped != 0;
        sargs->A = sw ? L.Bp[item] : L.Ap[item];
        sargs->B = sw ? L.Ap[item] : L.Bp[item];
        sargs->C = L.Cp[item];
        sargs->alpha = L.alpha[item];
        sargs->beta = L.beta[item];
      }
      cur_item = item;
    }
    __syncthreads();
    const GemmArgs& p = *sargs;
    const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
    const uint32_t tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
    uint32_t tm, tn, b;
    if (p.raster) {  // n-tiles fastest: the CTAs sharing an A panel run together
      tn = tile % tiles_n;
      tm = (tile / tiles_n) % tiles_m;
    } else {
      tm = tile % tiles_m;
      tn = (tile / tiles_m) % tiles_n;
    }
    b = tile / (tiles_n * tiles_m);
    int64_t bA, bB, bC;
    goff3(p.gb, b, bA, bB, bC);
    for (int i = tid; i < BM; i += kThreads) {
      const uint32_t m = tm * BM + i;
      int64_t oa = -1, oc = -1;
      if (m < M) goff2(p.gm, 0, 2, m, oa, oc);
      rowA[i] = oa;
      rowC[i] = oc;
    }
    for (int i = tid; i < BN; i += kThreads) {
      const uint32_t n = tn * BN + i;
      int64_t ob = -1, oc = -1;
      if (n < N) goff2(p.gn, 1, 2, n, ob, oc);
      rowB[i] = ob;
      colC[i] = oc;
    }
    __syncthreads();
    if (warp == 0) {  // may rows be read four at a time (16-byte vectors)?
      for (int which = 0; which < 2; ++which) {
        const int64_t* ro = which ? rowB : rowA;
        const bool mn = (which ? p.b_contig : p.a_contig) == CONTIG_MN;
        const uintptr_t base = reinterpret_cast<uintptr_t>(which ? p.B : p.A) +
                               (uintptr_t)((which ? bB : bA) * 4);
        bool ok = mn && (base & 15) == 0;
        for (int r = lane; r < 128 && ok; r += 32)
          ok = ro[r] >= 0 && (r % 4 == 0 ? (ro[r] & 3) == 0 : ro[r] == ro[r - 1] + 1);
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) rowvec[which] = ok ? 1 : 0;
      }
    }
    __syncthreads();

    const uint32_t nkb = (K + BK - 1) / BK;
    const uint32_t ckb = (uint32_t)max(p.chunk_kb, 1);  // K blocks per chunk
    const uint32_t nchunks = (nkb + ckb - 1) / ckb;

    if (warp < 4) {
      // ---------------------------------------------------------- producers
      const float* __restrict__ Xa = static_cast<const float*>(p.A) + bA;
      const float* __restrict__ Xb = static_cast<const float*>(p.B) + bB;
      const bool amn = p.a_contig == CONTIG_MN, bmn = p.b_contig == CONTIG_MN;
      for (uint32_t kb = 0; kb < nkb; ++kb, ++g_kb) {
        const int s = g_kb % S;
        const uint32_t ph = (g_kb / S) & 1;
        bool ok = true;
        if (g_kb >= (uint32_t)S) ok = warp_wait(&empty[s], ph ^ 1, abort);
        if (tid < BK) {
          const uint32_t k = kb * BK + tid;
          int64_t oa = -1, ob = -1;
          if (k < K) goff2(p.gk, 0, 1, k, oa, ob);
          koffA[s * BK + tid] = oa;
          koffB[s * BK + tid] = ob;
        }
        named_bar_sync(1, kProducers);
        if (tid < 16) {  // 8-wide K chunks that are contiguous and 4-element aligned
          const int64_t* ko = (tid < 8 ? koffA : koffB) + s * BK + (tid & 7) * 8;
          bool c = ko[0] >= 0 && (ko[0] & 3) == 0;
          bool al = true;  // every k offset a multiple of 4 (or beyond K)
          for (int j = 1; j < 8; ++j) c = c && ko[j] == ko[0] + j;
          for (int j = 0; j < 8; ++j) al = al && (ko[j] < 0 || (ko[j] & 3) == 0);
          (tid < 8 ? kvecA : kvecB)[s * 8 + (tid & 7)] = (c ? 1 : 0) | (al ? 2 : 0);
        }
        named_bar_sync(1, kProducers);
        bool kal[2] = {true, true};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          kal[0] = kal[0] && (kvecA[s * 8 + c] & 2);
          kal[1] = kal[1] && (kvecB[s * 8 + c] & 2);
        }
        if (ok && !*abort) {
          const uint32_t st = sbase + s * G::STAGE;
          produce<NT, BM>(Xa, rowA, koffA + s * BK, kvecA + s * 8, amn, rowvec[0] && kal[0], st,
                          tid);
          produce<NT, BN>(Xb, rowB, koffB + s * BK, kvecB + s * 8, bmn, rowvec[1] && kal[1],
                          st + NT * G::A_TERM, tid);
          fence_async_smem();
          mbar_arrive(&full[s]);
        }
      }
    } else if (warp < kMmaWarp) {
      // ----------------------------------------------------------- epilogue
      const int q = warp & 3;            // tensor-memory lane quadrant
      const int h = (warp - 4) >> 2;     // column half
      const int row = q * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + h * 64;
      const int64_t rc = rowC[row];
      float* __restrict__ Cp = static_cast<float*>(p.C) + bC;
      float lo[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) lo[i] = 0.0f;
      for (uint32_t j = 0; j < nchunks; ++j, ++g_chunk) {
        const uint32_t buf = g_chunk & 1;
        if (!warp_wait(&accf[buf], (g_chunk >> 1) & 1, abort)) {
          g_chunk += nchunks - j;
          break;
        }
        tc_fence_after();
        const uint32_t tmain = tl + COL_MAIN + buf * 128;
        if (j + 1 < nchunks) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t mv[16], hv[16];
            tmem_ld16(tmain + c * 16, mv);
            if (j > 0) tmem_ld16(tl + COL_HI + c * 16, hv);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float hi0 = j > 0 ? __uint_as_float(hv[i]) : 0.0f;
              float e;
              const float s = two_sum(hi0, __uint_as_float(mv[i]), e);
              lo[c * 16 + i] = __fadd_rn(lo[c * 16 + i], e);
              hv[i] = __float_as_uint(s);
            }
            tmem_st16(tl + COL_HI + c * 16, hv);
          }
          tmem_wait_st();
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t mv[8], hv[8], cv[8];
            tmem_ld8(tmain + c * 8, mv);
            if (j > 0) tmem_ld8(tl + COL_HI + c * 8, hv);
            if (NT > 1) tmem_ld8(tl + COL_CORR + c * 8, cv);
            tmem_wait_ld();
            if (rc >= 0) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const int64_t cc = colC[h * 64 + c * 8 + i];
                if (cc < 0) continue;
                double t = (double)__uint_as_float(mv[i]);
                if (j > 0) t += (double)__uint_as_float(hv[i]) + (double)lo[c * 8 + i];
                if (NT > 1) t += (double)__uint_as_float(cv[i]);
                float* dst = Cp + rc + cc;
                double v = p.alpha * t;
                if (p.beta != 0.0) v += p.beta * (double)*dst;
                *dst = (float)v;
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&acce[buf]);
      }
    } else if (lane == 0) {
      // ------------------------------------------------------ MMA issue
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      constexpr uint32_t LBO_A = (BM / 8) * 128, LBO_B = (BN / 8) * 128;
      uint32_t kb = 0;
      bool ok = !*abort;
      for (uint32_t j = 0; j < nchunks; ++j, ++g_chunk) {
        const uint32_t buf = g_chunk & 1;
        if (ok && g_chunk >= 2 && !mbar_wait(&acce[buf], ((g_chunk >> 1) - 1) & 1, abort, kTimeoutNs))
          ok = false;
        if (!ok) {
          g_kb += nkb - kb;
          g_chunk += nchunks - j;
          break;
        }
        tc_fence_after();
        const uint32_t dmain = tmem + COL_MAIN + buf * 128;
        const uint32_t kend = min(nkb, (j + 1) * ckb);
        const uint32_t kstart = kb;
        for (; kb < kend; ++kb, ++g_kb) {
          const int s = g_kb % S;
          if (!mbar_wait(&full[s], (g_kb / S) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = sbase + s * G::STAGE;
          const uint32_t sb = sa + NT * G::A_TERM;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            mma_bf16(dmain, smem_desc(sa + kk * 2 * LBO_A, LBO_A, 128),
                     smem_desc(sb + kk * 2 * LBO_B, LBO_B, 128), idesc,
                     (kb > kstart || kk > 0) ? 1u : 0u);
#pragma unroll
            for (int pi = 1; pi < nprod(NT); ++pi) {
              mma_bf16(tmem + COL_CORR,
                       smem_desc(sa + kProdA[pi] * G::A_TERM + kk * 2 * LBO_A, LBO_A, 128),
                       smem_desc(sb + kProdB[pi] * G::B_TERM + kk * 2 * LBO_B, LBO_B, 128),
                       idesc, (kb > 0 || kk > 0 || pi > 1) ? 1u : 0u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) {
          g_kb += nkb - kb;
          g_chunk += nchunks - j;
          break;
        }
        mma_commit(&accf[buf]);
      }
    } else {
      g_kb += nkb;  // other lanes of the MMA warp keep the counters in step
      g_chunk += nchunks;
    }
    __syncwarp();
    __syncthreads();  // the tile is finished (its last accumulator was drained)
  }

  if (warp == kMmaWarp && lane == 0) {
    mma_commit(done);  // arrives once every MMA issued by this thread has completed
    volatile int keep_waiting = 0;
    mbar_wait(done, 0, &keep_waiting, kTimeoutNs);
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

template <int NT>
int smem_bytes() {
  static int bytes = 0;
  if (bytes == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return -1;
    if (optin < (int)Cfg<NT>::BYTES) return -2;
    // The whole opt-in shared memory is requested: one CTA per SM (it owns all
    // 512 tensor-memory columns) and room beyond the last operand tile.
    if (cudaFuncSetAttribute(k_gemm_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
        cudaSuccess)
      return -1;
    bytes = optin;
  }
  return bytes;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
  }
  return n;
}

template <int NT>
tc_status launch(const Launch& L, cudaStream_t s) {
  if (L.nwork == 0) return TC_OK;
  const int bytes = smem_bytes<NT>();
  if (bytes == -2) return TC_ERR_UNSUPPORTED;
  const int sms = num_sms();
  if (bytes < 0 || sms <= 0) return TC_ERR_CUDA;
  const int grid = (int)std::min<int64_t>(L.nwork, sms);
  k_gemm_tc<NT><<<grid, kThreads, bytes, s>>>(L);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_math(const Launch& L, int math, cudaStream_t s) {
  switch (math) {
    case TC_MATH_BF16: return launch<1>(L, s);
    case TC_MATH_BF16X3: return launch<2>(L, s);
    case TC_MATH_BF16X6: return launch<3>(L, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

uint64_t tiles_of(const GemmArgs& a) {
  return (uint64_t)((a.M + BM - 1) / BM) * (uint64_t)((a.N + BN - 1) / BN) * (uint64_t)a.nbatch;
}

}  // namespace tcg

// Tile configurations of the tensor-core GEMM: K blocks (of 64) per chunk of
// the main accumulator.  Tile 0: one chunk for plain BF16 (its error is that of
// the BF16 inputs), 256-K chunks for the split forms; tile 1: 64-K chunks;
// tile 2: 1024-K chunks.
int num_tiles_tc() { return 3; }
int tc_chunk_kb(int math, int tile) {
  if (tile == 1) return 1;
  if (tile == 2) return 16;
  return math == TC_MATH_BF16 ? (1 << 30) : 4;
}

tc_status tc_gemm_read_status(int* h, void* stream) {
  return read_clear_status(h, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TC_OK
                                                                                : TC_ERR_CUDA;
}

tc_status launch_gemm_tc(const GemmArgs& a, int math, void* stream) {
  tcg::Launch L;
  std::memset(&L, 0, sizeof(L));
  L.single = a;
  L.nwork = (int64_t)tcg::tiles_of(a);
  if ((uint64_t)L.nwork > 0x7fffffffull) return TC_ERR_UNSUPPORTED;
  return tcg::launch_math(L, math, static_cast<cudaStream_t>(stream));
}

tc_status launch_gemm_tc_batch(const GemmArgs* d_items, const void* d_work, int64_t nwork,
                               const void* const* A, const void* const* B, void* const* C,
                               const double* alpha, const double* beta, int math, void* stream) {
  tcg::Launch L;
  std::memset(&L, 0, sizeof(L));
  L.items = d_items;
  L.work = static_cast<const tcg::Work*>(d_work);
  L.nwork = nwork;
  L.Ap = A;
  L.Bp = B;
  L.Cp = C;
  L.alpha = alpha;
  L.beta = beta;
  return tcg::launch_math(L, math, static_cast<cudaStream_t>(stream));
}

uint64_t tc_gemm_tiles(const GemmArgs& a) { return tcg::tiles_of(a); }

}  // namespace tc
