// k_tc.cu -- the tensor-core GEMM over gathered index groups (sm_103a, tcgen05):
// tile configurations 0-2 of a single contraction, and the slicing mapping's
// batches of GEMMs (whose batch group the packed kernel does not take).
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
//   warps 0-3   producers: copy FP32 elements of A and B, gathered through the
//               index groups (any strides: the permutation of a Class 3.1
//               operand is absorbed here, so no copy pass touches HBM), into a
//               shared-memory staging ring with cp.async (16-byte copies where
//               four elements are contiguous), several K blocks ahead; then
//               split each staged block into BF16 terms and store the terms in
//               the canonical K-major layout of the tensor cores;
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

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int kProducers = 128;
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = 4 + kEpiWarps;
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t COL_MAIN = 0, COL_CORR = 256, COL_HI = 384;
constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait

struct Launch {
  GemmArgs single;             // the contraction
  int64_t nwork;               // its tiles
};

template <int NT>
struct Cfg {
  static constexpr int S = NT == 1 ? 4 : NT == 2 ? 3 : 2;         // BF16 term stages
  static constexpr int D = NT == 1 ? 4 : 3;                       // FP32 staging depth
  static constexpr uint32_t A_TERM = BM * BK * 2;                  // bytes per A term
  static constexpr uint32_t B_TERM = BN * BK * 2;
  static constexpr uint32_t STAGE = NT * (A_TERM + B_TERM);
  // FP32 staging of one operand: [row][BK + 4] (K-contiguous or gathered
  // operands) or [k][128 + 4] (operands contiguous along rows).
  static constexpr uint32_t SOP = 128 * (BK + 4) * 4;
  static constexpr uint32_t OFF_STG = S * STAGE;
  static constexpr uint32_t OFF_KOFF = OFF_STG + D * 2 * SOP;       // int64 koffA[BK], koffB[BK]
  static constexpr uint32_t OFF_KFLAG = OFF_KOFF + 2 * BK * 8;      // uint8 kflag[2][BK / 4]
  static constexpr uint32_t OFF_ROWQ = OFF_KFLAG + 16;              // uint8 rowq[2][32]
  static constexpr uint32_t OFF_ROWS = OFF_ROWQ + 64;               // rowA, rowB, rowC, colC
  static constexpr uint32_t OFF_ARGS = OFF_ROWS + (2 * BM + 2 * BN) * 8;
  static constexpr uint32_t OFF_BAR = OFF_ARGS + ((sizeof(GemmArgs) + 15) / 16) * 16;
  static constexpr uint32_t NBAR = 2 * S + 5;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 32 + 1024;          // + alignment slack
};

// Products (term of A, term of B) of each form; product 0 is the main one.
// Terms of product pi: a_{prod_a(pi)} * b_{prod_b(pi)} (a0 b0; a0 b1, a1 b0;
// a0 b2, a1 b1, a2 b0).  Compile-time functions, so that the unrolled MMA
// loops fold them into their descriptor offsets.
__host__ __device__ constexpr int prod_a(int pi) {
  return pi == 2 || pi == 4 ? 1 : pi == 5 ? 2 : 0;
}
__host__ __device__ constexpr int prod_b(int pi) {
  return pi == 1 || pi == 4 ? 1 : pi == 3 ? 2 : 0;
}
__host__ __device__ constexpr int nprod(int nt) { return nt == 1 ? 1 : nt == 2 ? 3 : 6; }

// Copy one operand's FP32 block (ROWS x BK) into a staging slot.  Operands
// contiguous along their rows are staged [k][row]: lanes take row quads, one
// 16-byte copy per (quad, k) when the four rows are contiguous and aligned.
// Other operands are staged [row][k]: lanes take (row, 4-wide K group), one
// 16-byte copy when the four k are contiguous and aligned.  Elements outside
// the tensor are zero-filled.
// K offsets of a block: a shared table (K groups of several labels) or
// base + k * stride (one label); -1 marks k beyond K.
struct KOff {
  const int64_t* table;
  const uint8_t* flag;   // per 4-wide K group: contiguous (table mode)
  int64_t base, stride;
  int kvalid;
  __device__ __forceinline__ int64_t operator()(int k) const {
    if (table) return table[k];
    return k < kvalid ? base + (int64_t)k * stride : -1;
  }
  __device__ __forceinline__ bool contiguous4(int g) const {
    if (table) return flag[g] != 0;
    return stride == 1 && g * 4 + 3 < kvalid;
  }
};

template <int ROWS>
__device__ __forceinline__ void issue_copies(const float* __restrict__ X,
                                             const int64_t* rowoff, const uint8_t* rowq,
                                             const KOff& koff, bool contig_mn, uint32_t slot,
                                             int ptid) {
  if (contig_mn) {
    const int quad = ptid & (ROWS / 4 - 1);
    const int kg = ptid / (ROWS / 4);
    constexpr int NK = kProducers / (ROWS / 4);
    const bool q4 = rowq[quad] != 0;
#pragma unroll
    for (int r = 0; r < BK / NK; ++r) {
      const int k = kg + r * NK;
      const int64_t ko = koff(k);
      const uint32_t dst = slot + (uint32_t)(k * (ROWS + 4) + quad * 4) * 4;
      const float* src = X + rowoff[quad * 4] + ko;
      if (q4 && ko >= 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        cp_async16(dst, src);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t ro = rowoff[quad * 4 + i];
          const bool ok = ro >= 0 && ko >= 0;
          cp_async4(dst + 4 * i, ok ? (const void*)(X + ro + ko) : (const void*)X, ok ? 4u : 0u);
        }
      }
    }
  } else {
    const int kg = ptid & (BK / 4 - 1);
    constexpr int RSTEP = kProducers / (BK / 4);
    const bool k4 = koff.contiguous4(kg);
    const int64_t ko0 = koff(kg * 4);
#pragma unroll
    for (int r = 0; r < ROWS / RSTEP; ++r) {
      const int row = ptid / (BK / 4) + r * RSTEP;
      const int64_t ro = rowoff[row];
      const uint32_t dst = slot + (uint32_t)(row * (BK + 4) + kg * 4) * 4;
      const float* src = X + ro + ko0;
      if (k4 && ro >= 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        cp_async16(dst, src);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t ko = koff(kg * 4 + i);
          const bool ok = ro >= 0 && ko >= 0;
          cp_async4(dst + 4 * i, ok ? (const void*)(X + ro + ko) : (const void*)X, ok ? 4u : 0u);
        }
      }
    }
  }
}

// Split a staged FP32 block into NT BF16 terms in the canonical K-major layout
// (8-row x 16-byte core matrices; 8-wide K chunks LBO bytes apart).
template <int NT, int ROWS>
__device__ __forceinline__ void convert(const float* stg, bool contig_mn, uint32_t sbuf,
                                        int ptid) {
  constexpr uint32_t TERM = ROWS * BK * 2;
  constexpr uint32_t LBO = (ROWS / 8) * 128;
  const int row = ptid;  // ROWS == kProducers
#pragma unroll
  for (int chunk = 0; chunk < BK / 8; ++chunk) {
    float v[8];
    if (contig_mn) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = stg[(chunk * 8 + j) * (ROWS + 4) + row];
    } else {
      const float4 x0 = *reinterpret_cast<const float4*>(stg + row * (BK + 4) + chunk * 8);
      const float4 x1 = *reinterpret_cast<const float4*>(stg + row * (BK + 4) + chunk * 8 + 4);
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    }
    const uint32_t dst = sbuf + chunk * LBO + (row >> 3) * 128 + (row & 7) * 16;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        w[q] = pack_bf16x2(v[2 * q], v[2 * q + 1]);
        if (t + 1 < NT) {  // exact FP32 residuals
          v[2 * q] = __fsub_rn(v[2 * q], bf16_lo(w[q]));
          v[2 * q + 1] = __fsub_rn(v[2 * q + 1], bf16_hi(w[q]));
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
  int64_t* koffB = koffA + BK;
  uint8_t* kflagA = smem + G::OFF_KFLAG;
  uint8_t* kflagB = kflagA + BK / 4;
  uint8_t* rowqA = smem + G::OFF_ROWQ;
  uint8_t* rowqB = rowqA + 32;
  int64_t* rowA = reinterpret_cast<int64_t*>(smem + G::OFF_ROWS);
  int64_t* rowB = rowA + BM;
  int64_t* rowC = rowB + BN;
  int64_t* colC = rowC + BM;
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
  {  // the contraction's arguments, once
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&L.single);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sargs);
    for (int i = tid; i < (int)(sizeof(GemmArgs) / 4); i += kThreads) dst[i] = src[i];
  }

  for (int64_t w = blockIdx.x; w < L.nwork; w += gridDim.x) {
    const uint32_t tile = (uint32_t)w;
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
    if (tid < 64) {  // row quads that are valid and contiguous (16-byte copies)
      const int which = tid >> 5, q = tid & 31;
      const int64_t* ro = which ? rowB : rowA;
      bool ok = true;
      for (int i = 0; i < 4; ++i) ok = ok && ro[q * 4 + i] >= 0 && ro[q * 4 + i] == ro[q * 4] + i;
      (which ? rowqB : rowqA)[q] = ok ? 1 : 0;
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
      const uint32_t stg0 = sbase + G::OFF_STG;
      const float* stgp = reinterpret_cast<const float*>(smem + G::OFF_STG);
      // K offsets (and 4-wide contiguity flags) of block kk, then its copies
      // A K group of one (merged) label has offsets k * stride: the offsets
      // are computed where they are used and no barrier is needed; otherwise
      // one thread per k splits k into its labels and the producers
      // synchronise on the shared tables.
      const bool klin = p.gk.n <= 1;
      const int64_t ksa = p.gk.n ? p.gk.st[0][0] : 0, ksb = p.gk.n ? p.gk.st[1][0] : 0;
      auto load_block = [&](uint32_t kk, int slot) {
        const int kvalid = (int)min((uint32_t)BK, K - kk * BK);
        KOff ka{nullptr, nullptr, (int64_t)kk * BK * ksa, ksa, kvalid};
        KOff kb_{nullptr, nullptr, (int64_t)kk * BK * ksb, ksb, kvalid};
        if (!klin) {
          // the tables are rewritten: every producer has issued the copies of
          // the block before from them (back-to-back calls in the prologue and
          // into the main loop have no other barrier between them)
          named_bar_sync(1, kProducers);
          if (tid < BK) {
            const uint32_t k = kk * BK + tid;
            int64_t oa = -1, ob = -1;
            if (k < K) goff2(p.gk, 0, 1, k, oa, ob);
            koffA[tid] = oa;
            koffB[tid] = ob;
          }
          named_bar_sync(1, kProducers);
          if (tid < BK / 2) {
            const int which = tid / (BK / 4), g = tid % (BK / 4);
            const int64_t* ko = (which ? koffB : koffA) + g * 4;
            bool c = ko[0] >= 0;
            for (int i = 1; i < 4; ++i) c = c && ko[i] == ko[0] + i;
            (which ? kflagB : kflagA)[g] = c ? 1 : 0;
          }
          named_bar_sync(1, kProducers);
          ka = KOff{koffA, kflagA, 0, 0, kvalid};
          kb_ = KOff{koffB, kflagB, 0, 0, kvalid};
        }
        const uint32_t sl = stg0 + (uint32_t)slot * 2 * G::SOP;
        issue_copies<BM>(Xa, rowA, rowqA, ka, amn, sl, tid);
        issue_copies<BN>(Xb, rowB, rowqB, kb_, bmn, sl + G::SOP, tid);
      };
      constexpr int D = G::D;
      for (int d = 0; d < D - 1; ++d) {
        if ((uint32_t)d < nkb) load_block((uint32_t)d, d);
        cp_async_commit();
      }
      for (uint32_t kb = 0; kb < nkb; ++kb, ++g_kb) {
        if (kb + D - 1 < nkb) load_block(kb + D - 1, (int)((kb + D - 1) % D));
        cp_async_commit();
        cp_async_wait<D - 1>();              // this thread's copies of block kb landed
        named_bar_sync(1, kProducers);       // ... and every producer's
        const int s = g_kb % S;
        const uint32_t ph = (g_kb / S) & 1;
        bool ok = true;
        if (g_kb >= (uint32_t)S) ok = warp_wait(&empty[s], ph ^ 1, abort);
        if (ok && !*abort) {
          const uint32_t st = sbase + s * G::STAGE;
          const float* sl = stgp + (size_t)(kb % D) * 2 * (G::SOP / 4);
          convert<NT, BM>(sl, amn, st, tid);
          convert<NT, BN>(sl + G::SOP / 4, bmn, st + NT * G::A_TERM, tid);
          fence_async_smem();
          mbar_arrive(&full[s]);
        }
        named_bar_sync(1, kProducers);       // staging slot kb % D may be refilled
      }
      cp_async_wait<0>();
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
                       smem_desc(sa + prod_a(pi) * G::A_TERM + kk * 2 * LBO_A, LBO_A, 128),
                       smem_desc(sb + prod_b(pi) * G::B_TERM + kk * 2 * LBO_B, LBO_B, 128),
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

// Tile configurations of the tensor-core GEMM: K blocks (of 32) per chunk of
// the main accumulator.  Tile 0: one chunk for plain BF16 (its error is that of
// the BF16 inputs), 256-K chunks for the split forms; tile 1: 64-K chunks;
// tile 2: 1024-K chunks; tile 3: the chunks of tile 0 on packed operands
// (k_tcpk.cu: a pack pass splits the operands once, the GEMM moves the terms
// with bulk copies); tile 4: packed operands on 128 x 256 tiles with one
// accumulator per tile (BF16, FP16 and BF16x3 only).
int num_tiles_tc() { return 6; }
int tc_chunk_kb(int math, int tile) {
  if (tile == 1) return 2;
  if (tile == 2) return 32;
  // wide tiles: chunks of 256 K for BF16x3, one chunk per tile otherwise
  // one chunk per tile for BF16 and FP16 (their error is the operands'
  // rounding); 256-K chunks for the split forms
  if (tile == kTilePackedWide || tile == kTilePackedPair)
    return (math == TC_MATH_BF16X3 || math == TC_MATH_BF16X6) ? 8 : (1 << 30);
  return (math == TC_MATH_BF16 || math == TC_MATH_FP16) ? (1 << 30) : 8;
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

}  // namespace tc
