// k_tc.cu -- the tensor-core GEMM over gathered index groups (sm_103a, tcgen05).
//
// C[m, n, b] = alpha * sum_k A[m, k, b] * B[k, n, b] + beta * C[m, n, b] for
// FP32 tensors of any layout, computed as a sum of BF16 products:
//   BF16    a0 b0                                (1 term per operand)
//   BF16x3  a0 b0 + a0 b1 + a1 b0                 (2 terms)
//   BF16x6  + a0 b2 + a1 b1 + a2 b0               (3 terms)
// with x = x0 + x1 + x2 the split of an FP32 value into BF16 terms, each the
// round-to-nearest-even BF16 value of the remaining residual.
//
// One CTA computes a 128 x 128 tile of C.  Warp roles (288 threads):
//   warps 0-3  producers: read FP32 elements of A and B through the index
//              groups (any strides; the permutation of a Class 3.1 operand is
//              absorbed here, so no copy pass touches HBM), split them into
//              BF16 terms in registers and store the terms to shared memory in
//              the canonical K-major layout of the tensor cores;
//   warps 4-7  epilogue: drain each finished K-chunk accumulator from tensor
//              memory and add it to an FP64 running sum kept in tensor memory;
//              the last chunk is combined with alpha/beta and stored to C;
//   warp 8     tensor-memory allocation and the single thread issuing
//              tcgen05.mma for every product of every K-step.
// The K range is cut into chunks (a few hundred to a thousand K): each chunk
// is accumulated in FP32 in one of two tensor-memory accumulators (double
// buffered so the tensor cores keep running while the other is drained), and
// the chunks are summed in FP64, so FP32 rounding grows only over one chunk.
//
// Tensor memory (512 columns x 128 lanes): columns [0,128) and [128,256) are
// the two accumulators, [256,512) holds the FP64 running sums (two 32-bit
// columns per output column).
#include <cuda_runtime.h>

#include <algorithm>

#include "groups.cuh"
#include "sm100.cuh"
#include "tc_internal.h"

namespace tc {

namespace tcg {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int kThreads = 288;
constexpr int kProducers = 128;
constexpr int kEpiWarp0 = 4;
constexpr int kMmaWarp = 8;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait

template <int NT>
struct Cfg {
  static constexpr int S = NT == 1 ? 6 : NT == 2 ? 3 : 2;         // pipeline stages
  static constexpr uint32_t A_TERM = BM * BK * 2;                  // bytes per A term
  static constexpr uint32_t B_TERM = BN * BK * 2;
  static constexpr uint32_t STAGE = NT * (A_TERM + B_TERM);
  static constexpr uint32_t OFF_KOFF = S * STAGE;                   // int64 koffA[S][BK], koffB[S][BK]
  static constexpr uint32_t OFF_ROWS = OFF_KOFF + S * BK * 2 * 8;  // rowA[BM], rowB[BN], rowC[BM], colC[BN]
  static constexpr uint32_t OFF_BAR = OFF_ROWS + (2 * BM + 2 * BN) * 8;
  static constexpr uint32_t NBAR = 2 * S + 5;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;          // + alignment slack
};

// Products (term of A, term of B) of each form, largest first.
__constant__ int8_t kProdA[6] = {0, 0, 1, 0, 1, 2};
__constant__ int8_t kProdB[6] = {0, 1, 0, 2, 1, 0};
__host__ __device__ constexpr int nprod(int nt) { return nt == 1 ? 1 : nt == 2 ? 3 : 6; }

template <int NT, int ROWS>
__device__ __forceinline__ void produce(const float* __restrict__ X, const int64_t* rowoff,
                                        const int64_t* koff, bool contig_mn, uint32_t sbuf,
                                        int ptid) {
  constexpr int UNITS = ROWS * (BK / 8);
  constexpr uint32_t TERM = ROWS * BK * 2;
  constexpr uint32_t LBO = (ROWS / 8) * 128;
#pragma unroll 2
  for (int u = ptid; u < UNITS; u += kProducers) {
    int row, chunk;
    if (contig_mn) {  // lanes along rows: each k is a coalesced row segment
      row = u % ROWS;
      chunk = u / ROWS;
    } else {          // lanes along (row-in-8, chunk): 32-byte runs along k
      row = (u & 7) + 8 * (u >> 6);
      chunk = (u >> 3) & 7;
    }
    const int64_t ro = rowoff[row];
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t ko = koff[chunk * 8 + j];
      v[j] = (ro >= 0 && ko >= 0) ? __ldg(X + ro + ko) : 0.0f;
    }
    const uint32_t dst = sbuf + chunk * LBO + (row >> 3) * 128 + (row & 7) * 16;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        w[q] = pack_bf16x2(v[2 * q], v[2 * q + 1]);
        if (t + 1 < NT) {  // exact FP32 residuals
          v[2 * q] -= bf16_lo(w[q]);
          v[2 * q + 1] -= bf16_hi(w[q]);
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

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ GemmArgs p) {
  using G = Cfg<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  int64_t* koffA = reinterpret_cast<int64_t*>(smem + G::OFF_KOFF);
  int64_t* koffB = koffA + S * BK;
  int64_t* rowA = reinterpret_cast<int64_t*>(smem + G::OFF_ROWS);
  int64_t* rowB = rowA + BM;
  int64_t* rowC = rowB + BN;
  int64_t* colC = rowC + BM;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = bars + 2 * S + 2;
  uint64_t* done = bars + 2 * S + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t M = (uint32_t)p.M, N = (uint32_t)p.N, K = (uint32_t)p.K;
  const uint32_t tiles_m = (M + BM - 1) / BM, tiles_n = (N + BN - 1) / BN;
  uint32_t tm, tn, b;
  {
    const uint64_t t = blockIdx.x;
    if (p.raster) {  // n-tiles fastest: the CTAs sharing an A panel run together
      tn = (uint32_t)(t % tiles_n);
      tm = (uint32_t)((t / tiles_n) % tiles_m);
      b = (uint32_t)(t / ((uint64_t)tiles_n * tiles_m));
    } else {
      tm = (uint32_t)(t % tiles_m);
      tn = (uint32_t)((t / tiles_m) % tiles_n);
      b = (uint32_t)(t / ((uint64_t)tiles_n * tiles_m));
    }
  }
  int64_t bA, bB, bC;
  goff3(p.gb, b, bA, bB, bC);

  // ---- set-up: offsets, barriers, tensor memory
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
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], kProducers);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 128);
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

  const uint32_t nkb = (K + BK - 1) / BK;
  const uint32_t ckb = (uint32_t)max(p.chunk_kb, 1);  // K blocks per chunk
  const uint32_t nchunks = (nkb + ckb - 1) / ckb;
  const uint32_t sbase = smem_u32(smem);

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    const float* __restrict__ Xa = static_cast<const float*>(p.A) + bA;
    const float* __restrict__ Xb = static_cast<const float*>(p.B) + bB;
    const bool amn = p.a_contig == CONTIG_MN, bmn = p.b_contig == CONTIG_MN;
    for (uint32_t kb = 0; kb < nkb; ++kb) {
      const int s = kb % S;
      const uint32_t ph = (kb / S) & 1;
      bool ok = true;
      if (kb >= S) ok = warp_wait(&empty[s], ph ^ 1, abort);
      if (tid < BK) {
        const uint32_t k = kb * BK + tid;
        int64_t oa = -1, ob = -1;
        if (k < K) goff2(p.gk, 0, 1, k, oa, ob);
        koffA[s * BK + tid] = oa;
        koffB[s * BK + tid] = ob;
      }
      named_bar_sync(1, kProducers);
      if (ok && !*abort) {
        const uint32_t st = sbase + s * G::STAGE;
        produce<NT, BM>(Xa, rowA, koffA + s * BK, amn, st, tid);
        produce<NT, BN>(Xb, rowB, koffB + s * BK, bmn, st + NT * G::A_TERM, tid);
        fence_async_smem();
        mbar_arrive(&full[s]);
      }
    }
  } else if (warp < kMmaWarp) {
    // ------------------------------------------------------------- epilogue
    const int q = warp & 3;  // tensor-memory lane quadrant of this warp
    const int row = q * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16);
    const bool rvalid = rowC[row] >= 0;
    float* __restrict__ Cp = static_cast<float*>(p.C) + bC;
    for (uint32_t j = 0; j < nchunks; ++j) {
      const uint32_t buf = j & 1;
      if (!warp_wait(&accf[buf], (j >> 1) & 1, abort)) break;
      tc_fence_after();
      const bool last = j + 1 == nchunks;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t c[16], wl[16], wh[16];
        tmem_ld16(tl + buf * BN + c0, c);
        if (j > 0) {
          tmem_ld16(tl + 2 * BN + 2 * c0, wl);
          tmem_ld16(tl + 2 * BN + 2 * c0 + 16, wh);
        }
        tmem_wait_ld();
        double s[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          double prev = 0.0;
          if (j > 0) {
            const uint32_t lo = i < 8 ? wl[2 * i] : wh[2 * (i - 8)];
            const uint32_t hi = i < 8 ? wl[2 * i + 1] : wh[2 * (i - 8) + 1];
            prev = __hiloint2double((int)hi, (int)lo);
          }
          s[i] = prev + (double)__uint_as_float(c[i]);
        }
        if (!last) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            wl[2 * i] = (uint32_t)__double2loint(s[i]);
            wl[2 * i + 1] = (uint32_t)__double2hiint(s[i]);
            wh[2 * i] = (uint32_t)__double2loint(s[8 + i]);
            wh[2 * i + 1] = (uint32_t)__double2hiint(s[8 + i]);
          }
          tmem_st16(tl + 2 * BN + 2 * c0, wl);
          tmem_st16(tl + 2 * BN + 2 * c0 + 16, wh);
        } else if (rvalid) {
          const int64_t rc = rowC[row];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int64_t cc = colC[c0 + i];
            if (cc < 0) continue;
            float* dst = Cp + rc + cc;
            double v = p.alpha * s[i];
            if (p.beta != 0.0) v += p.beta * (double)*dst;
            *dst = (float)v;
          }
        }
      }
      if (!last) tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&acce[buf]);
    }
  } else {
    // -------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      constexpr uint32_t LBO_A = (BM / 8) * 128, LBO_B = (BN / 8) * 128;
      uint32_t kb = 0;
      bool ok = true;
      for (uint32_t j = 0; j < nchunks && ok; ++j) {
        const uint32_t buf = j & 1;
        if (j >= 2 && !mbar_wait(&acce[buf], ((j >> 1) - 1) & 1, abort, kTimeoutNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + buf * BN;
        uint32_t acc = 0;
        const uint32_t kend = min(nkb, (j + 1) * ckb);
        for (; kb < kend; ++kb) {
          const int s = kb % S;
          if (!mbar_wait(&full[s], (kb / S) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = sbase + s * G::STAGE;
          const uint32_t sb = sa + NT * G::A_TERM;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
            for (int pi = 0; pi < nprod(NT); ++pi) {
              const uint64_t ad =
                  smem_desc(sa + kProdA[pi] * G::A_TERM + kk * 2 * LBO_A, LBO_A, 128);
              const uint64_t bd =
                  smem_desc(sb + kProdB[pi] * G::B_TERM + kk * 2 * LBO_B, LBO_B, 128);
              mma_bf16(d, ad, bd, idesc, acc);
              acc = 1;
            }
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&accf[buf]);
      }
      mma_commit(done);  // every MMA issued above has completed when this arrives
      volatile int keep_waiting = 0;  // wait for in-flight MMAs even after an abort
      mbar_wait(done, 0, &keep_waiting, kTimeoutNs);
    }
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace tcg

// Tile configurations of the tensor-core GEMM: K blocks (of 64) per FP32
// accumulation chunk.  Tile 0 keeps one chunk for plain BF16 (its error is set
// by the BF16 rounding of the inputs) and 1024-K chunks for the split forms.
int num_tiles_tc() { return 3; }
int tc_chunk_kb(int math, int tile) {
  if (tile == 1) return 4;
  if (tile == 2) return 64;
  return math == TC_MATH_BF16 ? (1 << 30) : 16;
}

template <int NT>
static tc_status launch_tc_t(const GemmArgs& a, cudaStream_t s) {
  using G = tcg::Cfg<NT>;
  // The whole opt-in shared memory is requested: one CTA per SM (it owns all
  // 512 tensor-memory columns) and room beyond the last operand tile.
  static int smem_bytes = 0;
  if (smem_bytes == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return TC_ERR_CUDA;
    if (optin < (int)G::BYTES) return TC_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(tcg::k_gemm_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin) != cudaSuccess)
      return TC_ERR_CUDA;
    smem_bytes = optin;
  }
  const uint64_t tiles = (uint64_t)((a.M + tcg::BM - 1) / tcg::BM) *
                         (uint64_t)((a.N + tcg::BN - 1) / tcg::BN) * (uint64_t)a.nbatch;
  if (tiles == 0) return TC_OK;
  if (tiles > 0x7fffffffull) return TC_ERR_UNSUPPORTED;
  tcg::k_gemm_tc<NT><<<(unsigned)tiles, tcg::kThreads, smem_bytes, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_gemm_tc(const GemmArgs& a, int math, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (math) {
    case TC_MATH_BF16: return launch_tc_t<1>(a, s);
    case TC_MATH_BF16X3: return launch_tc_t<2>(a, s);
    case TC_MATH_BF16X6: return launch_tc_t<3>(a, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

}  // namespace tc
