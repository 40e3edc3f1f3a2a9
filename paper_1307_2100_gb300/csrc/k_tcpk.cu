// k_tcpk.cu -- the split-BF16 forms of a Class 3 contraction with packed
// operands: a pack pass and a GEMM fed by bulk copies (sm_103a, tcgen05).
//
// Same arithmetic as k_tc.cu (x = x0 + x1 + x2, BF16 terms of the residuals;
// BF16 keeps a0 b0, BF16x3 adds a0 b1 + a1 b0, BF16x6 adds a0 b2 + a1 b1 +
// a2 b0; the main product a0 b0 and the correction products in separate FP32
// accumulators, the main one emptied every K chunk into a compensated sum),
// but the FP32 operands are split once, not once per output tile:
//   k_bf16_pack<NT>  one CTA per (128-row tile, 128 K) of each operand:
//                    gathers the FP32 elements through the index groups,
//                    splits them into NT BF16 terms and writes, per 32-K
//                    block, NT canonical K-major blocks of 8 KB (byte
//                    (k / 8) * 2048 + row * 16 + (k % 8) * 2), term after term.
//   k_gemm_pk<NT>    persistent, one CTA per SM over 128 x 128 output tiles:
//                    warp 0     one thread moves each 32-K block of both
//                               operands (NT terms each) into a shared-memory
//                               ring with two bulk copies;
//                    warp 1     tensor-memory allocation; one thread issues
//                               the MMAs (main product into a double-buffered
//                               accumulator per K chunk, correction products
//                               into one accumulator per tile);
//                    warps 2-9  epilogue: two warps per lane quadrant, 64
//                               columns each; drain each K chunk into the
//                               compensated sum (TwoSum: high word in tensor
//                               memory, low word in registers); finish with
//                               hi + (lo + corrections), alpha, beta and a
//                               strided store.
// Tensor memory (512 columns): [0,256) main accumulators, [256,384) the
// correction accumulator, [384,512) the high word of the chunk sum.
#include <cuda.h>  // CUtensorMap and cuTensorMapEncodeTiled's types (entry point via the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "groups.cuh"
#include "sm100.cuh"
#include "storage.cuh"
#include "tc_internal.h"

namespace tc {

namespace pk {

constexpr int TILE = 128;
constexpr int BK = 32;                       // K per block (one stage)
constexpr int PK = 128;                      // K per pack CTA (4 blocks)
constexpr uint32_t TERM = TILE * BK * 2;     // bytes of one term of one block
constexpr int kPackThreads = 512;
constexpr int kRowThreads = kPackThreads / TILE;   // threads sharing one row (or one k)
constexpr int kLd = PK + 1;
constexpr uint32_t kPackSmem = TILE * kLd * 4 + 2 * TILE * 8;

constexpr int kEpiThreads = 256;
constexpr int kThreads = 64 + kEpiThreads;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t COL_CORR = 256, COL_HI = 384;
constexpr uint64_t kTimeoutNs = 2000000000ull;
constexpr uint32_t kRing = 192 * 1024;       // bytes of the stage ring

// A ring stage holds BPS consecutive 32-K blocks of A and of B.  Each stage
// costs a fixed hand-off (the producer's wait on its empty barrier, the MMA
// warp's wait on its full barrier, a commit), so forms whose stage holds few
// MMA cycles take two blocks per stage.
template <int NT>
struct Cfg {
  static constexpr int BPS = NT == 1 ? 4 : 2;  // blocks per stage
  static constexpr uint32_t STAGE = 2 * BPS * NT * TERM;  // A blocks then B blocks
  static constexpr int S = (int)(kRing / STAGE);      // 3, 3, 2
  static constexpr uint32_t OFF_COLC = S * STAGE;
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * TILE * 8;
  static constexpr uint32_t NBAR = 2 * S + 4 + 1;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;
};

struct PackArgs {
  Group gr[2];          // rows of operand o (the M and N groups); strides in slot o
  Group gk;             // K group; operand o's strides in slot o
  const void* in[2];    // elements of the pack kernel's input type
  uint8_t* q[2];        // [tile][block][term][TERM]
  int64_t rows[2];
  int64_t K;
  int64_t nblocks0;     // CTAs of operand 0
  int32_t tiles[2];
  int32_t nkb;          // 32-K blocks
  int32_t npk;          // pack CTAs per tile (128 K each)
  int32_t rows_fast[2];
};

// Shared memory of one pack CTA: the FP32 block and its row / K offsets.
struct PackSmem {
  float* tile;
  int64_t* roff;
  int64_t* koff;
};

__device__ __forceinline__ PackSmem pack_smem(float4* raw) {
  PackSmem m;
  m.tile = reinterpret_cast<float*>(raw);
  m.roff = reinterpret_cast<int64_t*>(m.tile + TILE * kLd);
  m.koff = m.roff + TILE;
  return m;
}

// Rows [128 t, 128 t + 128) x K [128 kc, 128 kc + 128) of operand o (strides
// in slot o of gr and gk), split into NT BF16 terms (F16T: rounded to one
// FP16 term) and stored in the operand's packed blocks Q (block kb of tile t
// at (t * nkb + kb) * NT * TERM).  In: FP32, BF16 or FP16 elements.
template <int NT, typename In, bool F16T>
__device__ __forceinline__ void pack_body(const Group& gr, const Group& gk, int o,
                                          const In* __restrict__ X, int64_t rows, int64_t K,
                                          int t, int kc, int nkb, bool rows_fast,
                                          uint8_t* __restrict__ Qop, const PackSmem& sm) {
  float* tile = sm.tile;
  int64_t* roff = sm.roff;
  int64_t* koff = sm.koff;
  const int tid = threadIdx.x;
  if (tid < TILE) {
    const int64_t r = (int64_t)t * TILE + tid;
    roff[tid] = r < rows ? goff(gr, o, (uint32_t)r) : -1;
  } else if (tid < 2 * TILE) {
    const int64_t k = (int64_t)kc * PK + (tid - TILE);
    koff[tid - TILE] = k < K ? goff(gk, o, (uint32_t)k) : -1;
  }
  __syncthreads();

  // gather: all of a thread's loads in flight, then their stores
  constexpr int NJ = TILE * PK / kPackThreads;
  if (rows_fast) {
    const int r = tid & (TILE - 1), k0 = tid / TILE;
    const int64_t ro = roff[r];
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int64_t ko = koff[k0 + kRowThreads * j];
      v[j] = (ro >= 0 && ko >= 0) ? ld_c(__ldg(X + ro + ko)) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) tile[r * kLd + k0 + kRowThreads * j] = v[j];
  } else {
    const int k = tid & (PK - 1), r0 = tid / PK;
    const int64_t ko = koff[k];
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int64_t ro = roff[r0 + kRowThreads * j];
      v[j] = (ro >= 0 && ko >= 0) ? ld_c(__ldg(X + ro + ko)) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) tile[(r0 + kRowThreads * j) * kLd + k] = v[j];
  }
  __syncthreads();

  // split and store: unit u = (k8 chunk) * 128 + row is one 16-byte row of a
  // core matrix (8 BF16 along K), at byte u * 16 of its term block
  const int nb = min(PK / BK, nkb - kc * (PK / BK));   // blocks of this CTA
  uint8_t* __restrict__ Q = Qop + ((int64_t)t * nkb + (int64_t)kc * (PK / BK)) * NT * TERM;
  for (int u = tid; u < nb * (BK / 8) * TILE; u += kPackThreads) {
    const int blk = u / ((BK / 8) * TILE);
    const int w = u % ((BK / 8) * TILE);
    const int c8 = w >> 7, r = w & (TILE - 1);
    const float* src = tile + r * kLd + blk * BK + c8 * 8;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = src[i];
    uint8_t* dst = Q + (size_t)blk * NT * TERM + (size_t)w * 16;
    static_assert(!F16T || NT == 1, "the FP16 form has one term");
#pragma unroll
    for (int tt = 0; tt < NT; ++tt) {
      uint32_t wd[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        wd[i] = F16T ? pack_f16x2(v[2 * i], v[2 * i + 1]) : pack_bf16x2(v[2 * i], v[2 * i + 1]);
        if (tt + 1 < NT) {  // exact FP32 residuals
          v[2 * i] = __fsub_rn(v[2 * i], bf16_lo(wd[i]));
          v[2 * i + 1] = __fsub_rn(v[2 * i + 1], bf16_hi(wd[i]));
        }
      }
      *reinterpret_cast<uint4*>(dst + (size_t)tt * TERM) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
  }
}

template <int NT, typename In, bool F16T>
__global__ void __launch_bounds__(kPackThreads) k_bf16_pack(const __grid_constant__ PackArgs P) {
  extern __shared__ float4 pk_smem[];
  int64_t bid = blockIdx.x;
  const int o = bid < P.nblocks0 ? 0 : 1;
  if (o) bid -= P.nblocks0;
  const int t = (int)(bid / P.npk), kc = (int)(bid % P.npk);
  pack_body<NT, In, F16T>(P.gr[o], P.gk, o, static_cast<const In*>(P.in[o]), P.rows[o], P.K, t,
                          kc, P.nkb, P.rows_fast[o] != 0, P.q[o], pack_smem(pk_smem));
}

// Batched pack pass: one CTA per entry (item, operand, row tile, 128-K
// chunk); the item's index groups are copied to shared memory first.
struct PackWork {
  int32_t item, o, t, kc;
};

template <int NT>
__global__ void __launch_bounds__(kPackThreads) k_bf16_pack_batch(
    const GemmArgs* __restrict__ items, const PkItem* __restrict__ pk, const PackWork* work,
    const void* const* Ap, const void* const* Bp) {
  extern __shared__ float4 pk_smem[];
  __shared__ Group sg[2];
  const PackWork wk = work[blockIdx.x];
  const GemmArgs& a = items[wk.item];
  {
    const uint32_t* src0 = reinterpret_cast<const uint32_t*>(wk.o ? &a.gn : &a.gm);
    const uint32_t* src1 = reinterpret_cast<const uint32_t*>(&a.gk);
    uint32_t* d0 = reinterpret_cast<uint32_t*>(&sg[0]);
    uint32_t* d1 = reinterpret_cast<uint32_t*>(&sg[1]);
    for (int i = threadIdx.x; i < (int)(sizeof(Group) / 4); i += kPackThreads) {
      d0[i] = src0[i];
      d1[i] = src1[i];
    }
  }
  __syncthreads();
  const bool sw = a.swapped != 0;
  const float* X = static_cast<const float*>(
      wk.o == 0 ? (sw ? Bp[wk.item] : Ap[wk.item]) : (sw ? Ap[wk.item] : Bp[wk.item]));
  const PkItem& it = pk[wk.item];
  pack_body<NT, float, false>(sg[0], sg[1], wk.o, X, wk.o ? a.N : a.M, a.K, wk.t, wk.kc, it.nkb,
                (wk.o ? a.b_contig : a.a_contig) == CONTIG_MN,
                const_cast<uint8_t*>(wk.o ? it.qb : it.qa), pack_smem(pk_smem));
}

// One GEMM on packed operands (a single contraction, or one item of a batch).
// The launch holds it in kernel parameters, a batch in device memory.
struct PkLaunch {
  CUtensorMap tma_a, tma_b;  // CTA pairs: the packed operands as rows of 2 KB
  PkItem single;             // items == nullptr: tiles 0 .. nwork - 1 of this GEMM
  void* C;                   // elements of out_type
  float alpha, beta;
  uint32_t idesc;            // MMA instruction descriptor (BF16 or FP16 operands)
  int32_t out_type;          // C's storage: 0 FP32, 1 BF16, 2 FP16 (batches: FP32)
  const PkItem* items;       // batch: per-item GEMMs and (item, tile, K range) work entries
  const int32_t* work;
  void* const* Cp;
  const double* alpha_p;
  const double* beta_p;
  int64_t nwork;
};

// The tile and K range of work entry w (one contraction: split-major, the
// ksplit ranges of every tile; a batch: as listed in its work entries).
struct Job {
  const PkItem* it;
  int tm, tn;
  int64_t tile;
  int split, k0, k1;  // K blocks [k0, k1)
  void* C;
  float alpha, beta;
};

__device__ __forceinline__ Job job_of(const PkLaunch& L, int64_t w) {
  Job j;
  int64_t tile = w;
  j.split = 0;
  if (L.items) {
    const int32_t item = L.work[3 * w];
    tile = L.work[3 * w + 1];
    j.split = L.work[3 * w + 2];
    j.it = L.items + item;
    j.C = L.Cp[item];
    j.alpha = (float)L.alpha_p[item];
    j.beta = (float)L.beta_p[item];
  } else {
    j.it = &L.single;
    j.C = L.C;
    j.alpha = L.alpha;
    j.beta = L.beta;
    const int64_t ntiles = (int64_t)L.single.tiles_m * L.single.tiles_n;
    j.split = (int)(w / ntiles);
    tile = w % ntiles;
  }
  const PkItem& P = *j.it;
  j.tile = tile;
  // balanced K ranges, none empty (ksplit <= nkb)
  j.k0 = (int)((int64_t)j.split * P.nkb / P.ksplit);
  j.k1 = (int)((int64_t)(j.split + 1) * P.nkb / P.ksplit);
  if (P.raster) {
    j.tn = (int)(tile % P.tiles_n);
    j.tm = (int)(tile / P.tiles_n);
  } else {
    j.tm = (int)(tile % P.tiles_m);
    j.tn = (int)(tile / P.tiles_m);
  }
  return j;
}

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

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  bool ok = (*abort == 0) && mbar_wait(bar, parity, abort, kTimeoutNs);
  return __all_sync(0xffffffffu, ok);
}

// C[off] = x (+ beta * C[off]) in C's storage type, rounded to nearest even.
__device__ __forceinline__ void store_out(void* C, int64_t off, int out_type, float x,
                                          float beta) {
  if (out_type == 0) {
    float* d = static_cast<float*>(C) + off;
    if (beta != 0.0f) x = fmaf(beta, *d, x);
    *d = x;
  } else if (out_type == 1) {
    __nv_bfloat16* d = static_cast<__nv_bfloat16*>(C) + off;
    if (beta != 0.0f) x = fmaf(beta, __bfloat162float(*d), x);
    *d = __float2bfloat16_rn(x);
  } else {
    __half* d = static_cast<__half*>(C) + off;
    if (beta != 0.0f) x = fmaf(beta, __half2float(*d), x);
    *d = __float2half_rn(x);
  }
}

// C[rc + ch[i]] = alpha * v[i] (+ beta * C[...]) for NC columns of one row,
// in C's storage type O (columns with ch[i] < 0 lie outside C).  One unrolled
// loop per storage type keeps the epilogue's registers for its sums.
template <typename O, int NC>
__device__ __forceinline__ void store_row(void* C, int64_t rc, const int64_t* ch,
                                          const float (&v)[NC], float alpha, float beta) {
  O* Cr = static_cast<O*>(C) + rc;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int64_t ci = ch[i];
    if (ci < 0) continue;
    float x = alpha * v[i];
    if (beta != 0.0f) x = fmaf(beta, ld_c(Cr[ci]), x);
    Cr[ci] = st_cf<O>(x);
  }
}

// s + e == a + b exactly (Knuth's TwoSum).  When s is infinite or NaN (an
// FP16 operand overflowed, or the data hold infinities) e is 0, so that the
// compensation keeps the infinity instead of turning it into a NaN.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
  if (!(fabsf(s) <= 3.402823466e38f)) e = 0.0f;
  return s;
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_pk(const __grid_constant__ PkLaunch L) {
  using G = Cfg<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t pk_gemm_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(pk_gemm_raw) + 1023) & ~(uintptr_t)1023);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + G::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], kEpiThreads);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  constexpr uint32_t OPB = NT * TERM;          // bytes of one operand's block

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      uint32_t g = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; ok && w < L.nwork; w += gridDim.x) {
        const Job J = job_of(L, w);
        const int nkb = J.it->nkb;
        const uint8_t* a = J.it->qa + (size_t)J.tm * nkb * OPB;
        const uint8_t* b = J.it->qb + (size_t)J.tn * nkb * OPB;
        for (int kb = J.k0; kb < J.k1; kb += G::BPS, ++g) {
          const int s = (int)(g % S);
          if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          // blocks [kb, kb + nb): consecutive, so one copy per operand
          const uint32_t nb = (uint32_t)min(G::BPS, J.k1 - kb);
          const uint32_t dst = sbase + (uint32_t)s * G::STAGE;
          mbar_arrive_expect_tx(&full[s], 2 * nb * OPB);
          bulk_g2s(dst, a + (size_t)kb * OPB, nb * OPB, &full[s]);
          bulk_g2s(dst + G::BPS * OPB, b + (size_t)kb * OPB, nb * OPB, &full[s]);
        }
      }
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&full[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issue
      const uint32_t idesc = L.idesc;
      constexpr uint32_t LBO = (TILE / 8) * 128;
      uint32_t g = 0, gc = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; ok && w < L.nwork; w += gridDim.x) {
        const Job J = job_of(L, w);
        const int ckb = max(J.it->chunk_kb, 1);
        const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
        // the correction accumulator and both main buffers are free once the
        // previous tile's last chunk has been drained
        if (gc >= 1 && !mbar_wait(&acce[(gc - 1) & 1], ((gc - 1) >> 1) & 1, abort, kTimeoutNs)) {
          ok = false;
          break;
        }
        int kb = J.k0;
        for (int j = 0; ok && j < nchunks; ++j, ++gc) {
          const uint32_t buf = gc & 1;
          if (gc >= 2 && !mbar_wait(&acce[buf], ((gc >> 1) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dmain = tmem + buf * TILE;
          const int kend = min(J.k1, J.k0 + (j + 1) * ckb), kstart = kb;
          // stages start at the range's first block and hold BPS blocks;
          // chunks hold a multiple of BPS blocks, so no stage straddles one
          for (; kb < kend; kb += G::BPS, ++g) {
            const int s = (int)(g % S);
            if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const int nb = min(G::BPS, kend - kb);
            for (int bi = 0; bi < nb; ++bi) {
              const uint32_t sa = sbase + (uint32_t)s * G::STAGE + bi * OPB;
              const uint32_t sb = sa + G::BPS * OPB;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const bool first = bi == 0 && kk == 0;
                mma_bf16(dmain, smem_desc(sa + kk * 2 * LBO, LBO, 128),
                         smem_desc(sb + kk * 2 * LBO, LBO, 128), idesc,
                         (kb > kstart || !first) ? 1u : 0u);
#pragma unroll
                for (int pi = 1; pi < nprod(NT); ++pi)
                  mma_bf16(tmem + COL_CORR,
                           smem_desc(sa + prod_a(pi) * TERM + kk * 2 * LBO, LBO, 128),
                           smem_desc(sb + prod_b(pi) * TERM + kk * 2 * LBO, LBO, 128), idesc,
                           (kb > J.k0 || !first || pi > 1) ? 1u : 0u);
              }
            }
            mma_commit(&empty[s]);
          }
          if (!ok) break;
          mma_commit(&accf[buf]);
        }
      }
      mma_commit(done);
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int ew = warp - 2;
    const int q = warp & 3;
    const int h = ew >> 2;
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)h * 64;
    uint32_t gc = 0;
    int64_t it = 0;
    bool live = true;  // after a wait gave up, tiles are walked without work so
                       // that every epilogue warp still meets each named barrier
    // A tile's setup (its job, the C offsets of its columns and of this
    // thread's row) is done one tile ahead, while the MMAs of the tile before
    // run: column offsets go to the other half of the double-buffered table.
    auto setup = [&](int64_t w, int64_t* cc, Job& J, int64_t& rc) {
      J = job_of(L, w);
      const PkItem& P = *J.it;
      if (etid < TILE) {
        const int64_t n = (int64_t)J.tn * TILE + etid;
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      const int64_t m = (int64_t)J.tm * TILE + row;
      rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
    };
    Job Jn;
    int64_t rcn = -1;
    if (blockIdx.x < L.nwork) setup(blockIdx.x, colC, Jn, rcn);
    named_bar_sync(1, kEpiThreads);
    for (int64_t w = blockIdx.x; w < L.nwork; w += gridDim.x, ++it) {
      const Job J = Jn;
      const int64_t rc = rcn;
      const PkItem& P = *J.it;
      int64_t* cc = colC + (it & 1) * TILE;
      // the other half was last read by the stores of the tile before, which
      // every epilogue thread finished before the barrier that ended it
      if (w + gridDim.x < L.nwork) setup(w + gridDim.x, colC + ((it + 1) & 1) * TILE, Jn, rcn);
      if (!live) {
        named_bar_sync(1, kEpiThreads);
        continue;
      }
      const int ckb = max(P.chunk_kb, 1);
      const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
      const bool partial = P.ksplit > 1;
      // partial sums of this K range: [split][tile][col][row], the compensated
      // pair (s, r) in FP32 (the FP64 sum is formed by the reduction)
      float2* pp = partial ? P.part + ((size_t)J.split * P.tiles_m * P.tiles_n + J.tile) *
                                          (size_t)(TILE * TILE) + (size_t)h * 64 * TILE + row
                           : nullptr;
      float lo[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) lo[i] = 0.0f;
      for (int j = 0; j < nchunks; ++j, ++gc) {
        const uint32_t buf = gc & 1;
        if (!warp_wait(&accf[buf], (gc >> 1) & 1, abort)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t tmain = tl + buf * TILE;
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
          tc_fence_before();
          mbar_arrive(&acce[buf]);
        } else {
          // the finished sums replace the low words in lo[]
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t mv[16], hv[16], cv[16];
            tmem_ld16(tmain + c * 16, mv);
            if (j > 0) tmem_ld16(tl + COL_HI + c * 16, hv);
            if (NT > 1) tmem_ld16(tl + COL_CORR + c * 16, cv);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float hi0 = j > 0 ? __uint_as_float(hv[i]) : 0.0f;
              float e;
              const float s = two_sum(hi0, __uint_as_float(mv[i]), e);
              float r = __fadd_rn(lo[c * 16 + i], e);
              if (NT > 1) r = __fadd_rn(r, __uint_as_float(cv[i]));
              if (partial) pp[(size_t)(c * 16 + i) * TILE] = make_float2(s, r);
              else lo[c * 16 + i] = __fadd_rn(s, r);
            }
          }
          tc_fence_before();
          mbar_arrive(&acce[buf]);  // main, correction and high word are free
          if (!partial && rc >= 0) {
            const int64_t* ch = cc + h * 64;
            if (L.out_type == 0) store_row<float, 64>(J.C, rc, ch, lo, J.alpha, J.beta);
            else if (L.out_type == 1)
              store_row<__nv_bfloat16, 64>(J.C, rc, ch, lo, J.alpha, J.beta);
            else store_row<__half, 64>(J.C, rc, ch, lo, J.alpha, J.beta);
          }
        }
      }
      named_bar_sync(1, kEpiThreads);  // this tile's columns read; the next tile's written
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Wide tiles (tile configuration 4): 128 x 256 outputs per CTA for the BF16,
// FP16 and BF16x3 forms.  Every product of a K chunk goes into one FP32
// accumulator of 256 columns; tensor memory double-buffers it ([0,256) and
// [256,512), each two N = 128 halves), and eight epilogue warps (one lane
// quadrant and 128 columns each) add every drained chunk into a running FP32
// sum held in registers.  The tensor cores' FP32 accumulation is not round-to-nearest, so
// its error grows with the number of blocks it adds: BF16x3 drains every
// 256 K (as the 128 x 128 kernel does), BF16 and FP16 (whose error is their
// operands' rounding) once per tile.  A 32-K block moves NT x 8 KB of A for
// NT x 16 KB of B: 27 % fewer operand bytes per multiply-add than the
// 128 x 128 tile; each stage's A block is shared by the two N = 128 MMAs of
// the two halves.  BF16x6 is not taken here: its FP32-class sum needs the
// separate correction accumulator, for which there is no room (it runs on the
// 128 x 128 tiles, or on CTA pairs over 256 x 128 tiles).
// ---------------------------------------------------------------------------
constexpr int TILE_W = 256;

template <int NT>
struct CfgW {
  static constexpr int BPS = NT == 1 ? 2 : 1;                 // 32-K blocks per stage
  static constexpr uint32_t OPA = NT * TERM;                   // one block of A (NT terms)
  static constexpr uint32_t OPH = NT * TERM;                   // one block of one B half
  static constexpr uint32_t STAGE = BPS * (OPA + 2 * OPH);     // A blocks, B half 0, B half 1
  static constexpr int S = (int)(kRing / STAGE);               // 4 stages of 48 KB
  static constexpr uint32_t OFF_COLC = S * STAGE;              // int64 colC[2][256]
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * TILE_W * 8;
  static constexpr uint32_t NBAR = 2 * S + 4 + 1;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;
};

// Work entry w of a wide launch: split-major over the 128 x 256 tiles of one
// GEMM (n-pairs fastest when raster, else m-tiles fastest).
struct JobW {
  int tm, tn0;       // 128-row tile of A; first of the two 128-column tiles of B
  bool h1;           // the second half exists (tn0 + 1 < tiles_n)
  int split, k0, k1;
};

__device__ __forceinline__ JobW jobw_of(const PkItem& P, int64_t w) {
  JobW j;
  const int tn2 = (P.tiles_n + 1) / 2;
  const int64_t ntiles = (int64_t)P.tiles_m * tn2;
  j.split = (int)(w / ntiles);
  const int64_t t = w % ntiles;
  int tp;
  if (P.raster) {
    tp = (int)(t % tn2);
    j.tm = (int)(t / tn2);
  } else {
    j.tm = (int)(t % P.tiles_m);
    tp = (int)(t / P.tiles_m);
  }
  j.tn0 = 2 * tp;
  j.h1 = j.tn0 + 1 < P.tiles_n;
  j.k0 = (int)((int64_t)j.split * P.nkb / P.ksplit);
  j.k1 = (int)((int64_t)(j.split + 1) * P.nkb / P.ksplit);
  return j;
}

// Index of 128 x 128 tile (tm, tn) in the split-K partial buffer, in the
// order k_pk_reduce reads it.
__device__ __forceinline__ int64_t tile128_index(const PkItem& P, int tm, int tn) {
  return P.raster ? (int64_t)tm * P.tiles_n + tn : (int64_t)tn * P.tiles_m + tm;
}

constexpr int kEpiThreadsW = 256;
constexpr int kThreadsW = 64 + kEpiThreadsW;

template <int NT>
__global__ void __launch_bounds__(kThreadsW, 1) k_gemm_pkw(const __grid_constant__ PkLaunch L) {
  using G = CfgW<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t pkw_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(pkw_raw) + 1023) & ~(uintptr_t)1023);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + G::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);
  const PkItem& P = L.single;
  const int ckb = max(P.chunk_kb, 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], kEpiThreadsW);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      uint32_t g = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; ok && w < L.nwork; w += gridDim.x) {
        const JobW J = jobw_of(P, w);
        const uint8_t* a = P.qa + (size_t)J.tm * P.nkb * G::OPA;
        const uint8_t* b0 = P.qb + (size_t)J.tn0 * P.nkb * G::OPH;
        const uint8_t* b1 = b0 + (size_t)P.nkb * G::OPH;
        for (int kb = J.k0; kb < J.k1; kb += G::BPS, ++g) {
          const int s = (int)(g % S);
          if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          const uint32_t nb = (uint32_t)min(G::BPS, J.k1 - kb);
          const uint32_t dst = sbase + (uint32_t)s * G::STAGE;
          mbar_arrive_expect_tx(&full[s], nb * (G::OPA + (J.h1 ? 2 : 1) * G::OPH));
          bulk_g2s(dst, a + (size_t)kb * G::OPA, nb * G::OPA, &full[s]);
          bulk_g2s(dst + G::BPS * G::OPA, b0 + (size_t)kb * G::OPH, nb * G::OPH, &full[s]);
          if (J.h1)
            bulk_g2s(dst + G::BPS * (G::OPA + G::OPH), b1 + (size_t)kb * G::OPH, nb * G::OPH,
                     &full[s]);
        }
      }
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&full[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issue
      // chunk gc (counted over the launch) goes to accumulator buffer gc % 2,
      // free once the epilogue drained chunk gc - 2
      const uint32_t idesc = L.idesc;
      constexpr uint32_t LBO = (TILE / 8) * 128;
      uint32_t g = 0, gc = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; ok && w < L.nwork; w += gridDim.x) {
        const JobW J = jobw_of(P, w);
        const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
        int kb = J.k0;
        for (int j = 0; ok && j < nchunks; ++j, ++gc) {
          const uint32_t buf = gc & 1;
          if (gc >= 2 && !mbar_wait(&acce[buf], ((gc >> 1) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + buf * TILE_W;
          const int kend = min(J.k1, J.k0 + (j + 1) * ckb), kstart = kb;
          for (; kb < kend; kb += G::BPS, ++g) {
            const int s = (int)(g % S);
            if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const int nb = min(G::BPS, kend - kb);
            const uint32_t st = sbase + (uint32_t)s * G::STAGE;
            for (int bi = 0; bi < nb; ++bi) {
              const uint32_t sa = st + bi * G::OPA;
              const uint32_t sb0 = st + G::BPS * G::OPA + bi * G::OPH;
              const uint32_t sb1 = sb0 + G::BPS * G::OPH;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                for (int pi = 0; pi < nprod(NT); ++pi) {
                  const uint32_t acc = (kb > kstart || bi > 0 || kk > 0 || pi > 0) ? 1u : 0u;
                  const uint64_t da = smem_desc(sa + prod_a(pi) * TERM + kk * 2 * LBO, LBO, 128);
                  mma_bf16(dacc, da,
                           smem_desc(sb0 + prod_b(pi) * TERM + kk * 2 * LBO, LBO, 128), idesc,
                           acc);
                  if (J.h1)
                    mma_bf16(dacc + TILE, da,
                             smem_desc(sb1 + prod_b(pi) * TERM + kk * 2 * LBO, LBO, 128), idesc,
                             acc);
                }
              }
            }
            mma_commit(&empty[s]);
          }
          if (!ok) break;
          mma_commit(&accf[buf]);
        }
      }
      mma_commit(done);
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    // warps 2-9: lane quadrant q = warp % 4 and N-half hh = (warp - 2) / 4;
    // each thread owns one row and the 128 columns of its half, whose running
    // sums stay in registers
    const int ew = warp - 2;
    const int q = warp & 3;
    const int hh = ew >> 2;
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    uint32_t gc = 0, it = 0;
    bool live = true;
    auto setup = [&](int64_t w, int64_t* cc, JobW& J, int64_t& rc) {
      J = jobw_of(P, w);
      if (etid < TILE_W) {
        const int64_t n = (int64_t)J.tn0 * TILE + etid;
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      const int64_t m = (int64_t)J.tm * TILE + row;
      rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
    };
    JobW Jn;
    int64_t rcn = -1;
    if (blockIdx.x < L.nwork) setup(blockIdx.x, colC, Jn, rcn);
    named_bar_sync(1, kEpiThreadsW);
    for (int64_t w = blockIdx.x; w < L.nwork; w += gridDim.x, ++it) {
      const JobW J = Jn;
      const int64_t rc = rcn;
      int64_t* cc = colC + (it & 1) * TILE_W;
      if (w + gridDim.x < L.nwork)
        setup(w + gridDim.x, colC + ((it + 1) & 1) * TILE_W, Jn, rcn);
      if (!live) {
        named_bar_sync(1, kEpiThreadsW);
        continue;
      }
      const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
      float hi[128];
      for (int j = 0; j < nchunks; ++j, ++gc) {
        const uint32_t buf = gc & 1;
        if (!warp_wait(&accf[buf], (gc >> 1) & 1, abort)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * TILE_W + hh * TILE;
        if (j == 0) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t r[16];
            tmem_ld16(tl + c * 16, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) hi[c * 16 + i] = __uint_as_float(r[i]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t r[16];
            tmem_ld16(tl + c * 16, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) hi[c * 16 + i] = __fadd_rn(hi[c * 16 + i],
                                                                    __uint_as_float(r[i]));
          }
        }
        tc_fence_before();
        mbar_arrive(&acce[buf]);  // this buffer may take the chunk after next
      }
      if (live && (hh == 0 || J.h1)) {
        if (P.ksplit > 1) {
          float2* pp = P.part + ((size_t)J.split * P.tiles_m * P.tiles_n +
                                 tile128_index(P, J.tm, J.tn0 + hh)) * (size_t)(TILE * TILE) +
                       row;
#pragma unroll
          for (int i = 0; i < 128; ++i) pp[(size_t)i * TILE] = make_float2(hi[i], 0.0f);
        } else if (rc >= 0) {
          const int64_t* ch = cc + hh * TILE;
          if (L.out_type == 0) store_row<float, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
          else if (L.out_type == 1)
            store_row<__nv_bfloat16, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
          else store_row<__half, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
        }
      }
      named_bar_sync(1, kEpiThreadsW);  // this tile's columns read; the next tile's written
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// CTA pairs on 256 x 256 tiles (tile configuration 5): the arithmetic of the
// wide tiles (BF16, FP16, BF16x3: every product of a chunk into one FP32
// accumulator, chunks added in registers), with two SMs on one tile.  Each
// CTA of the pair holds its own 128 rows of A and its own 128-row half of B;
// one thread of the first CTA issues tcgen05.mma.cta_group::2 (M = 256,
// N = 256), which reads both CTAs' shared memory and leaves each CTA's 128
// rows of D in that CTA's tensor memory.  A 32-K block thus moves NT x 16 KB
// per SM for a 128 x 256 share of the outputs, against NT x 24 KB on the
// wide tiles: a third fewer operand bytes per SM per multiply-add.
// Hand-offs: each CTA's producer fills its own ring with tiled TMA loads
// (tensor maps viewing the packed operands as rows of 2 KB) that complete on
// the first CTA's full barrier (cta_group::2), whose expected byte count
// covers both CTAs' loads; the MMA thread's commits arrive on both CTAs'
// empty and accf barriers; both CTAs' epilogues arrive on the first CTA's
// acce barrier.
// ---------------------------------------------------------------------------
template <int NT>
struct CfgP {
  static constexpr int BPS = NT == 1 ? 4 : 1;                 // 32-K blocks per stage
  static constexpr uint32_t OPA = NT * TERM;                   // own A block (128 rows)
  static constexpr uint32_t OPB = NT * TERM;                   // own B half block (128 rows)
  static constexpr uint32_t STAGE = BPS * (OPA + OPB);         // A blocks, then B blocks
  static constexpr int S = (int)(kRing / STAGE);               // 3 x 64 KB, 6 x 32 KB, 4 x 48 KB
  static constexpr uint32_t OFF_COLC = S * STAGE;              // int64 colC[2][256]
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * TILE_W * 8;
  static constexpr uint32_t NBAR = 2 * S + 4 + 1;              // full, empty, acc*, done
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;
};

// Work entry w of a pair launch: split-major over 256 x 256 pair tiles; with
// a tail split, whole tiles first, then the tail tiles' K ranges.
struct JobP {
  int tmp, tnp;       // pair tile: A tiles 2 tmp, 2 tmp + 1; B tiles 2 tnp, 2 tnp + 1
  int split, k0, k1;
  int tail;           // tail split: the tail tile's index (-1: a whole tile)
};

__device__ __forceinline__ JobP jobp_of(const PkItem& P, int64_t w) {
  JobP j;
  const int mp = (P.tiles_m + 1) / 2, np = (P.tiles_n + 1) / 2;
  const int64_t ntiles = (int64_t)mp * np;
  j.tail = -1;
  int64_t t;
  if (P.tsplit > 1) {
    if (w < P.nfull) {
      t = w;
      j.split = 0;
      j.k0 = 0;
      j.k1 = P.nkb;
    } else {
      const int64_t r = w - P.nfull;
      j.tail = (int)(r / P.tsplit);
      t = P.nfull + j.tail;
      j.split = (int)(r % P.tsplit);
      j.k0 = (int)((int64_t)j.split * P.nkb / P.tsplit);
      j.k1 = (int)((int64_t)(j.split + 1) * P.nkb / P.tsplit);
    }
    if (P.raster) {
      j.tnp = (int)(t % np);
      j.tmp = (int)(t / np);
    } else {
      j.tmp = (int)(t % mp);
      j.tnp = (int)(t / mp);
    }
    return j;
  }
  j.split = (int)(w / ntiles);
  t = w % ntiles;
  if (P.raster) {
    j.tnp = (int)(t % np);
    j.tmp = (int)(t / np);
  } else {
    j.tmp = (int)(t % mp);
    j.tnp = (int)(t / mp);
  }
  j.k0 = (int)((int64_t)j.split * P.nkb / P.ksplit);
  j.k1 = (int)((int64_t)(j.split + 1) * P.nkb / P.ksplit);
  return j;
}

template <int NT>
__global__ void __launch_bounds__(kThreadsW, 1) k_gemm_pkp(const __grid_constant__ PkLaunch L) {
  using G = CfgP<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t pkp_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(pkp_raw) + 1023) & ~(uintptr_t)1023);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + G::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);
  const PkItem& P = L.single;
  const int ckb = max(P.chunk_kb, 1);
  const uint32_t rank = cluster_ctarank();
  const bool lead = rank == 0;
  const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 2 * kEpiThreadsW);  // both CTAs' epilogue threads
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync();  // both CTAs' barriers exist before any remote arrival
  if (warp == 1) tmem_alloc2(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      // this CTA's 128 rows of A and its 128-row half of B, into its own ring;
      // the loads of both CTAs complete on the first CTA's full barrier
      uint32_t g = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < L.nwork; w += npairs) {
        const JobP J = jobp_of(P, w);
        const int tm0 = 2 * J.tmp, tn0 = 2 * J.tnp;
        const int tm = tm0 + (int)rank, tn = tn0 + (int)rank;
        const bool va = tm < P.tiles_m, vb = tn < P.tiles_n;   // else: rows the pair discards
        const uint32_t pair_block = (tm0 < P.tiles_m ? G::OPA : 0u) +
                                    (tm0 + 1 < P.tiles_m ? G::OPA : 0u) +
                                    (tn0 < P.tiles_n ? G::OPB : 0u) +
                                    (tn0 + 1 < P.tiles_n ? G::OPB : 0u);
        for (int kb = J.k0; kb < J.k1; kb += G::BPS, ++g) {
          const int s = (int)(g % S);
          if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          const int nb = min(G::BPS, J.k1 - kb);
          const uint32_t dst = sbase + (uint32_t)s * G::STAGE;
          if (lead) mbar_arrive_expect_tx(&full[s], (uint32_t)nb * pair_block);
          const uint32_t mb = mapa_shared(smem_u32(&full[s]), 0);
          for (int bi = 0; bi < nb; ++bi) {
            if (va)
              tma_load_2d_pair(dst + bi * G::OPA, &L.tma_a, 0,
                               (int32_t)(((int64_t)tm * P.nkb + kb + bi) * (G::OPA / 2048)), mb);
            if (vb)
              tma_load_2d_pair(dst + G::BPS * G::OPA + bi * G::OPB, &L.tma_b, 0,
                               (int32_t)(((int64_t)tn * P.nkb + kb + bi) * (G::OPB / 2048)), mb);
          }
        }
      }
      // before exit: the pair's last commits have arrived on this CTA's empty
      // barriers (so its MMAs, and the loads they read, are done)
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&empty[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // ------------------------------------------- MMA issue (first CTA)
      const uint32_t idesc = L.idesc;
      constexpr uint32_t LBO = (TILE / 8) * 128;
      uint32_t g = 0, gc = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < L.nwork; w += npairs) {
        const JobP J = jobp_of(P, w);
        const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
        int kb = J.k0;
        for (int j = 0; ok && j < nchunks; ++j, ++gc) {
          const uint32_t buf = gc & 1;
          // both CTAs' epilogues drained chunk gc - 2 of this buffer
          if (gc >= 2 && !mbar_wait(&acce[buf], ((gc >> 1) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dacc = tmem + buf * TILE_W;
          const int kend = min(J.k1, J.k0 + (j + 1) * ckb), kstart = kb;
          for (; kb < kend; kb += G::BPS, ++g) {
            const int s = (int)(g % S);
            if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const int nb = min(G::BPS, kend - kb);
            const uint32_t st = sbase + (uint32_t)s * G::STAGE;
            for (int bi = 0; bi < nb; ++bi) {
              const uint32_t sa = st + bi * G::OPA;
              const uint32_t sb = st + G::BPS * G::OPA + bi * G::OPB;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                for (int pi = 0; pi < nprod(NT); ++pi) {
                  const uint32_t acc = (kb > kstart || bi > 0 || kk > 0 || pi > 0) ? 1u : 0u;
                  mma_bf16_pair(dacc, smem_desc(sa + prod_a(pi) * TERM + kk * 2 * LBO, LBO, 128),
                                smem_desc(sb + prod_b(pi) * TERM + kk * 2 * LBO, LBO, 128),
                                idesc, acc);
                }
              }
            }
            mma_commit_pair(&empty[s], 3);  // both CTAs may refill this stage
          }
          if (!ok) break;
          mma_commit_pair(&accf[buf], 3);   // both CTAs' epilogues may drain it
        }
      }
      mma_commit_pair(done, 1);
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    // warps 2-9 of each CTA: lane quadrant q = warp % 4 and N-half hh =
    // (warp - 2) / 4 of this CTA's 128 rows x 256 columns
    const int ew = warp - 2;
    const int q = warp & 3;
    const int hh = ew >> 2;
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    uint32_t gc = 0, it = 0;
    bool live = true;
    auto setup = [&](int64_t w, int64_t* cc, JobP& J, int64_t& rc) {
      J = jobp_of(P, w);
      if (etid < TILE_W) {
        const int64_t n = (int64_t)J.tnp * TILE_W + etid;
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      const int64_t m = (int64_t)(2 * J.tmp + (int)rank) * TILE + row;
      rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
    };
    JobP Jn;
    int64_t rcn = -1;
    if (pair < L.nwork) setup(pair, colC, Jn, rcn);
    named_bar_sync(1, kEpiThreadsW);
    for (int64_t w = pair; w < L.nwork; w += npairs, ++it) {
      const JobP J = Jn;
      const int64_t rc = rcn;
      int64_t* cc = colC + (it & 1) * TILE_W;
      if (w + npairs < L.nwork) setup(w + npairs, colC + ((it + 1) & 1) * TILE_W, Jn, rcn);
      if (!live) {
        named_bar_sync(1, kEpiThreadsW);
        continue;
      }
      const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
      float hi[128];
      for (int j = 0; j < nchunks; ++j, ++gc) {
        const uint32_t buf = gc & 1;
        if (!warp_wait(&accf[buf], (gc >> 1) & 1, abort)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + buf * TILE_W + hh * TILE;
        if (j == 0) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t r[16];
            tmem_ld16(tl + c * 16, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) hi[c * 16 + i] = __uint_as_float(r[i]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            uint32_t r[16];
            tmem_ld16(tl + c * 16, r);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) hi[c * 16 + i] = __fadd_rn(hi[c * 16 + i],
                                                                    __uint_as_float(r[i]));
          }
        }
        tc_fence_before();
        if (lead) {
          mbar_arrive(&acce[buf]);
        } else {  // one arrival of 32 per warp on the first CTA's barrier
          __syncwarp();
          if (lane == 0) mbar_arrive_remote(&acce[buf], 0, 32);
        }
      }
      const int tm = 2 * J.tmp + (int)rank, tn = 2 * J.tnp + hh;
      if (live && tm < P.tiles_m && tn < P.tiles_n) {
        if (J.tail >= 0) {  // a tail tile's K range: partial sums of this quarter
          const int64_t ntail = (((int64_t)(P.tiles_m + 1) / 2) * ((P.tiles_n + 1) / 2)) - P.nfull;
          float2* pp = P.part + (((size_t)J.split * ntail + J.tail) * 4 + rank * 2 + hh) *
                                    (size_t)(TILE * TILE) + row;
#pragma unroll
          for (int i = 0; i < 128; ++i) pp[(size_t)i * TILE] = make_float2(hi[i], 0.0f);
        } else if (P.ksplit > 1) {
          float2* pp = P.part + ((size_t)J.split * P.tiles_m * P.tiles_n +
                                 tile128_index(P, tm, tn)) * (size_t)(TILE * TILE) + row;
#pragma unroll
          for (int i = 0; i < 128; ++i) pp[(size_t)i * TILE] = make_float2(hi[i], 0.0f);
        } else if (rc >= 0) {
          const int64_t* ch = cc + hh * TILE;
          if (L.out_type == 0) store_row<float, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
          else if (L.out_type == 1)
            store_row<__nv_bfloat16, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
          else store_row<__half, 128>(L.C, rc, ch, hi, L.alpha, L.beta);
        }
      }
      named_bar_sync(1, kEpiThreadsW);  // this tile's columns read; the next tile's written
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the pair's MMAs and both epilogues are done with both CTAs' memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc2(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// CTA pairs for the split forms with compensated sums (tile configuration 5
// with BF16x6): the arithmetic of the 128 x 128 kernel -- the main product in
// a double-buffered accumulator emptied every chunk into a compensated sum,
// the correction products in an accumulator of their own -- on 256 x 128
// tiles shared by two SMs (tcgen05.mma.cta_group::2, M = 256, N = 128).  Each
// CTA holds its own 128 rows of A and a 64-row half of the tile's B (the rows
// of its rank, taken by TMA at an x offset of 1 KB from the packed 128-row
// blocks): 25 % fewer operand bytes per SM per multiply-add, while each CTA's
// tensor memory keeps the 128 x 128 kernel's layout for its own rows.  The
// loads of both CTAs complete on the first CTA's full barrier; the MMA
// thread's commits arrive on both CTAs' barriers; both epilogues arrive on the
// first CTA's acce barrier.
// ---------------------------------------------------------------------------
template <int NT>
struct CfgP6 {
  static constexpr int BPS = 2;                                // 32-K blocks per stage
  static constexpr uint32_t OPA = NT * TERM;                   // own A block (128 rows)
  static constexpr uint32_t HTERM = TERM / 2;                  // one term of a 64-row B half
  static constexpr uint32_t OPB = NT * HTERM;                  // own B half block
  static constexpr uint32_t STAGE = BPS * (OPA + OPB);         // 72 KB for BF16x6
  static constexpr uint32_t RING = 216 * 1024;
  static constexpr int S = (int)(RING / STAGE);                // 3 stages
  static constexpr uint32_t OFF_COLC = S * STAGE;              // int64 colC[2][128]
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * TILE * 8;
  static constexpr uint32_t NBAR = 2 * S + 4 + 1;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;
};

// Work entry w: split-major over the 256 x 128 pair tiles (A tiles 2 tmp and
// 2 tmp + 1, B tile tn).
struct JobP6 {
  int tmp, tn, split, k0, k1;
};

__device__ __forceinline__ JobP6 jobp6_of(const PkItem& P, int64_t w) {
  JobP6 j;
  const int mp = (P.tiles_m + 1) / 2;
  const int64_t ntiles = (int64_t)mp * P.tiles_n;
  j.split = (int)(w / ntiles);
  const int64_t t = w % ntiles;
  if (P.raster) {
    j.tn = (int)(t % P.tiles_n);
    j.tmp = (int)(t / P.tiles_n);
  } else {
    j.tmp = (int)(t % mp);
    j.tn = (int)(t / mp);
  }
  j.k0 = (int)((int64_t)j.split * P.nkb / P.ksplit);
  j.k1 = (int)((int64_t)(j.split + 1) * P.nkb / P.ksplit);
  return j;
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_pkp6(const __grid_constant__ PkLaunch L) {
  using G = CfgP6<NT>;
  constexpr int S = G::S;
  extern __shared__ uint8_t pkp6_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(pkp6_raw) + 1023) & ~(uintptr_t)1023);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + G::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 2;
  uint64_t* done = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + G::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + G::OFF_MISC + 4);
  const PkItem& P = L.single;
  const int ckb = max(P.chunk_kb, 1);
  const uint32_t rank = cluster_ctarank();
  const bool lead = rank == 0;
  const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 2 * kEpiThreads);  // both CTAs' epilogue threads
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync();  // both CTAs' barriers exist before any remote arrival
  if (warp == 1) tmem_alloc2(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      // this CTA's 128 rows of A and the 64 rows of B of its rank
      uint32_t g = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < L.nwork; w += npairs) {
        const JobP6 J = jobp6_of(P, w);
        const int tm0 = 2 * J.tmp, tm = tm0 + (int)rank;
        const bool va = tm < P.tiles_m;   // else: rows the pair discards
        const uint32_t pair_block = (tm0 < P.tiles_m ? G::OPA : 0u) +
                                    (tm0 + 1 < P.tiles_m ? G::OPA : 0u) + 2 * G::OPB;
        for (int kb = J.k0; kb < J.k1; kb += G::BPS, ++g) {
          const int s = (int)(g % S);
          if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          const int nb = min(G::BPS, J.k1 - kb);
          const uint32_t dst = sbase + (uint32_t)s * G::STAGE;
          if (lead) mbar_arrive_expect_tx(&full[s], (uint32_t)nb * pair_block);
          const uint32_t mb = mapa_shared(smem_u32(&full[s]), 0);
          for (int bi = 0; bi < nb; ++bi) {
            if (va)
              tma_load_2d_pair(dst + bi * G::OPA, &L.tma_a, 0,
                               (int32_t)(((int64_t)tm * P.nkb + kb + bi) * (G::OPA / 2048)), mb);
            // the NT terms of this CTA's 64-row half of B: 4 NT rows of 2 KB from
            // x = 1 KB * rank, landing term after term (HTERM apart)
            const int64_t brow = ((int64_t)J.tn * P.nkb + kb + bi) * (NT * TERM / 2048);
            tma_load_2d_pair(dst + G::BPS * G::OPA + bi * G::OPB, &L.tma_b, (int32_t)(rank * 128),
                             (int32_t)brow, mb);
          }
        }
      }
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&empty[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // ------------------------------------------- MMA issue (first CTA)
      const uint32_t idesc = L.idesc;
      constexpr uint32_t LBOA = (TILE / 8) * 128;        // 128-row A blocks
      constexpr uint32_t LBOB = (TILE / 2 / 8) * 128;    // 64-row B halves
      uint32_t g = 0, gc = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < L.nwork; w += npairs) {
        const JobP6 J = jobp6_of(P, w);
        const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
        // the correction accumulator, both main buffers and the high words are
        // free once both CTAs drained the previous tile's last chunk
        if (gc >= 1 && !mbar_wait(&acce[(gc - 1) & 1], ((gc - 1) >> 1) & 1, abort, kTimeoutNs)) {
          ok = false;
          break;
        }
        int kb = J.k0;
        for (int j = 0; ok && j < nchunks; ++j, ++gc) {
          const uint32_t buf = gc & 1;
          if (gc >= 2 && !mbar_wait(&acce[buf], ((gc >> 1) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dmain = tmem + buf * TILE;
          const int kend = min(J.k1, J.k0 + (j + 1) * ckb), kstart = kb;
          for (; kb < kend; kb += G::BPS, ++g) {
            const int s = (int)(g % S);
            if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const int nb = min(G::BPS, kend - kb);
            const uint32_t st = sbase + (uint32_t)s * G::STAGE;
            // descriptors of the stage's first blocks; every operand of the
            // stage is a compile-time offset from them (the address field is
            // the byte address / 16, and shared memory stays below 256 KB)
            const uint64_t da0 = smem_desc(st, LBOA, 128);
            const uint64_t db0 = smem_desc(st + G::BPS * G::OPA, LBOB, 128);
#pragma unroll
            for (int bi = 0; bi < G::BPS; ++bi) {
              if (bi >= nb) break;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const bool first = bi == 0 && kk == 0;
                mma_bf16_pair(dmain, da0 + ((bi * G::OPA + kk * 2 * LBOA) >> 4),
                              db0 + ((bi * G::OPB + kk * 2 * LBOB) >> 4), idesc,
                              (kb > kstart || !first) ? 1u : 0u);
#pragma unroll
                for (int pi = 1; pi < nprod(NT); ++pi)
                  mma_bf16_pair(tmem + COL_CORR,
                                da0 + ((bi * G::OPA + prod_a(pi) * TERM + kk * 2 * LBOA) >> 4),
                                db0 + ((bi * G::OPB + prod_b(pi) * G::HTERM + kk * 2 * LBOB) >> 4),
                                idesc, (kb > J.k0 || !first || pi > 1) ? 1u : 0u);
              }
            }
            mma_commit_pair(&empty[s], 3);  // both CTAs may refill this stage
          }
          if (!ok) break;
          mma_commit_pair(&accf[buf], 3);   // both CTAs' epilogues may drain it
        }
      }
      mma_commit_pair(done, 1);
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else {
    // ------------------------------------------------------------- epilogue
    // each CTA drains its own 128 rows: two warps per lane quadrant, 64
    // columns each, as in the 128 x 128 kernel
    const int ew = warp - 2;
    const int q = warp & 3;
    const int h = ew >> 2;
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)h * 64;
    uint32_t gc = 0;
    int64_t it = 0;
    bool live = true;
    auto release = [&](uint32_t buf) {  // this CTA's epilogue is done with buffer buf
      if (lead) {
        mbar_arrive(&acce[buf]);
      } else {
        __syncwarp();
        if (lane == 0) mbar_arrive_remote(&acce[buf], 0, 32);
      }
    };
    auto setup = [&](int64_t w, int64_t* cc, JobP6& J, int64_t& rc) {
      J = jobp6_of(P, w);
      if (etid < TILE) {
        const int64_t n = (int64_t)J.tn * TILE + etid;
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      const int64_t m = (int64_t)(2 * J.tmp + (int)rank) * TILE + row;
      rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
    };
    JobP6 Jn;
    int64_t rcn = -1;
    if (pair < L.nwork) setup(pair, colC, Jn, rcn);
    named_bar_sync(1, kEpiThreads);
    for (int64_t w = pair; w < L.nwork; w += npairs, ++it) {
      const JobP6 J = Jn;
      const int64_t rc = rcn;
      int64_t* cc = colC + (it & 1) * TILE;
      if (w + npairs < L.nwork) setup(w + npairs, colC + ((it + 1) & 1) * TILE, Jn, rcn);
      if (!live) {
        named_bar_sync(1, kEpiThreads);
        continue;
      }
      const int nchunks = (J.k1 - J.k0 + ckb - 1) / ckb;
      const int tm = 2 * J.tmp + (int)rank;
      const bool partial = P.ksplit > 1;
      float2* pp = (partial && tm < P.tiles_m)
                       ? P.part + ((size_t)J.split * P.tiles_m * P.tiles_n +
                                   tile128_index(P, tm, J.tn)) * (size_t)(TILE * TILE) +
                             (size_t)h * 64 * TILE + row
                       : nullptr;
      float lo[64], hi[64];  // the compensated sum of the drained chunks
#pragma unroll
      for (int i = 0; i < 64; ++i) lo[i] = hi[i] = 0.0f;
      for (int j = 0; j < nchunks; ++j, ++gc) {
        const uint32_t buf = gc & 1;
        if (!warp_wait(&accf[buf], (gc >> 1) & 1, abort)) {
          live = false;
          break;
        }
        tc_fence_after();
        const uint32_t tmain = tl + buf * TILE;
        if (j + 1 < nchunks) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t mv[16];
            tmem_ld16(tmain + c * 16, mv);
            tmem_wait_ld();
            if (c == 3) {
              tc_fence_before();
              release(buf);  // the chunk is in registers
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              float e;
              hi[c * 16 + i] = two_sum(hi[c * 16 + i], __uint_as_float(mv[i]), e);
              lo[c * 16 + i] = __fadd_rn(lo[c * 16 + i], e);
            }
          }
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) {  // eight columns at a time: few registers live
            uint32_t mv[8], cv[8];
            tmem_ld8(tmain + c * 8, mv);
            if (NT > 1) tmem_ld8(tl + COL_CORR + c * 8, cv);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float e;
              const float s = two_sum(hi[c * 8 + i], __uint_as_float(mv[i]), e);
              float r = __fadd_rn(lo[c * 8 + i], e);
              if (NT > 1) r = __fadd_rn(r, __uint_as_float(cv[i]));
              if (pp) pp[(size_t)(c * 8 + i) * TILE] = make_float2(s, r);
              else lo[c * 8 + i] = __fadd_rn(s, r);
            }
          }
          tc_fence_before();
          release(buf);  // main, correction and high word are free
          if (!partial && rc >= 0) {
            const int64_t* ch = cc + h * 64;
            if (L.out_type == 0) store_row<float, 64>(L.C, rc, ch, lo, L.alpha, L.beta);
            else if (L.out_type == 1)
              store_row<__nv_bfloat16, 64>(L.C, rc, ch, lo, L.alpha, L.beta);
            else store_row<__half, 64>(L.C, rc, ch, lo, L.alpha, L.beta);
          }
        }
      }
      named_bar_sync(1, kEpiThreads);  // this tile's columns read; the next tile's written
    }
  }

  __syncwarp();
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the pair's MMAs and both epilogues are done with both CTAs' memory
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc2(tmem, kTmemCols);
  }
}

// Split-K: C = alpha * (sum of the K ranges' partial sums, in order) + beta * C.
__global__ void __launch_bounds__(256) k_pk_reduce(const __grid_constant__ PkLaunch L) {
  const PkItem& P = L.single;
  const int64_t ntiles = (int64_t)P.tiles_m * P.tiles_n;
  const int64_t total = ntiles * TILE * TILE;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = e / (TILE * TILE);
    const int col = (int)((e / TILE) % TILE), row = (int)(e % TILE);
    int tm, tn;
    if (P.raster) {
      tn = (int)(tile % P.tiles_n);
      tm = (int)(tile / P.tiles_n);
    } else {
      tm = (int)(tile % P.tiles_m);
      tn = (int)(tile / P.tiles_m);
    }
    const int64_t m = (int64_t)tm * TILE + row, n = (int64_t)tn * TILE + col;
    if (m >= P.M || n >= P.N) continue;
    double t = 0.0;
    for (int sp = 0; sp < P.ksplit; ++sp) {
      const float2 v = P.part[(size_t)sp * total + e];
      t += (double)v.x + (double)v.y;
    }
    store_out(L.C, goff(P.gm, 2, (uint32_t)m) + goff(P.gn, 2, (uint32_t)n), L.out_type,
              (float)(L.alpha * t), L.beta);
  }
}

// Tail split of CTA pairs: C of the tail tiles = alpha * (sum of their K
// ranges' partial sums, in order) + beta * C.
__global__ void __launch_bounds__(256) k_pkp_reduce_tail(const __grid_constant__ PkLaunch L) {
  const PkItem& P = L.single;
  const int mp = (P.tiles_m + 1) / 2, np = (P.tiles_n + 1) / 2;
  const int64_t ntail = (int64_t)mp * np - P.nfull;
  const int64_t total = ntail * 4 * TILE * TILE;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sub = e / (TILE * TILE);
    const int64_t tail = sub / 4;
    const int quarter = (int)(sub % 4);
    const int col = (int)((e / TILE) % TILE), row = (int)(e % TILE);
    const int64_t t = P.nfull + tail;
    int tmp, tnp;
    if (P.raster) {
      tnp = (int)(t % np);
      tmp = (int)(t / np);
    } else {
      tmp = (int)(t % mp);
      tnp = (int)(t / mp);
    }
    const int tm = 2 * tmp + (quarter >> 1), tn = 2 * tnp + (quarter & 1);
    const int64_t m = (int64_t)tm * TILE + row, n = (int64_t)tn * TILE + col;
    if (tm >= P.tiles_m || tn >= P.tiles_n || m >= P.M || n >= P.N) continue;
    double s = 0.0;
    for (int sp = 0; sp < P.tsplit; ++sp) {
      const float2 v = P.part[(size_t)sp * total + e];
      s += (double)v.x + (double)v.y;
    }
    store_out(L.C, goff(P.gm, 2, (uint32_t)m) + goff(P.gn, 2, (uint32_t)n), L.out_type,
              (float)(L.alpha * s), L.beta);
  }
}

// Batched split-K: a block adds the K ranges of 1/kRedParts of one
// (item, tile), in order, applies the item's alpha and beta and stores
// through its groups.
constexpr int kRedParts = 16;
__global__ void __launch_bounds__(256) k_pk_reduce_batch(const PkItem* __restrict__ items,
                                                         const int32_t* __restrict__ red,
                                                         int64_t n_red, void* const* Cp,
                                                         const double* alpha_p,
                                                         const double* beta_p) {
  for (int64_t rp = blockIdx.x; rp < n_red * kRedParts; rp += gridDim.x) {
    const int64_t r = rp / kRedParts;
    const int part = (int)(rp % kRedParts);
    const int32_t item = red[2 * r];
    const int64_t tile = red[2 * r + 1];
    const PkItem& P = items[item];
    const int64_t ntiles = (int64_t)P.tiles_m * P.tiles_n;
    const int64_t total = ntiles * TILE * TILE;
    const int tm = (int)(tile % P.tiles_m), tn = (int)(tile / P.tiles_m);
    const float alpha = (float)alpha_p[item], beta = (float)beta_p[item];
    float* C = static_cast<float*>(Cp[item]);
    constexpr int kPart = TILE * TILE / kRedParts;
    for (int e = part * kPart + threadIdx.x; e < (part + 1) * kPart; e += blockDim.x) {
      const int col = e / TILE, row = e % TILE;
      const int64_t m = (int64_t)tm * TILE + row, n = (int64_t)tn * TILE + col;
      if (m >= P.M || n >= P.N) continue;
      double t = 0.0;
      for (int sp = 0; sp < P.ksplit; ++sp) {
        const float2 v = P.part[(size_t)sp * total + (size_t)tile * TILE * TILE + e];
        t += (double)v.x + (double)v.y;
      }
      float* dst = C + goff(P.gm, 2, (uint32_t)m) + goff(P.gn, 2, (uint32_t)n);
      float x = (float)(alpha * t);
      if (beta != 0.0f) x = fmaf(beta, *dst, x);
      *dst = x;
    }
  }
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
int set_smem() {
  static int bytes = 0;
  if (bytes == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
      return -1;
    if (optin < (int)Cfg<NT>::BYTES) return -2;
    if (cudaFuncSetAttribute(k_bf16_pack_batch<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPackSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_pk<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<NT>::BYTES) != cudaSuccess)
      return -1;
    bytes = (int)Cfg<NT>::BYTES;
  }
  return bytes;
}

// Shared memory of one pack kernel instantiation (set once).
template <int NT, typename In, bool F16T>
bool set_pack_smem() {
  static bool done = false;
  if (!done)
    done = cudaFuncSetAttribute(k_bf16_pack<NT, In, F16T>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kPackSmem) == cudaSuccess;
  return done;
}

// One GEMM: operands of type In packed into NT BF16 terms (F16T: one FP16
// term), C stored as out_type (0 FP32, 1 BF16, 2 FP16).
template <int NT, typename In, bool F16T>
tc_status launch(const GemmArgs& a, const PkLayout& L, void* ws, cudaStream_t s, int out_type) {
  const int sm = set_smem<NT>();
  if (sm == -2) return TC_ERR_UNSUPPORTED;
  if (!set_pack_smem<NT, In, F16T>()) return TC_ERR_CUDA;
  const int sms = num_sms();
  if (sm < 0 || sms <= 0) return TC_ERR_CUDA;
  uint8_t* w = static_cast<uint8_t*>(ws);
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.gr[0] = a.gm;
  pa.gr[1] = a.gn;
  pa.gk = a.gk;
  pa.in[0] = a.A;
  pa.in[1] = a.B;
  pa.q[0] = w + L.off_qa;
  pa.q[1] = w + L.off_qb;
  pa.rows[0] = a.M;
  pa.rows[1] = a.N;
  pa.K = a.K;
  pa.tiles[0] = (int32_t)L.tiles_m;
  pa.tiles[1] = (int32_t)L.tiles_n;
  pa.nkb = (int32_t)L.nkb;
  pa.npk = (int32_t)((L.nkb + PK / BK - 1) / (PK / BK));
  pa.nblocks0 = L.tiles_m * pa.npk;
  pa.rows_fast[0] = a.a_contig == CONTIG_MN;
  pa.rows_fast[1] = a.b_contig == CONTIG_MN;
  const int64_t nblocks = (L.tiles_m + L.tiles_n) * pa.npk;
  if (nblocks > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  k_bf16_pack<NT, In, F16T><<<(unsigned)nblocks, kPackThreads, kPackSmem, s>>>(pa);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;

  PkLaunch g;
  std::memset(&g, 0, sizeof(g));
  PkItem& it = g.single;
  it.gm = a.gm;
  it.gn = a.gn;
  it.qa = pa.q[0];
  it.qb = pa.q[1];
  it.M = a.M;
  it.N = a.N;
  it.tiles_m = (int32_t)L.tiles_m;
  it.tiles_n = (int32_t)L.tiles_n;
  it.nkb = (int32_t)L.nkb;
  it.chunk_kb = a.chunk_kb;
  if (max(a.chunk_kb, 1) % Cfg<NT>::BPS != 0) return TC_ERR_UNSUPPORTED;  // a stage per chunk part
  it.raster = a.raster;
  it.ksplit = pk_ksplit(a);
  it.part = it.ksplit > 1 ? reinterpret_cast<float2*>(w + L.bytes) : nullptr;
  g.C = a.C;
  g.alpha = (float)a.alpha;
  g.beta = (float)a.beta;
  g.idesc = F16T ? idesc_f16(TILE, TILE) : idesc_bf16(TILE, TILE);
  g.out_type = out_type;
  g.nwork = L.tiles_m * L.tiles_n * it.ksplit;
  const int grid = (int)std::min<int64_t>(g.nwork, sms);
  k_gemm_pk<NT><<<grid, kThreads, sm, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (it.ksplit > 1) {
    const int64_t total = L.tiles_m * L.tiles_n * TILE * TILE;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
    k_pk_reduce<<<rgrid, 256, 0, s>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

// One GEMM on wide tiles (tile configuration 4), same arguments as launch.
template <int NT, typename In, bool F16T>
tc_status launch_w(const GemmArgs& a, const PkLayout& L, void* ws, cudaStream_t s, int out_type) {
  static int sm = 0;
  if (sm == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
      return TC_ERR_CUDA;
    if (optin < (int)CfgW<NT>::BYTES) return TC_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k_gemm_pkw<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CfgW<NT>::BYTES) != cudaSuccess)
      return TC_ERR_CUDA;
    sm = (int)CfgW<NT>::BYTES;
  }
  if (!set_pack_smem<NT, In, F16T>()) return TC_ERR_CUDA;
  const int sms = num_sms();
  if (sms <= 0) return TC_ERR_CUDA;
  uint8_t* w = static_cast<uint8_t*>(ws);
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.gr[0] = a.gm;
  pa.gr[1] = a.gn;
  pa.gk = a.gk;
  pa.in[0] = a.A;
  pa.in[1] = a.B;
  pa.q[0] = w + L.off_qa;
  pa.q[1] = w + L.off_qb;
  pa.rows[0] = a.M;
  pa.rows[1] = a.N;
  pa.K = a.K;
  pa.tiles[0] = (int32_t)L.tiles_m;
  pa.tiles[1] = (int32_t)L.tiles_n;
  pa.nkb = (int32_t)L.nkb;
  pa.npk = (int32_t)((L.nkb + PK / BK - 1) / (PK / BK));
  pa.nblocks0 = L.tiles_m * pa.npk;
  pa.rows_fast[0] = a.a_contig == CONTIG_MN;
  pa.rows_fast[1] = a.b_contig == CONTIG_MN;
  const int64_t nblocks = (L.tiles_m + L.tiles_n) * pa.npk;
  if (nblocks > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  k_bf16_pack<NT, In, F16T><<<(unsigned)nblocks, kPackThreads, kPackSmem, s>>>(pa);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;

  PkLaunch g;
  std::memset(&g, 0, sizeof(g));
  PkItem& it = g.single;
  it.gm = a.gm;
  it.gn = a.gn;
  it.qa = pa.q[0];
  it.qb = pa.q[1];
  it.M = a.M;
  it.N = a.N;
  it.tiles_m = (int32_t)L.tiles_m;
  it.tiles_n = (int32_t)L.tiles_n;
  it.nkb = (int32_t)L.nkb;
  it.chunk_kb = a.chunk_kb;
  it.raster = a.raster;
  it.ksplit = pk_ksplit_w(a);
  it.part = it.ksplit > 1 ? reinterpret_cast<float2*>(w + L.bytes) : nullptr;
  g.C = a.C;
  g.alpha = (float)a.alpha;
  g.beta = (float)a.beta;
  g.idesc = F16T ? idesc_f16(TILE, TILE) : idesc_bf16(TILE, TILE);
  g.out_type = out_type;
  g.nwork = L.tiles_m * ((L.tiles_n + 1) / 2) * it.ksplit;
  const int grid = (int)std::min<int64_t>(g.nwork, sms);
  k_gemm_pkw<NT><<<grid, kThreadsW, sm, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (it.ksplit > 1) {
    const int64_t total = L.tiles_m * L.tiles_n * TILE * TILE;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
    k_pk_reduce<<<rgrid, 256, 0, s>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// links no driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The packed blocks of one operand as a 2-D tensor of 8-byte elements in rows
// of 2 KB (256 elements); a box is box_x elements (box_x x 8 bytes) of
// box_bytes / 2048 rows.  Loads start at x = 0, or at x = 128 for the second
// half of a row (1 KB: a 16-byte multiple, as tiled TMA copies need).
bool rows_map(CUtensorMap* m, const void* base, size_t bytes, uint32_t box_bytes,
              uint32_t box_x = 256) {
  EncodeTiledFn f = encode_tiled();
  if (!f || bytes == 0 || bytes % 2048 || box_bytes % 2048 || box_bytes / 2048 > 256 ||
      box_x == 0 || box_x > 256 || (reinterpret_cast<uintptr_t>(base) & 15))
    return false;
  cuuint64_t dims[2] = {256, (cuuint64_t)(bytes / 2048)};
  cuuint64_t strides[1] = {2048};
  cuuint32_t box[2] = {box_x, box_bytes / 2048};
  cuuint32_t es[2] = {1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One GEMM on CTA pairs (tile configuration 5), same arguments as launch.
// The grid is two CTAs per pair, as many pairs as fit at once (persistent).
template <int NT, typename In, bool F16T>
tc_status launch_p(const GemmArgs& a, const PkLayout& L, void* ws, cudaStream_t s, int out_type) {
  if (max(a.chunk_kb, 1) % CfgP<NT>::BPS != 0) return TC_ERR_UNSUPPORTED;  // chunks end on stages
  static int max_pairs = 0;
  if (max_pairs == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
      return TC_ERR_CUDA;
    if (optin < (int)CfgP<NT>::BYTES) return TC_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k_gemm_pkp<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CfgP<NT>::BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_pkp<NT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0) !=
            cudaSuccess)
      return TC_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * 152, 1, 1);
    cfg.blockDim = dim3(kThreadsW, 1, 1);
    cfg.dynamicSmemBytes = CfgP<NT>::BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_gemm_pkp<NT>, &cfg) != cudaSuccess || n <= 0)
      return TC_ERR_UNSUPPORTED;
    max_pairs = n;
  }
  if (!set_pack_smem<NT, In, F16T>()) return TC_ERR_CUDA;
  uint8_t* w = static_cast<uint8_t*>(ws);
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.gr[0] = a.gm;
  pa.gr[1] = a.gn;
  pa.gk = a.gk;
  pa.in[0] = a.A;
  pa.in[1] = a.B;
  pa.q[0] = w + L.off_qa;
  pa.q[1] = w + L.off_qb;
  pa.rows[0] = a.M;
  pa.rows[1] = a.N;
  pa.K = a.K;
  pa.tiles[0] = (int32_t)L.tiles_m;
  pa.tiles[1] = (int32_t)L.tiles_n;
  pa.nkb = (int32_t)L.nkb;
  pa.npk = (int32_t)((L.nkb + PK / BK - 1) / (PK / BK));
  pa.nblocks0 = L.tiles_m * pa.npk;
  pa.rows_fast[0] = a.a_contig == CONTIG_MN;
  pa.rows_fast[1] = a.b_contig == CONTIG_MN;
  const int64_t nblocks = (L.tiles_m + L.tiles_n) * pa.npk;
  if (nblocks > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  k_bf16_pack<NT, In, F16T><<<(unsigned)nblocks, kPackThreads, kPackSmem, s>>>(pa);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;

  PkLaunch g;
  std::memset(&g, 0, sizeof(g));
  PkItem& it = g.single;
  it.gm = a.gm;
  it.gn = a.gn;
  it.qa = pa.q[0];
  it.qb = pa.q[1];
  it.M = a.M;
  it.N = a.N;
  it.tiles_m = (int32_t)L.tiles_m;
  it.tiles_n = (int32_t)L.tiles_n;
  it.nkb = (int32_t)L.nkb;
  it.chunk_kb = a.chunk_kb;
  it.raster = a.raster;
  it.ksplit = pk_ksplit_p(a);
  int64_t nfull = 0;
  it.tsplit = pk_tail_split_p(a, &nfull);
  it.nfull = nfull;
  it.part = (it.ksplit > 1 || it.tsplit > 1) ? reinterpret_cast<float2*>(w + L.bytes) : nullptr;
  g.C = a.C;
  g.alpha = (float)a.alpha;
  g.beta = (float)a.beta;
  g.idesc = F16T ? idesc_f16(2 * TILE, TILE_W) : idesc_bf16(2 * TILE, TILE_W);
  g.out_type = out_type;
  const int64_t ptiles = ((L.tiles_m + 1) / 2) * ((L.tiles_n + 1) / 2);
  g.nwork = it.tsplit > 1 ? nfull + (ptiles - nfull) * it.tsplit : ptiles * it.ksplit;
  if (!rows_map(&g.tma_a, it.qa, (size_t)L.tiles_m * L.nkb * CfgP<NT>::OPA, CfgP<NT>::OPA) ||
      !rows_map(&g.tma_b, it.qb, (size_t)L.tiles_n * L.nkb * CfgP<NT>::OPB, CfgP<NT>::OPB))
    return TC_ERR_CUDA;
  const int pairs = (int)std::min<int64_t>(g.nwork, max_pairs);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * pairs, 1, 1);
  cfg.blockDim = dim3(kThreadsW, 1, 1);
  cfg.dynamicSmemBytes = CfgP<NT>::BYTES;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_gemm_pkp<NT>, g) != cudaSuccess) return TC_ERR_CUDA;
  if (it.tsplit > 1) {
    const int64_t total = (ptiles - nfull) * 4 * TILE * TILE;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)152 * 8);
    k_pkp_reduce_tail<<<rgrid, 256, 0, s>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  if (it.ksplit > 1) {
    const int64_t total = L.tiles_m * L.tiles_n * TILE * TILE;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)152 * 8);
    k_pk_reduce<<<rgrid, 256, 0, s>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

// BF16x6 on CTA pairs (tile configuration 5): FP32 storage.
template <int NT>
tc_status launch_p6(const GemmArgs& a, const PkLayout& L, void* ws, cudaStream_t s) {
  static int max_pairs = 0;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  if (max_pairs == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
      return TC_ERR_CUDA;
    if (optin < (int)CfgP6<NT>::BYTES) return TC_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k_gemm_pkp6<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CfgP6<NT>::BYTES) != cudaSuccess)
      return TC_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 152, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = CfgP6<NT>::BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_gemm_pkp6<NT>, &cfg) != cudaSuccess || n <= 0)
      return TC_ERR_UNSUPPORTED;
    max_pairs = n;
  }
  if (!set_pack_smem<NT, float, false>()) return TC_ERR_CUDA;
  uint8_t* w = static_cast<uint8_t*>(ws);
  PackArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.gr[0] = a.gm;
  pa.gr[1] = a.gn;
  pa.gk = a.gk;
  pa.in[0] = a.A;
  pa.in[1] = a.B;
  pa.q[0] = w + L.off_qa;
  pa.q[1] = w + L.off_qb;
  pa.rows[0] = a.M;
  pa.rows[1] = a.N;
  pa.K = a.K;
  pa.tiles[0] = (int32_t)L.tiles_m;
  pa.tiles[1] = (int32_t)L.tiles_n;
  pa.nkb = (int32_t)L.nkb;
  pa.npk = (int32_t)((L.nkb + PK / BK - 1) / (PK / BK));
  pa.nblocks0 = L.tiles_m * pa.npk;
  pa.rows_fast[0] = a.a_contig == CONTIG_MN;
  pa.rows_fast[1] = a.b_contig == CONTIG_MN;
  const int64_t nblocks = (L.tiles_m + L.tiles_n) * pa.npk;
  if (nblocks > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  k_bf16_pack<NT, float, false><<<(unsigned)nblocks, kPackThreads, kPackSmem, s>>>(pa);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;

  PkLaunch g;
  std::memset(&g, 0, sizeof(g));
  PkItem& it = g.single;
  it.gm = a.gm;
  it.gn = a.gn;
  it.qa = pa.q[0];
  it.qb = pa.q[1];
  it.M = a.M;
  it.N = a.N;
  it.tiles_m = (int32_t)L.tiles_m;
  it.tiles_n = (int32_t)L.tiles_n;
  it.nkb = (int32_t)L.nkb;
  it.chunk_kb = a.chunk_kb;
  if (max(a.chunk_kb, 1) % CfgP6<NT>::BPS != 0) return TC_ERR_UNSUPPORTED;
  it.raster = a.raster;
  it.ksplit = pk_ksplit_p6(a);
  it.part = it.ksplit > 1 ? reinterpret_cast<float2*>(w + L.bytes) : nullptr;
  g.C = a.C;
  g.alpha = (float)a.alpha;
  g.beta = (float)a.beta;
  g.idesc = idesc_bf16(2 * TILE, TILE);
  g.out_type = 0;
  g.nwork = ((L.tiles_m + 1) / 2) * L.tiles_n * it.ksplit;
  if (!rows_map(&g.tma_a, it.qa, (size_t)L.tiles_m * L.nkb * CfgP6<NT>::OPA, CfgP6<NT>::OPA) ||
      !rows_map(&g.tma_b, it.qb, (size_t)L.tiles_n * L.nkb * NT * TERM, NT * 4 * 2048, 128))
    return TC_ERR_CUDA;
  const int pairs = (int)std::min<int64_t>(g.nwork, max_pairs);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = CfgP6<NT>::BYTES;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_gemm_pkp6<NT>, g) != cudaSuccess) return TC_ERR_CUDA;
  if (it.ksplit > 1) {
    const int64_t total = L.tiles_m * L.tiles_n * TILE * TILE;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)152 * 8);
    k_pk_reduce<<<rgrid, 256, 0, s>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

template <int NT>
tc_status launch_batch(const PkBatch& b, const void* const* A, const void* const* B,
                       void* const* C, const double* alpha, const double* beta, cudaStream_t s) {
  if (b.n_work == 0) return TC_OK;
  const int sm = set_smem<NT>();
  if (sm == -2) return TC_ERR_UNSUPPORTED;
  const int sms = num_sms();
  if (sm < 0 || sms <= 0) return TC_ERR_CUDA;
  if (b.n_pack > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  if (b.n_pack > 0) {
    k_bf16_pack_batch<NT><<<(unsigned)b.n_pack, kPackThreads, kPackSmem, s>>>(
        b.items, b.pk, reinterpret_cast<const PackWork*>(b.pack_work), A, B);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  PkLaunch g;
  std::memset(&g, 0, sizeof(g));
  g.items = b.pk;
  g.idesc = idesc_bf16(TILE, TILE);
  g.out_type = 0;
  g.work = b.work;
  g.Cp = C;
  g.alpha_p = alpha;
  g.beta_p = beta;
  g.nwork = b.n_work;
  const int grid = (int)std::min<int64_t>(g.nwork, sms);
  k_gemm_pk<NT><<<grid, kThreads, sm, s>>>(g);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  if (b.n_red > 0) {
    const int rgrid = (int)std::min<int64_t>(b.n_red * kRedParts, (int64_t)sms * 8);
    k_pk_reduce_batch<<<rgrid, 256, 0, s>>>(b.pk, b.red, b.n_red, C, alpha, beta);
    if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;
  }
  return TC_OK;
}

}  // namespace pk

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int terms_of(int math) {
  return (math == TC_MATH_BF16 || math == TC_MATH_FP16) ? 1
         : math == TC_MATH_BF16X3 ? 2 : math == TC_MATH_BF16X6 ? 3 : 0;
}

// Split-K: tiles fewer than the SMs share out their K blocks, so that about
// two work entries per SM exist, each of at least 512 K (16 blocks).
int pk_ksplit(const GemmArgs& a) {
  const int64_t tiles = ((a.M + pk::TILE - 1) / pk::TILE) * ((a.N + pk::TILE - 1) / pk::TILE);
  const int64_t nkb = (a.K + pk::BK - 1) / pk::BK;
  if (tiles <= 0 || tiles >= 152) return 1;
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, nkb / 16, 64}));
}

// Split-K of the wide tiles: the same rule over 128 x 256 tiles.
int pk_ksplit_w(const GemmArgs& a) {
  const int64_t tiles =
      ((a.M + pk::TILE - 1) / pk::TILE) * (((a.N + pk::TILE - 1) / pk::TILE + 1) / 2);
  const int64_t nkb = (a.K + pk::BK - 1) / pk::BK;
  if (tiles <= 0 || tiles >= 152) return 1;
  const int64_t want = (2 * 152 + tiles - 1) / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, nkb / 16, 64}));
}

// Split-K of the CTA pairs: pair tiles fewer than the pairs that fit share
// out their K blocks, at most one work entry per pair (a second, partial
// round of entries would double the time), each >= 512 K.
int pk_ksplit_p(const GemmArgs& a) {
  const int64_t tiles = (((a.M + pk::TILE - 1) / pk::TILE + 1) / 2) *
                        (((a.N + pk::TILE - 1) / pk::TILE + 1) / 2);
  const int64_t nkb = (a.K + pk::BK - 1) / pk::BK;
  if (tiles <= 0 || tiles >= 76) return 1;
  const int64_t want = 76 / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, nkb / 16, 64}));
}

// Tail split of the CTA pairs: with more pair tiles than pairs (76) and a
// last round of entries that would leave pairs idle, the tiles of that round
// share out their K blocks (each part >= 512 K), at most one entry per pair;
// the other tiles are whole entries.  Returns the parts per tail tile (1: no
// tail split) and sets *nfull, the whole entries.
int pk_tail_split_p(const GemmArgs& a, int64_t* nfull) {
  const int64_t tiles = (((a.M + pk::TILE - 1) / pk::TILE + 1) / 2) *
                        (((a.N + pk::TILE - 1) / pk::TILE + 1) / 2);
  const int64_t nkb = (a.K + pk::BK - 1) / pk::BK;
  *nfull = tiles;
  if (tiles <= 76 || tiles % 76 == 0) return 1;
  const int64_t rem = tiles % 76;
  const int64_t parts = std::min<int64_t>(76 / rem, nkb / 16);
  if (parts < 2) return 1;
  *nfull = tiles - rem;
  return (int)parts;
}

// Split-K of the BF16x6 CTA pairs (256 x 128 pair tiles): the same rule.
int pk_ksplit_p6(const GemmArgs& a) {
  const int64_t tiles = (((a.M + pk::TILE - 1) / pk::TILE + 1) / 2) *
                        ((a.N + pk::TILE - 1) / pk::TILE);
  const int64_t nkb = (a.K + pk::BK - 1) / pk::BK;
  if (tiles <= 0 || tiles >= 76) return 1;
  const int64_t want = 76 / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, nkb / 16, 64}));
}

size_t pk_part_bytes(const GemmArgs& a, int tile) {
  const int sp = tile == kTilePackedWide ? pk_ksplit_w(a)
                 : tile == kTilePackedPair ? (a.math == TC_MATH_BF16X6 ? pk_ksplit_p6(a)
                                                                       : pk_ksplit_p(a))
                 : pk_ksplit(a);
  if (tile == kTilePackedPair && a.math != TC_MATH_BF16X6) {
    int64_t nfull = 0;
    const int ts = pk_tail_split_p(a, &nfull);
    if (ts > 1) {
      const int64_t ptiles = (((a.M + pk::TILE - 1) / pk::TILE + 1) / 2) *
                             (((a.N + pk::TILE - 1) / pk::TILE + 1) / 2);
      return (size_t)ts * (size_t)(ptiles - nfull) * 4 * pk::TILE * pk::TILE * sizeof(float2);
    }
  }
  if (sp <= 1) return 0;
  const int64_t tiles = ((a.M + pk::TILE - 1) / pk::TILE) * ((a.N + pk::TILE - 1) / pk::TILE);
  return (size_t)sp * (size_t)tiles * pk::TILE * pk::TILE * sizeof(float2);
}

PkLayout pk_layout(const GemmArgs& a, int math) {
  PkLayout L;
  std::memset(&L, 0, sizeof(L));
  const int nt = terms_of(math);
  L.tiles_m = (a.M + pk::TILE - 1) / pk::TILE;
  L.tiles_n = (a.N + pk::TILE - 1) / pk::TILE;
  L.nkb = (a.K + pk::BK - 1) / pk::BK;
  L.off_qa = 0;
  L.off_qb = align256((size_t)L.tiles_m * L.nkb * nt * pk::TERM);
  L.bytes = L.off_qb + align256((size_t)L.tiles_n * L.nkb * nt * pk::TERM);
  return L;
}

int pk_stage_blocks(int math) {
  return (math == TC_MATH_BF16 || math == TC_MATH_FP16) ? pk::Cfg<1>::BPS
         : math == TC_MATH_BF16X3 ? pk::Cfg<2>::BPS : pk::Cfg<3>::BPS;
}

tc_status launch_gemm_tc_packed(const GemmArgs& a, int math, tc_dtype dt, int tile, void* ws,
                                void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const PkLayout L = pk_layout(a, math);
  if (L.tiles_m == 0 || L.tiles_n == 0 || L.nkb == 0) return TC_OK;
  if (tile == kTilePackedPair && math == TC_MATH_BF16X6)
    return dt == TC_F32 ? pk::launch_p6<3>(a, L, ws, s) : TC_ERR_UNSUPPORTED;
  if (tile == kTilePackedPair) {
    if (dt == TC_BF16 && math == TC_MATH_BF16)
      return pk::launch_p<1, __nv_bfloat16, false>(a, L, ws, s, 1);
    if (dt == TC_F16 && math == TC_MATH_FP16)
      return pk::launch_p<1, __half, true>(a, L, ws, s, 2);
    if (dt != TC_F32) return TC_ERR_UNSUPPORTED;
    switch (math) {
      case TC_MATH_BF16: return pk::launch_p<1, float, false>(a, L, ws, s, 0);
      case TC_MATH_FP16: return pk::launch_p<1, float, true>(a, L, ws, s, 0);
      case TC_MATH_BF16X3: return pk::launch_p<2, float, false>(a, L, ws, s, 0);
      default: return TC_ERR_UNSUPPORTED;
    }
  }
  if (tile == kTilePackedWide) {
    if (dt == TC_BF16 && math == TC_MATH_BF16)
      return pk::launch_w<1, __nv_bfloat16, false>(a, L, ws, s, 1);
    if (dt == TC_F16 && math == TC_MATH_FP16)
      return pk::launch_w<1, __half, true>(a, L, ws, s, 2);
    if (dt != TC_F32) return TC_ERR_UNSUPPORTED;
    switch (math) {
      case TC_MATH_BF16: return pk::launch_w<1, float, false>(a, L, ws, s, 0);
      case TC_MATH_FP16: return pk::launch_w<1, float, true>(a, L, ws, s, 0);
      case TC_MATH_BF16X3: return pk::launch_w<2, float, false>(a, L, ws, s, 0);
      default: return TC_ERR_UNSUPPORTED;
    }
  }
  if (dt == TC_BF16 && math == TC_MATH_BF16)
    return pk::launch<1, __nv_bfloat16, false>(a, L, ws, s, 1);
  if (dt == TC_F16 && math == TC_MATH_FP16) return pk::launch<1, __half, true>(a, L, ws, s, 2);
  if (dt != TC_F32) return TC_ERR_UNSUPPORTED;
  switch (math) {
    case TC_MATH_BF16: return pk::launch<1, float, false>(a, L, ws, s, 0);
    case TC_MATH_FP16: return pk::launch<1, float, true>(a, L, ws, s, 0);
    case TC_MATH_BF16X3: return pk::launch<2, float, false>(a, L, ws, s, 0);
    case TC_MATH_BF16X6: return pk::launch<3, float, false>(a, L, ws, s, 0);
    default: return TC_ERR_UNSUPPORTED;
  }
}

tc_status launch_gemm_tc_packed_batch(const PkBatch& b, const void* const* A,
                                      const void* const* B, void* const* C, const double* alpha,
                                      const double* beta, int math, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (math) {
    case TC_MATH_BF16: return pk::launch_batch<1>(b, A, B, C, alpha, beta, s);
    case TC_MATH_BF16X3: return pk::launch_batch<2>(b, A, B, C, alpha, beta, s);
    case TC_MATH_BF16X6: return pk::launch_batch<3>(b, A, B, C, alpha, beta, s);
    default: return TC_ERR_UNSUPPORTED;
  }
}

tc_status tc_pk_read_status(int* h, void* stream) {
  return read_clear_status(h, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TC_OK
                                                                                : TC_ERR_CUDA;
}

}  // namespace tc
