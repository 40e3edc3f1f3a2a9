// k_fp8.cu -- the FP8-E4M3 form of a Class 3 contraction on the tensor cores
// (sm_103a, tcgen05 kind::mxf8f6f4), with one power-of-two scale per operand
// row and block of 128 consecutive K.
//
// The GEMM view is that of the fused mapping (M = free indices of the first
// operand, N = those of the second, K = the contracted indices in ascending
// order of their strides in A).  Row m of the first operand is cut into
// blocks k in [128 j, 128 j + 128); its block j is stored as E4M3 codes of
// x / 2^e with e = e_A(m, j) the smallest integer for which the block's
// largest |x| / 2^e <= 448 (never below -126); the same for the columns of
// the second operand.  Then
//   C[m, n] = alpha * sum_j 2^(e_A(m, j) + e_B(n, j)) * sum_{k in block j} qa qb
//           + beta * C[m, n].
//
// Two kernels:
//   k_fp8_pack   one CTA per (128-row tile, K block) of each operand: gathers
//                the FP32 block through the index groups (coalesced along the
//                operand's contiguous index), finds each row's exponent,
//                rounds to E4M3 and writes the 16 KB block in the tensor
//                cores' canonical K-major layout (8-row x 16-byte core
//                matrices: byte (k / 16) * 2048 + row * 16 + k % 16), plus each
//                row's scale as an exponent byte e + 127 (UE8M0).  The operand
//                is read from HBM once; the GEMM never touches the FP32 data.
//   k_gemm_fp8   persistent, one CTA per SM over 128 x 256 output tiles, on
//                the block-scaled MMA (kind::mxf8f6f4): the tensor cores
//                multiply each K = 32 step by 2^(e_A + e_B) of its rows and
//                columns and accumulate all of K in FP32 in tensor memory.
//                Each block of A feeds two N = 128 MMAs (one per half of the
//                tile), a third more multiply-adds per byte moved than a
//                128 x 128 tile.
//                warp 0     one thread moves each (tile, block) triple of packed
//                           blocks (A and both halves of B) into a 4-stage
//                           shared-memory ring with bulk copies
//                           (cp.async.bulk, mbarrier transaction count);
//                warp 1     tensor-memory allocation; one thread issues the
//                           eight K = 32 MMAs of each block;
//                warps 2-5  one per lane quadrant: write the scale bytes of
//                           four consecutive blocks into tensor memory (a ring
//                           of 4 x 12 columns) ahead of the MMAs;
//                warps 6-13 epilogue, once per tile: two warps per lane
//                           quadrant, one per half, read 64 accumulator
//                           columns at a time (the accumulator, 256 columns,
//                           is released after the last read), apply alpha and
//                           beta and store through C's strides.
//   k_gemm_fp8<true> (tile configuration 1, on request) packs the first
//                operand inside the GEMM launch: four more warps per CTA
//                quantise half tiles of A loaded by TMA and release them to
//                the producers through per-block counts (see pack_warps);
//                only the second operand is packed by k_fp8_pack first.
// Scale bytes in tensor memory (one layout for A and B, in all four lane
// quadrants): lane 32 q + l, column c of a group, byte j holds the exponent of
// row (A) or column (B) 32 c + l for the group's block j.  The MMA takes row
// m's from lane m, column m / 32, and column n's (for the rows of quadrant q)
// from lane 32 q + n % 32, column n / 32; the instruction descriptor selects
// the byte.
// The products of E4M3 values and their power-of-two scaling are exact; the
// error against the exact sum of the dequantised products is that of the
// tensor cores' FP32 accumulation over K.
#include <cuda.h>  // CUtensorMap and cuTensorMapEncodeTiled's types (entry point via the runtime)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "groups.cuh"
#include "sm100.cuh"
#include "tc_internal.h"

namespace tc {

namespace fp8 {

constexpr int TILE = 128;                 // rows of a tile (M and N)
constexpr int KB = 128;                   // K block: one scale, one pipeline stage
constexpr uint32_t CHUNK = TILE * KB;     // bytes of one packed (tile, block)
constexpr int kPackThreads = 512;
constexpr int kRowThreads = kPackThreads / TILE;  // threads sharing one row (or one k)
constexpr int kLd = KB + 1;               // shared-memory row pitch of the pack tile (floats)
constexpr uint32_t kPackSmem =
    TILE * kLd * 4 + 2 * TILE * 8 + TILE * 4 + kRowThreads * TILE * 4;

// The GEMM's output tile is 128 x 256: two N = 128 halves share each block
// of the first operand (one 16 KB block of A and two of B per stage).
constexpr uint32_t STAGE = 3 * CHUNK;
constexpr int NG = 4;                     // groups of scale columns in tensor memory
constexpr uint32_t COL_SF = 2 * TILE;     // accumulator halves at 0 and 128; then the scales,
                                          // 12 columns per group (A 0-3, B halves 4-7, 8-11)
constexpr int kEpiThreads = 256;
constexpr int kThreads = 64 + 128 + kEpiThreads;
constexpr int kPackWarpThreads = 128;     // in-kernel packing: four more warps
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kTimeoutNs = 2000000000ull;
// In-kernel packing of the first operand takes it in half tiles: 64 rows x one
// 128-K block of FP32 (32 KB), two in flight per CTA.
constexpr int HROWS = 64;
constexpr uint32_t HALF_BYTES = HROWS * KB * 4;

// Shared memory of the GEMM: the operand ring (4 stages; 3 when the CTA
// packs the first operand too, whose two half-tile buffers follow it), C's
// column offsets, the barriers.
template <bool FUSE>
struct Cfg {
  static constexpr int S = FUSE ? 3 : 4;
  static constexpr int THREADS = kThreads + (FUSE ? kPackWarpThreads : 0);
  static constexpr uint32_t OFF_PK = S * STAGE;
  static constexpr uint32_t OFF_COLC = OFF_PK + (FUSE ? 2 * HALF_BYTES : 0);  // int64 colC[2][256]
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * 2 * TILE * 8;
  static constexpr uint32_t NBAR = 2 * S + 2 + 2 * NG + 1 + 2;   // ring, acc, scales, done, pack
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  // misc: TMEM address, abort flag, pack units [2], pack failure; then the
  // pack warps' partial row maxima [4 warps][64 rows]
  static constexpr uint32_t OFF_PM = (OFF_MISC + 32 + 15) & ~15u;
  static constexpr uint32_t BYTES = OFF_PM + 4 * HROWS * 4 + 128;  // + alignment slack
};

// Scale bytes of one operand: per (tile, group of 4 blocks) 512 bytes laid
// out as the tensor-memory cells of one lane quadrant: [l][c][j] = row
// 32 c + l, block 4 g + j.
__host__ __device__ constexpr int64_t sf_index(int64_t tile, int64_t ngroups, int kb, int r) {
  return ((tile * ngroups + kb / 4) * 32 + (r & 31)) * 16 + (r >> 5) * 4 + (kb & 3);
}

// Exponent e of a row block whose largest |x| is m (m >= 0): the smallest
// integer with m / 2^e <= 448, never below -126.  With m = f * 2^E, f in
// [1, 2): m <= 448 * 2^e  <=>  e >= E - 8 (f <= 1.75) or e >= E - 7
// (f > 1.75); zero and FP32-subnormal maxima give -126.
__device__ __forceinline__ int row_exponent(float m) {
  const uint32_t b = __float_as_uint(m);
  const int be = (int)(b >> 23);
  const int e = be == 0 ? -126 : be - 135 + ((b & 0x7FFFFFu) > 0x600000u ? 1 : 0);
  return max(e, -126);
}

// E4M3 codes of 16 consecutive K of one row (src[0..15] times the row's
// factor), as the 16-byte row of a core matrix.
__device__ __forceinline__ uint4 e4m3_row16(const float* src, int stride, float mul) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = pack_e4m3x2(src[(4 * i) * stride] * mul, src[(4 * i + 1) * stride] * mul);
    const uint32_t hi =
        pack_e4m3x2(src[(4 * i + 2) * stride] * mul, src[(4 * i + 3) * stride] * mul);
    w[i] = lo | (hi << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// The same for component J of v[0..15] (16 consecutive K of one row held as
// one component of 16 float4 registers).
template <int J>
__device__ __forceinline__ float comp(const float4& x) {
  return J == 0 ? x.x : J == 1 ? x.y : J == 2 ? x.z : x.w;
}
template <int J>
__device__ __forceinline__ uint4 e4m3_row16_of(const float4 (&v)[16], float mul) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t lo = pack_e4m3x2(comp<J>(v[4 * i]) * mul, comp<J>(v[4 * i + 1]) * mul);
    const uint32_t hi = pack_e4m3x2(comp<J>(v[4 * i + 2]) * mul, comp<J>(v[4 * i + 3]) * mul);
    w[i] = lo | (hi << 16);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

struct PackArgs {
  Group gr[2];          // rows of operand o (the M and N groups); strides in slot o
  Group gk;             // K group; operand o's strides in slot o
  const float* in[2];
  uint8_t* q[2];        // packed blocks [tile][block][CHUNK]
  uint8_t* sf[2];       // scale bytes e + 127, sf_index layout
  int64_t rows[2];
  int64_t K;
  int64_t nblocks0;     // CTAs of operand 0 (tiles[0] * nkb)
  int32_t tiles[2];
  int32_t nkb, ngroups;
  int32_t rows_fast[2]; // operand contiguous along its rows: load row-fastest
};

__global__ void __launch_bounds__(kPackThreads) k_fp8_pack(const __grid_constant__ PackArgs P) {
  extern __shared__ float4 pack_smem[];
  float* tile = reinterpret_cast<float*>(pack_smem);
  int64_t* roff = reinterpret_cast<int64_t*>(tile + TILE * kLd);
  int64_t* koff = roff + TILE;
  float* qmul = reinterpret_cast<float*>(koff + KB);
  float* pmax4 = qmul + TILE;  // [kRowThreads][128] partial row maxima (rows_fast)

  int64_t bid = blockIdx.x;
  const int o = bid < P.nblocks0 ? 0 : 1;
  if (o) bid -= P.nblocks0;
  const int t = (int)(bid / P.nkb), kb = (int)(bid % P.nkb);
  const int tid = threadIdx.x;
  if (tid < TILE) {
    const int64_t r = (int64_t)t * TILE + tid;
    roff[tid] = r < P.rows[o] ? goff(P.gr[o], o, (uint32_t)r) : -1;
  } else if (tid < 2 * TILE) {
    const int64_t k = (int64_t)kb * KB + (tid - TILE);
    koff[tid - TILE] = k < P.K ? goff(P.gk, o, (uint32_t)k) : -1;
  }
  __syncthreads();

  // gather the FP32 block; consecutive threads take consecutive elements of
  // the operand's contiguous index.  All of a thread's loads are issued before
  // their shared-memory stores, so that they are in flight at once.
  const float* __restrict__ X = P.in[o];
  constexpr int NJ = TILE * KB / kPackThreads;
  float* pmax = qmul;  // row maxima, then (below) the rows' quantisation factors
  if (P.rows_fast[o]) {
    const int r = tid & (TILE - 1), k0 = tid / TILE;
    const int64_t ro = roff[r];
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int64_t ko = koff[k0 + kRowThreads * j];
      v[j] = (ro >= 0 && ko >= 0) ? __ldg(X + ro + ko) : 0.0f;
    }
    float m = 0.0f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      tile[r * kLd + k0 + kRowThreads * j] = v[j];
      m = fmaxf(m, fabsf(v[j]));
    }
    pmax4[k0 * TILE + r] = m;
    __syncthreads();
    if (tid < TILE) {
      float mm = pmax4[tid];
#pragma unroll
      for (int i = 1; i < kRowThreads; ++i) mm = fmaxf(mm, pmax4[i * TILE + tid]);
      pmax[tid] = mm;
    }
  } else {
    const int k = tid & (KB - 1), r0 = tid / KB;
    const int64_t ko = koff[k];
    float v[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int64_t ro = roff[r0 + kRowThreads * j];
      v[j] = (ro >= 0 && ko >= 0) ? __ldg(X + ro + ko) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) tile[(r0 + kRowThreads * j) * kLd + k] = v[j];
    __syncthreads();
    if (tid < TILE) {  // one thread per row: consecutive rows fall in distinct banks
      float m = 0.0f;
#pragma unroll 8
      for (int j = 0; j < KB; ++j) m = fmaxf(m, fabsf(tile[tid * kLd + j]));
      pmax[tid] = m;
    }
  }
  __syncthreads();

  // exponent of each row
  if (tid < TILE) {
    const int r = tid;
    const int e = row_exponent(pmax[r]);
    qmul[r] = __uint_as_float((uint32_t)(127 - e) << 23);                   // 2^-e
    P.sf[o][sf_index(t, P.ngroups, kb, r)] = (uint8_t)(127 + e);
  }
  __syncthreads();

  // round to E4M3 and store: unit u = (k / 16) * 128 + row is the 16-byte row
  // of a core matrix, at byte u * 16 of the block
  uint8_t* __restrict__ Q = P.q[o] + ((int64_t)t * P.nkb + kb) * CHUNK;
#pragma unroll
  for (int j = 0; j < (int)(CHUNK / 16) / kPackThreads; ++j) {
    const int u = tid + j * kPackThreads;
    const int kc = u >> 7, r = u & (TILE - 1);
    *reinterpret_cast<uint4*>(Q + (size_t)u * 16) = e4m3_row16(tile + r * kLd + kc * 16, 1, qmul[r]);
  }
}

struct GemmFp8 {
  CUtensorMap tma_a;     // in-kernel packing: A's FP32 elements as [K][M], M contiguous
  CUtensorMap tma_qa;    // CTA pairs: the packed blocks of A and B as rows of 2 KB
  CUtensorMap tma_qb;
  Group gm, gn;          // C offsets in slot 2
  uint8_t* qa;           // packed blocks (written by the pack warps when they pack A)
  const uint8_t* qb;
  uint8_t* sfa;          // scale bytes, sf_index layout
  const uint8_t* sfb;
  uint32_t* ready;       // in-kernel packing: half tiles packed per (tile of A, block)
  uint32_t* next_unit;   // in-kernel packing: the pack units' claim counter
  float* C;
  int64_t M, N, ntiles;
  int64_t units;         // in-kernel packing: half-tile units (tiles_m * nkb * 2)
  float alpha, beta;
  int32_t tiles_m, tiles_n, tiles_p, nkb, ngroups, raster;  // tiles_p: pairs of 128-column tiles
  int32_t group_tiles;   // in-kernel packing: tiles of A per group of pack units
};

// Output tile w: 128-row tile tm and the pair tp of 128-column tiles 2 tp and
// 2 tp + 1 (the second exists when 2 tp + 1 < tiles_n).
__device__ __forceinline__ void tile_coords(const GemmFp8& P, int64_t w, int& tm, int& tp) {
  if (P.raster) {
    tp = (int)(w % P.tiles_p);
    tm = (int)(w / P.tiles_p);
  } else {
    tm = (int)(w % P.tiles_m);
    tp = (int)(w / P.tiles_m);
  }
}

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  bool ok = (*abort == 0) && mbar_wait(bar, parity, abort, kTimeoutNs);
  return __all_sync(0xffffffffu, ok);
}

// In-kernel packing of the first operand (FUSE): the four pack warps of every
// CTA take half-tile units (64 rows of A x one 128-K block) in the order the
// GEMM's tiles need them (groups of `group_tiles` tiles of A, block-major
// within a group), claimed from a global counter in batches of four; a batch
// is prefetched into L2 when the one before it starts, and each unit is then
// loaded by TMA (zero fill outside A) into one of two buffers.  It is
// quantised exactly as k_fp8_pack does (thread t: rows 4 (t % 16) .. + 3 and
// K [16 (t / 16), + 16); one pass over shared memory for the row maxima, one
// for the codes).  The codes (the packed block's layout restricted to the
// unit's rows) and the unit's scale bytes (within the zeroed 512-byte cell
// record of its group of four blocks) are staged in the unit's buffer and
// written by a bulk store and a bulk OR; the unit is counted in
// ready[tile * nkb + block], with release semantics, once they have completed
// (checked one unit later, so that the wait is rarely felt).  The pack warps
// wait on nothing but their own copies, so every claimed unit is finished
// whichever CTAs are resident: the GEMM's waits on `ready` always end.
constexpr int kClaim = 4;  // pack units per claim

// Warp-wide bounded poll of the pack counts of one tile of A: returns the
// number n >= need of consecutive blocks kb, kb + 1, ... (up to 32; blocks
// from nkb on count as packed) whose two halves are packed, or 0 once the
// wait has given up (*abort set by any thread, or the time limit: then it
// records TC_ERR_TIMEOUT and sets *abort).  Every exit is warp-uniform.
__device__ __forceinline__ int poll_packed(const uint32_t* row, int kb, int nkb, int need,
                                           volatile int* abort) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  for (;;) {
    const int q = kb + lane;
    const bool rdy = q >= nkb || ld_acquire_gpu(row + q) >= 2u;
    const uint32_t msk = __ballot_sync(0xffffffffu, rdy);
    const int n = msk == 0xffffffffu ? 32 : __ffs(~msk) - 1;
    if (n >= need) return n;
    if (__any_sync(0xffffffffu, *abort != 0)) return 0;
    const uint64_t now = __shfl_sync(0xffffffffu, globaltimer_ns(), 0);
    if (t0 == 0) {
      t0 = now;
    } else if (now - t0 > kTimeoutNs) {
      if (lane == 0) {
        *abort = 1;
        atomicExch(&g_device_status, 1);
      }
      return 0;
    }
    __nanosleep(64);
  }
}

template <class Cf>
__device__ __forceinline__ void pack_warps(const GemmFp8& P, uint8_t* smem, uint64_t* pbar) {
  const int pt = threadIdx.x - kThreads;  // 0 .. 127
  const int rg = pt & 15, kc = pt >> 4;   // rows 4 rg .. 4 rg + 3, K [16 kc, 16 kc + 16)
  const int pw = pt >> 5;
  volatile int32_t* unit = reinterpret_cast<volatile int32_t*>(smem + Cf::OFF_MISC + 8);
  volatile int* pk_fail = reinterpret_cast<volatile int*>(smem + Cf::OFF_MISC + 16);
  float4* pm = reinterpret_cast<float4*>(smem + Cf::OFF_PM);  // [4 warps][16 row groups]
  const uint32_t buf0 = smem_u32(smem + Cf::OFF_PK);
  const int64_t units = P.units;
  const int nkb = P.nkb;
  const int64_t gsz = (int64_t)P.group_tiles * nkb * 2;
  auto coords = [&](int64_t u, int& tm, int& kb, int& hf) {
    const int64_t gi = u / gsz, r = u - gi * gsz;
    const int g0 = (int)(gi * P.group_tiles);
    const int gcnt = min(P.group_tiles, P.tiles_m - g0);
    kb = (int)(r / (2 * gcnt));
    const int rem = (int)(r % (2 * gcnt));
    tm = g0 + (rem >> 1);
    hf = rem & 1;
  };
  auto issue = [&](int32_t u, int b) {
    int tm, kb, hf;
    coords(u, tm, kb, hf);
    mbar_arrive_expect_tx(&pbar[b], HALF_BYTES);
    tma_load_2d(buf0 + (uint32_t)b * HALF_BYTES, &P.tma_a, tm * TILE + hf * HROWS, kb * KB,
                &pbar[b]);
  };
  auto prefetch = [&](int32_t base) {
    for (int q = 0; q < kClaim; ++q) {
      if (base + q >= units) break;
      int tm, kb, hf;
      coords(base + q, tm, kb, hf);
      tma_prefetch_2d(&P.tma_a, tm * TILE + hf * HROWS, kb * KB);
    }
  };
  auto release = [&](int32_t u) {  // thread 0, once unit u's bulk writes are complete
    fence_proxy_async_global();
    int tm, kb, hf;
    coords(u, tm, kb, hf);
    red_release_gpu_add(P.ready + (size_t)tm * nkb + kb, 1u);
  };
  // thread 0's units: batch `cur` (next index k), then `nxt` (prefetched),
  // then `nxt2` (claimed; its value is first used a batch later)
  int32_t cur = 0, nxt = 0, nxt2 = 0, done_u = -1;
  int k = kClaim;
  auto seq = [&]() -> int32_t {
    if (k == kClaim) {
      cur = nxt;
      nxt = nxt2;
      k = 0;
      if (nxt < units) prefetch(nxt);
      nxt2 = (int32_t)atomicAdd(P.next_unit, (uint32_t)kClaim);
    }
    return cur + k++;
  };
  if (pt == 0) {
    nxt = (int32_t)atomicAdd(P.next_unit, (uint32_t)kClaim);
    if (nxt < units) prefetch(nxt);
    nxt2 = (int32_t)atomicAdd(P.next_unit, (uint32_t)kClaim);
    const int32_t u0 = seq(), u1 = seq();
    unit[0] = u0;
    unit[1] = u1;
    *pk_fail = 0;
    if (u0 < units) issue(u0, 0);
    if (u1 < units) issue(u1, 1);
  }
  named_bar_sync(2, kPackWarpThreads);
  for (uint32_t i = 0;; ++i) {
    const int b = (int)(i & 1);
    const int32_t u = unit[b];
    if (u >= units) break;
    if (pt == 0) {
      volatile int never = 0;
      if (!mbar_wait(&pbar[b], (i >> 1) & 1, &never, kTimeoutNs)) *pk_fail = 1;
    }
    named_bar_sync(2, kPackWarpThreads);
    if (*pk_fail) {  // written by thread 0 before the barrier: a uniform decision
      if (pt == 0) {  // let the other buffer's copy (if any) land before exit
        volatile int never = 0;
        if (unit[b ^ 1] < units) mbar_wait(&pbar[b ^ 1], ((i + 1) >> 1) & 1, &never, kTimeoutNs);
      }
      break;
    }
    int tm, kb, hf;
    coords(u, tm, kb, hf);
    uint8_t* X = smem + Cf::OFF_PK + (uint32_t)b * HALF_BYTES;
    const float4* X4 = reinterpret_cast<const float4*>(X);  // [k][16 row groups]
    // pass 1: row maxima of this thread's 16 K, then across the 8 K chunks
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 v = X4[(kc * 16 + q) * 16 + rg];
      m.x = fmaxf(m.x, fabsf(v.x));
      m.y = fmaxf(m.y, fabsf(v.y));
      m.z = fmaxf(m.z, fabsf(v.z));
      m.w = fmaxf(m.w, fabsf(v.w));
    }
    // the two K chunks of a warp share row groups (lanes l and l + 16)
    m.x = fmaxf(m.x, __shfl_xor_sync(0xffffffffu, m.x, 16));
    m.y = fmaxf(m.y, __shfl_xor_sync(0xffffffffu, m.y, 16));
    m.z = fmaxf(m.z, __shfl_xor_sync(0xffffffffu, m.z, 16));
    m.w = fmaxf(m.w, __shfl_xor_sync(0xffffffffu, m.w, 16));
    if ((pt & 31) < 16) pm[pw * 16 + rg] = m;
    named_bar_sync(2, kPackWarpThreads);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float4 o = pm[w * 16 + rg];
      m.x = fmaxf(m.x, o.x);
      m.y = fmaxf(m.y, o.y);
      m.z = fmaxf(m.z, o.z);
      m.w = fmaxf(m.w, o.w);
    }
    const float f0 = __uint_as_float((uint32_t)(127 - row_exponent(m.x)) << 23);  // 2^-e
    const float f1 = __uint_as_float((uint32_t)(127 - row_exponent(m.y)) << 23);
    const float f2 = __uint_as_float((uint32_t)(127 - row_exponent(m.z)) << 23);
    const float f3 = __uint_as_float((uint32_t)(127 - row_exponent(m.w)) << 23);
    // this thread's word of the group's scale-cell record: lane l = pt / 4,
    // column c = pt % 4 (row 32 c + l), byte kb % 4; rows of the other half 0
    uint32_t sfw = 0;
    {
      const int c = pt & 3, l = pt >> 2;
      if ((c >> 1) == hf) {
        const int hr = 32 * (c & 1) + l;  // row within the half
        float mm = 0.0f;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const float4 o = pm[w * 16 + (hr >> 2)];
          const float x = (hr & 3) == 0 ? o.x : (hr & 3) == 1 ? o.y : (hr & 3) == 2 ? o.z : o.w;
          mm = fmaxf(mm, x);
        }
        sfw = (uint32_t)(127 + row_exponent(mm)) << (8 * (kb & 3));
      }
    }
    // pass 2: E4M3 codes, two K at a time; word q of a row's 16 bytes holds
    // K 4 q .. 4 q + 3 (the row layout of e4m3_row16)
    uint32_t q0[4], q1[4], q2[4], q3[4];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 a = X4[(kc * 16 + 2 * q) * 16 + rg];
      const float4 c = X4[(kc * 16 + 2 * q + 1) * 16 + rg];
      const uint32_t h0 = pack_e4m3x2(a.x * f0, c.x * f0), h1 = pack_e4m3x2(a.y * f1, c.y * f1);
      const uint32_t h2 = pack_e4m3x2(a.z * f2, c.z * f2), h3 = pack_e4m3x2(a.w * f3, c.w * f3);
      if ((q & 1) == 0) {
        q0[q >> 1] = h0;
        q1[q >> 1] = h1;
        q2[q >> 1] = h2;
        q3[q >> 1] = h3;
      } else {
        q0[q >> 1] |= h0 << 16;
        q1[q >> 1] |= h1 << 16;
        q2[q >> 1] |= h2 << 16;
        q3[q >> 1] |= h3 << 16;
      }
    }
    named_bar_sync(2, kPackWarpThreads);  // every read of X done: stage into it
    uint4* st = reinterpret_cast<uint4*>(X + kc * 1024 + rg * 64);
    st[0] = make_uint4(q0[0], q0[1], q0[2], q0[3]);
    st[1] = make_uint4(q1[0], q1[1], q1[2], q1[3]);
    st[2] = make_uint4(q2[0], q2[1], q2[2], q2[3]);
    st[3] = make_uint4(q3[0], q3[1], q3[2], q3[3]);
    reinterpret_cast<uint32_t*>(X + 8192)[pt] = sfw;
    fence_proxy_async_shared();  // the staged bytes are read by bulk copies
    named_bar_sync(2, kPackWarpThreads);
    if (pt == 0) {
      uint8_t* Q = P.qa + ((size_t)tm * nkb + kb) * CHUNK + (size_t)hf * 1024;
      const uint32_t xs = smem_u32(X);
#pragma unroll
      for (int q = 0; q < KB / 16; ++q) bulk_s2g(Q + (size_t)q * 2048, xs + q * 1024, 1024);
      bulk_or_s2g(P.sfa + ((size_t)tm * P.ngroups + (kb >> 2)) * 512, xs + 8192, 512);
      bulk_commit();
      if (done_u >= 0) {  // the previous unit: complete by now, as a rule
        bulk_wait<1>();
        release(done_u);
      }
      done_u = u;
      // buffer b takes the unit after next once its staged bytes are read
      const int32_t un = seq();
      unit[b] = un;
      if (un < units) {
        bulk_wait_read<0>();
        issue(un, b);
      }
    }
  }
  if (pt == 0) {
    bulk_wait<0>();
    if (done_u >= 0) release(done_u);
  }
}

template <bool FUSE>
__global__ void __launch_bounds__(Cfg<FUSE>::THREADS, 1) k_gemm_fp8(const __grid_constant__ GemmFp8 P) {
  using Cf = Cfg<FUSE>;
  constexpr int S = Cf::S;
  extern __shared__ uint8_t fp8_smem_raw[];
  // the operand layouts have no swizzle: 128-byte alignment is enough
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(fp8_smem_raw) + 127) & ~(uintptr_t)127);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + Cf::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cf::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 1;
  uint64_t* sff = acce + 1;
  uint64_t* sfe = sff + NG;
  uint64_t* done = sfe + NG;
  uint64_t* pbar = done + 1;  // pack warps' two half-tile buffers (FUSE)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cf::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + Cf::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, kEpiThreads);
    for (int i = 0; i < NG; ++i) {
      mbar_init(&sff[i], 128);
      mbar_init(&sfe[i], 1);
    }
    mbar_init(done, 1);
    mbar_init(&pbar[0], 1);
    mbar_init(&pbar[1], 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(smem);
  const int nkb = P.nkb, ngroups = P.ngroups;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // One thread issues the copies; with in-kernel packing the warp first
    // polls the pack counts of up to 32 blocks of A at a time.
    uint32_t g = 0;
    bool ok = true;
    for (int64_t w = blockIdx.x; ok && w < P.ntiles; w += gridDim.x) {
      int tm, tp;
      tile_coords(P, w, tm, tp);
      const bool h1 = 2 * tp + 1 < P.tiles_n;
      const uint8_t* a = P.qa + (size_t)tm * nkb * CHUNK;
      const uint8_t* b = P.qb + (size_t)(2 * tp) * nkb * CHUNK;
      int horizon = 0;  // blocks [0, horizon) of this tile of A known packed
      for (int kb = 0; kb < nkb; ++kb, ++g) {
        const int s = (int)(g % S);
        if (g >= (uint32_t)S) {
          const bool got =
              lane != 0 || mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs);
          if (!__all_sync(0xffffffffu, got)) {
            ok = false;
            break;
          }
        }
        if constexpr (FUSE) {
          if (kb >= horizon) {
            const int n = poll_packed(P.ready + (size_t)tm * nkb, kb, nkb, 1, abort);
            if (n == 0) {
              ok = false;
              break;
            }
            horizon = kb + n;
            fence_proxy_async_global();  // the packed bytes are read by bulk copies
          }
        }
        if (lane == 0) {
          const uint32_t dst = sbase + (uint32_t)s * STAGE;
          mbar_arrive_expect_tx(&full[s], (h1 ? 3 : 2) * CHUNK);
          bulk_g2s(dst, a + (size_t)kb * CHUNK, CHUNK, &full[s]);
          bulk_g2s(dst + CHUNK, b + (size_t)kb * CHUNK, CHUNK, &full[s]);
          if (h1) bulk_g2s(dst + 2 * CHUNK, b + (size_t)(nkb + kb) * CHUNK, CHUNK, &full[s]);
        }
        __syncwarp();
      }
    }
    if (lane == 0) {
      // the copies still in flight (at most the last S blocks) land before exit
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&full[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issue
      constexpr uint32_t LBO = (TILE / 8) * 128;   // next 16-byte K chunk
      uint32_t g = 0, G = 0, t = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; ok && w < P.ntiles; w += gridDim.x, ++t) {
        int tm, tp;
        tile_coords(P, w, tm, tp);
        const bool h1 = 2 * tp + 1 < P.tiles_n;
        // the accumulator is free once the epilogue has read the previous tile
        if (t >= 1 && !mbar_wait(acce, (t - 1) & 1, abort, kTimeoutNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const uint32_t slot = G % NG;
          if ((kb & 3) == 0) {  // the group's scale columns are written
            if (!mbar_wait(&sff[slot], (G / NG) & 1, abort, kTimeoutNs)) {
              ok = false;
              break;
            }
          }
          const int s = (int)(g % S);
          if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = sbase + (uint32_t)s * STAGE;
          const uint32_t id = (uint32_t)(kb & 3);
          const uint32_t idesc = idesc_mx_e4m3(TILE, TILE, id, id);
          const uint32_t tsf = tmem + COL_SF + slot * 12;
#pragma unroll
          for (int kk = 0; kk < KB / 32; ++kk) {
            const uint64_t da = smem_desc(sa + kk * 2 * LBO, LBO, 128);
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            mma_mx_e4m3(tmem, da, smem_desc(sa + CHUNK + kk * 2 * LBO, LBO, 128), idesc, tsf,
                        tsf + 4, acc);
            if (h1)
              mma_mx_e4m3(tmem + TILE, da, smem_desc(sa + 2 * CHUNK + kk * 2 * LBO, LBO, 128),
                          idesc, tsf, tsf + 8, acc);
          }
          mma_commit(&empty[s]);
          if ((kb & 3) == 3 || kb == nkb - 1) {
            mma_commit(&sfe[slot]);  // the group's scale columns may be rewritten
            ++G;
          }
        }
        if (!ok) break;
        mma_commit(accf);
      }
      mma_commit(done);  // arrives once every MMA issued above has completed
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else if (warp < 6) {
    // --------------------------------------------------- scale-byte writers
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t G = 0;
    bool ok = true;
    // the bytes of the next group are loaded while the current one waits
    int64_t w = blockIdx.x;
    int gi = 0;
    auto load = [&](int64_t ww, int gg, uint4& va, uint4& vb0, uint4& vb1) {
      int tm, tp;
      tile_coords(P, ww, tm, tp);
      if constexpr (FUSE) {
        // the group's blocks of A are packed in this launch (a wait that
        // gives up sets *abort, which ends this warp's loop below)
        poll_packed(P.ready + (size_t)tm * nkb, 4 * gg, nkb, min(4, nkb - 4 * gg), abort);
        va = __ldcg(reinterpret_cast<const uint4*>(P.sfa + sf_index(tm, ngroups, 4 * gg, 0)) +
                    lane);
      } else {
        va = __ldg(reinterpret_cast<const uint4*>(P.sfa + sf_index(tm, ngroups, 4 * gg, 0)) +
                   lane);
      }
      vb0 = __ldg(reinterpret_cast<const uint4*>(P.sfb + sf_index(2 * tp, ngroups, 4 * gg, 0)) +
                  lane);
      if (2 * tp + 1 < P.tiles_n)
        vb1 = __ldg(
            reinterpret_cast<const uint4*>(P.sfb + sf_index(2 * tp + 1, ngroups, 4 * gg, 0)) +
            lane);
      else
        vb1 = vb0;  // no second half: its columns are not read
    };
    uint4 va, vb0, vb1;
    if (w < P.ntiles) load(w, 0, va, vb0, vb1);
    while (ok && w < P.ntiles) {
      int64_t w2 = w;
      int g2 = gi + 1;
      if (g2 == ngroups) {
        g2 = 0;
        w2 += gridDim.x;
      }
      uint4 na = va, nb0 = vb0, nb1 = vb1;
      // unfused: the next group's bytes are in flight during the wait below;
      // fused, they are loaded after this group is written (its blocks may
      // still be packing)
      if (!FUSE && w2 < P.ntiles) load(w2, g2, na, nb0, nb1);
      const uint32_t slot = G % NG;
      if (G >= (uint32_t)NG && !warp_wait(&sfe[slot], ((G / NG) - 1) & 1, abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t ra[4] = {va.x, va.y, va.z, va.w};
      const uint32_t r0[4] = {vb0.x, vb0.y, vb0.z, vb0.w};
      const uint32_t r1[4] = {vb1.x, vb1.y, vb1.z, vb1.w};
      tmem_st4(tl + COL_SF + slot * 12, ra);
      tmem_st4(tl + COL_SF + slot * 12 + 4, r0);
      tmem_st4(tl + COL_SF + slot * 12 + 8, r1);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&sff[slot]);
      if (FUSE && w2 < P.ntiles) load(w2, g2, na, nb0, nb1);
      ++G;
      w = w2;
      gi = g2;
      va = na;
      vb0 = nb0;
      vb1 = nb1;
    }
  } else if (!FUSE || warp < kThreads / 32) {
    // ------------------------------------------------------------- epilogue
    const int ew = warp - 6;
    const int q = warp & 3;                 // tensor-memory lane quadrant of this warp
    const int h = ew >> 2;                  // 128-column half of the tile
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)h * TILE;
    uint32_t t = 0;
    bool live = true;  // after a wait gave up, tiles are walked without work so
                       // that every epilogue warp still meets each named barrier
    for (int64_t w = blockIdx.x; w < P.ntiles; w += gridDim.x, ++t) {
      int tm, tp;
      tile_coords(P, w, tm, tp);
      int64_t* cc = colC + (t & 1) * 2 * TILE;
      {
        const int64_t n = (int64_t)tp * 2 * TILE + etid;   // 256 columns, one per thread
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      named_bar_sync(1, kEpiThreads);
      if (!live) continue;
      const int64_t m = (int64_t)tm * TILE + row;
      const int64_t rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
      if (!warp_wait(accf, t & 1, abort)) {
        live = false;
        continue;
      }
      tc_fence_after();
      // two passes of 64 columns; the accumulator is released after the last load
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        uint32_t v[4][16];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(tl + pass * 64 + c * 16, v[c]);
        tmem_wait_ld();
        if (pass == 1) {
          tc_fence_before();
          mbar_arrive(acce);  // the accumulator may take the next tile
        }
        if (rc >= 0) {
          float* Cr = P.C + rc;
#pragma unroll
          for (int i = 0; i < 64; ++i) {
            const int64_t ci = cc[h * TILE + pass * 64 + i];
            if (ci < 0) continue;
            float x = P.alpha * __uint_as_float(v[i / 16][i % 16]);
            if (P.beta != 0.0f) x = fmaf(P.beta, Cr[ci], x);
            Cr[ci] = x;
          }
        }
      }
    }
  } else {
    // ---------------------------------------------------------- pack warps
    if constexpr (FUSE) pack_warps<Cf>(P, smem, pbar);
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
// CTA pairs (tile configuration 2): 256 x 256 output tiles shared by two SMs
// (cluster of two, tcgen05.mma.cta_group::2, M = 256, N = 256, K = 32).  Each
// CTA holds its own 128-row tile of A and its own 128-column tile of B: per
// SM and K block 32 KB of operands for 128 x 256 outputs, against 48 KB on
// the one-CTA 128 x 256 tile.  Each CTA's half of the MMA reads the scale
// cells in its own tensor memory (A's for its own rows, B's for all 256
// columns, in the layout above), so both CTAs' scale writers fill the same
// 12-column groups from their own tiles and arrive on the first CTA's sff
// barrier.  The loads of both CTAs (tiled TMA, the packed blocks viewed as
// rows of 2 KB) complete on the first CTA's full barrier; the MMA thread's
// commits arrive on both CTAs' barriers; both epilogues arrive on the first
// CTA's acce barrier.  A stage holds two K blocks (64 KB), three stages.
// ---------------------------------------------------------------------------
constexpr int BPS_P = 1;  // K blocks per stage
struct CfgP8 {
  static constexpr uint32_t STAGE = BPS_P * 2 * CHUNK;     // A blocks, then B blocks
  static constexpr int S = (int)((192u * 1024u) / STAGE);
  static constexpr uint32_t OFF_COLC = S * STAGE;          // int64 colC[2][256]
  static constexpr uint32_t OFF_BAR = OFF_COLC + 2 * 2 * TILE * 8;
  static constexpr uint32_t NBAR = 2 * S + 2 + 2 * NG + 1;
  static constexpr uint32_t OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr uint32_t BYTES = OFF_MISC + 16 + 1024;  // + alignment slack
};

// Pair tile w: 128-row tiles 2 tmp, 2 tmp + 1 of A; 128-column tiles 2 tp,
// 2 tp + 1 of B.
__device__ __forceinline__ void pair_coords(const GemmFp8& P, int64_t w, int& tmp, int& tp) {
  const int mp = (P.tiles_m + 1) / 2;
  if (P.raster) {
    tp = (int)(w % P.tiles_p);
    tmp = (int)(w / P.tiles_p);
  } else {
    tmp = (int)(w % mp);
    tp = (int)(w / mp);
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_gemm_fp8p(const __grid_constant__ GemmFp8 P) {
  using Cf = CfgP8;
  constexpr int S = Cf::S;
  extern __shared__ uint8_t fp8p_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(fp8p_raw) + 1023) & ~(uintptr_t)1023);
  int64_t* colC = reinterpret_cast<int64_t*>(smem + Cf::OFF_COLC);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cf::OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* accf = bars + 2 * S;
  uint64_t* acce = accf + 1;
  uint64_t* sff = acce + 1;
  uint64_t* sfe = sff + NG;
  uint64_t* done = sfe + NG;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + Cf::OFF_MISC);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + Cf::OFF_MISC + 4);
  const uint32_t rank = cluster_ctarank();
  const bool lead = rank == 0;
  const int64_t pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 2 * kEpiThreads);  // both CTAs' epilogue threads
    for (int i = 0; i < NG; ++i) {
      mbar_init(&sff[i], 2 * 128);     // both CTAs' scale writers
      mbar_init(&sfe[i], 1);
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
  const int nkb = P.nkb, ngroups = P.ngroups;
  // arrive on the first CTA's barrier: every thread of a warp (count 1 each)
  auto arrive_lead = [&](uint64_t* bar) {
    if (lead) {
      mbar_arrive(bar);
    } else {
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(bar, 0, 32);
    }
  };

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      uint32_t g = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < P.ntiles; w += npairs) {
        int tmp, tp;
        pair_coords(P, w, tmp, tp);
        const int tm0 = 2 * tmp, tn0 = 2 * tp;
        const int tm = tm0 + (int)rank, tn = tn0 + (int)rank;
        const bool va = tm < P.tiles_m, vb = tn < P.tiles_n;  // else: outputs the pair discards
        const uint32_t pair_block = (tm0 < P.tiles_m ? CHUNK : 0u) +
                                    (tm0 + 1 < P.tiles_m ? CHUNK : 0u) +
                                    (tn0 < P.tiles_n ? CHUNK : 0u) +
                                    (tn0 + 1 < P.tiles_n ? CHUNK : 0u);
        for (int kb = 0; kb < nkb; kb += BPS_P, ++g) {
          const int s = (int)(g % S);
          if (g >= (uint32_t)S && !mbar_wait(&empty[s], ((g / S) - 1) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          const int nb = min(BPS_P, nkb - kb);
          const uint32_t dst = sbase + (uint32_t)s * Cf::STAGE;
          if (lead) mbar_arrive_expect_tx(&full[s], (uint32_t)nb * pair_block);
          const uint32_t mb = mapa_shared(smem_u32(&full[s]), 0);
          for (int bi = 0; bi < nb; ++bi) {
            if (va)
              tma_load_2d_pair(dst + bi * CHUNK, &P.tma_qa, 0,
                               (int32_t)(((int64_t)tm * nkb + kb + bi) * (CHUNK / 2048)), mb);
            if (vb)
              tma_load_2d_pair(dst + (BPS_P + bi) * CHUNK, &P.tma_qb, 0,
                               (int32_t)(((int64_t)tn * nkb + kb + bi) * (CHUNK / 2048)), mb);
          }
        }
      }
      // the copies still in flight (at most the last S stages) land before exit
      volatile int never = 0;
      for (uint32_t i = g > (uint32_t)S ? g - S : 0; i < g; ++i)
        mbar_wait(&empty[i % S], (i / S) & 1, &never, kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0 && lead) {
      // ------------------------------------------- MMA issue (first CTA)
      constexpr uint32_t LBO = (TILE / 8) * 128;  // next 16-byte K chunk
      uint32_t g = 0, G = 0, t = 0;
      bool ok = true;
      for (int64_t w = pair; ok && w < P.ntiles; w += npairs, ++t) {
        // the accumulator is free once both epilogues have read the previous tile
        if (t >= 1 && !mbar_wait(acce, (t - 1) & 1, abort, kTimeoutNs)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; ok && kb < nkb; kb += BPS_P, ++g) {
          const int s = (int)(g % S);
          if (!mbar_wait(&full[s], (g / S) & 1, abort, kTimeoutNs)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int nb = min(BPS_P, nkb - kb);
          for (int bi = 0; bi < nb; ++bi) {
            const int k = kb + bi;
            const uint32_t slot = G % NG;
            if ((k & 3) == 0) {  // both CTAs wrote the group's scale columns
              if (!mbar_wait(&sff[slot], (G / NG) & 1, abort, kTimeoutNs)) {
                ok = false;
                break;
              }
              tc_fence_after();
            }
            const uint32_t sa = sbase + (uint32_t)s * Cf::STAGE + bi * CHUNK;
            const uint32_t sb = sbase + (uint32_t)s * Cf::STAGE + (BPS_P + bi) * CHUNK;
            const uint32_t id = (uint32_t)(k & 3);
            const uint32_t idesc = idesc_mx_e4m3(2 * TILE, 2 * TILE, id, id);
            const uint32_t tsf = tmem + COL_SF + slot * 12;
#pragma unroll
            for (int kk = 0; kk < KB / 32; ++kk)
              mma_mx_e4m3_pair(tmem, smem_desc(sa + kk * 2 * LBO, LBO, 128),
                               smem_desc(sb + kk * 2 * LBO, LBO, 128), idesc, tsf, tsf + 4,
                               (k > 0 || kk > 0) ? 1u : 0u);
            if ((k & 3) == 3 || k == nkb - 1) {
              mma_commit_pair(&sfe[slot], 3);  // both CTAs may rewrite the group's columns
              ++G;
            }
          }
          if (!ok) break;
          mma_commit_pair(&empty[s], 3);  // both CTAs may refill this stage
        }
        if (!ok) break;
        mma_commit_pair(accf, 3);  // both CTAs' epilogues may read the accumulator
      }
      mma_commit_pair(done, 1);  // arrives once every MMA issued above has completed
      volatile int never = 0;
      mbar_wait(done, 0, &never, kTimeoutNs);
    }
  } else if (warp < 6) {
    // --------------------------------------------------- scale-byte writers
    // A's cells for this CTA's own 128 rows, B's for both column tiles
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t G = 0;
    int64_t w = pair;
    int gi = 0;
    auto load = [&](int64_t ww, int gg, uint4& va, uint4& vb0, uint4& vb1) {
      int tmp, tp;
      pair_coords(P, ww, tmp, tp);
      const int tm = min(2 * tmp + (int)rank, P.tiles_m - 1);  // a missing tile: rows discarded
      va = __ldg(reinterpret_cast<const uint4*>(P.sfa + sf_index(tm, ngroups, 4 * gg, 0)) + lane);
      vb0 = __ldg(reinterpret_cast<const uint4*>(P.sfb + sf_index(2 * tp, ngroups, 4 * gg, 0)) +
                  lane);
      if (2 * tp + 1 < P.tiles_n)
        vb1 = __ldg(
            reinterpret_cast<const uint4*>(P.sfb + sf_index(2 * tp + 1, ngroups, 4 * gg, 0)) +
            lane);
      else
        vb1 = vb0;  // no second column tile: its columns are discarded
    };
    uint4 va, vb0, vb1;
    if (w < P.ntiles) load(w, 0, va, vb0, vb1);
    while (w < P.ntiles) {
      int64_t w2 = w;
      int g2 = gi + 1;
      if (g2 == ngroups) {
        g2 = 0;
        w2 += npairs;
      }
      uint4 na = va, nb0 = vb0, nb1 = vb1;
      if (w2 < P.ntiles) load(w2, g2, na, nb0, nb1);
      const uint32_t slot = G % NG;
      if (G >= (uint32_t)NG && !warp_wait(&sfe[slot], ((G / NG) - 1) & 1, abort)) break;
      tc_fence_after();
      const uint32_t ra[4] = {va.x, va.y, va.z, va.w};
      const uint32_t r0[4] = {vb0.x, vb0.y, vb0.z, vb0.w};
      const uint32_t r1[4] = {vb1.x, vb1.y, vb1.z, vb1.w};
      tmem_st4(tl + COL_SF + slot * 12, ra);
      tmem_st4(tl + COL_SF + slot * 12 + 4, r0);
      tmem_st4(tl + COL_SF + slot * 12 + 8, r1);
      tmem_wait_st();
      tc_fence_before();
      arrive_lead(&sff[slot]);
      ++G;
      w = w2;
      gi = g2;
      va = na;
      vb0 = nb0;
      vb1 = nb1;
    }
  } else {
    // ------------------------------------------------------------- epilogue
    const int ew = warp - 6;
    const int q = warp & 3;                 // tensor-memory lane quadrant of this warp
    const int h = ew >> 2;                  // 128-column half of the tile
    const int row = q * 32 + lane;
    const int etid = ew * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)h * TILE;
    uint32_t t = 0;
    bool live = true;  // after a wait gave up, tiles are walked without work so
                       // that every epilogue warp still meets each named barrier
    for (int64_t w = pair; w < P.ntiles; w += npairs, ++t) {
      int tmp, tp;
      pair_coords(P, w, tmp, tp);
      int64_t* cc = colC + (t & 1) * 2 * TILE;
      {
        const int64_t n = (int64_t)tp * 2 * TILE + etid;  // 256 columns, one per thread
        cc[etid] = n < P.N ? goff(P.gn, 2, (uint32_t)n) : -1;
      }
      named_bar_sync(1, kEpiThreads);
      if (!live) continue;
      const int64_t m = (int64_t)(2 * tmp + (int)rank) * TILE + row;
      const int64_t rc = m < P.M ? goff(P.gm, 2, (uint32_t)m) : -1;
      if (!warp_wait(accf, t & 1, abort)) {
        live = false;
        continue;
      }
      tc_fence_after();
      // two passes of 64 columns; the accumulator is released after the last load
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        uint32_t v[4][16];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(tl + pass * 64 + c * 16, v[c]);
        tmem_wait_ld();
        if (pass == 1) {
          tc_fence_before();
          arrive_lead(acce);  // the accumulator may take the next tile
        }
        if (rc >= 0) {
          float* Cr = P.C + rc;
#pragma unroll
          for (int i = 0; i < 64; ++i) {
            const int64_t ci = cc[h * TILE + pass * 64 + i];
            if (ci < 0) continue;
            float x = P.alpha * __uint_as_float(v[i / 16][i % 16]);
            if (P.beta != 0.0f) x = fmaf(P.beta, Cr[ci], x);
            Cr[ci] = x;
          }
        }
      }
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

// Shared memory of the kernels, set once per process (first call).
int set_smem() {
  static int bytes = 0;
  if (bytes == 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
      return -1;
    if (optin < (int)Cfg<false>::BYTES || optin < (int)Cfg<true>::BYTES ||
        optin < (int)CfgP8::BYTES)
      return -2;
    if (cudaFuncSetAttribute(k_fp8_pack, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPackSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_fp8<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<false>::BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_gemm_fp8<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg<true>::BYTES) != cudaSuccess)
      return -1;
    bytes = 1;
  }
  return bytes;
}

// cuTensorMapEncodeTiled through the runtime's driver entry-point query.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
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

// Packed blocks as a 2-D tensor of 8-byte elements in rows of 2 KB; a box is
// one 16 KB block (8 rows).
bool packed_map(CUtensorMap* m, const void* base, size_t bytes) {
  EncodeTiledFn fn = encoder();
  if (!fn || bytes == 0 || bytes % 2048 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  cuuint64_t dims[2] = {256, (cuuint64_t)(bytes / 2048)};
  cuuint64_t strides[1] = {2048};
  cuuint32_t box[2] = {256, CHUNK / 2048};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pairs that run at once (cluster occupancy of k_gemm_fp8p), looked up once.
int max_pairs() {
  static int n = -1;
  if (n < 0) {
    n = 0;
    if (cudaFuncSetAttribute(k_gemm_fp8p, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CfgP8::BYTES) != cudaSuccess)
      return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = CfgP8::BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_gemm_fp8p, &cfg) == cudaSuccess && c > 0) n = c;
  }
  return n;
}

// A's FP32 elements as the 2-D tensor [K][M] (M contiguous, K rows `ldk`
// elements apart); boxes of 64 rows of A by 128 K, zero outside A.
bool first_operand_map(CUtensorMap* m, const GemmArgs& a) {
  EncodeTiledFn fn = encoder();
  if (!fn || (reinterpret_cast<uintptr_t>(a.A) & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)a.M, (cuuint64_t)a.K};
  cuuint64_t strides[1] = {(cuuint64_t)a.gk.st[0][0] * 4};
  cuuint32_t box[2] = {(cuuint32_t)HROWS, (cuuint32_t)KB};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(a.A), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace fp8

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Fp8Layout fp8_layout(const GemmArgs& a) {
  Fp8Layout L;
  std::memset(&L, 0, sizeof(L));
  L.tiles_m = (a.M + fp8::TILE - 1) / fp8::TILE;
  L.tiles_n = (a.N + fp8::TILE - 1) / fp8::TILE;
  L.nkb = (a.K + fp8::KB - 1) / fp8::KB;
  L.off_qa = 0;
  L.off_qb = align256((size_t)L.tiles_m * L.nkb * fp8::CHUNK);
  L.ngroups = (L.nkb + 3) / 4;
  L.off_sa = L.off_qb + align256((size_t)L.tiles_n * L.nkb * fp8::CHUNK);
  L.off_sb = L.off_sa + align256((size_t)L.tiles_m * L.ngroups * 512);
  L.off_ready = L.off_sb + align256((size_t)L.tiles_n * L.ngroups * 512);
  L.ready_bytes = 16 + (size_t)L.tiles_m * L.nkb * 4;
  L.bytes = L.off_ready + align256(L.ready_bytes);
  return L;
}

// The first operand can be packed inside the GEMM launch (tile configuration
// 1) when it is a plain matrix with M contiguous: one M label of stride 1, one
// K label whose stride is a multiple of 16 bytes, no batch labels.
bool fp8_fusable(const GemmArgs& a) {
  if (a.a_contig != CONTIG_MN || a.gm.n != 1 || a.gk.n != 1 || a.gb.n != 0 || a.nbatch != 1)
    return false;
  const int64_t ldk = a.gk.st[0][0];
  if (a.gm.st[0][0] != 1 || ldk <= 0 || ldk % 4 != 0 || ldk >= (1ll << 37)) return false;
  if (a.M <= 0 || a.K <= 0 || a.M >= (1ll << 31) || a.K >= (1ll << 31)) return false;
  const Fp8Layout L = fp8_layout(a);
  return L.tiles_m * L.nkb * 2 < (1ll << 30);  // unit ids (claims run a few batches past) fit 31 bits
}

tc_status launch_gemm_fp8(const GemmArgs& a, int tile, void* ws, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Fp8Layout L = fp8_layout(a);
  if (L.tiles_m == 0 || L.tiles_n == 0 || L.nkb == 0) return TC_OK;
  const int sm = fp8::set_smem();
  if (sm == -2) return TC_ERR_UNSUPPORTED;
  const int sms = fp8::num_sms();
  if (sm < 0 || sms <= 0) return TC_ERR_CUDA;
  uint8_t* w = static_cast<uint8_t*>(ws);

  fp8::GemmFp8 g;
  std::memset(&g, 0, sizeof(g));
  // tile 1: the GEMM packs A itself (B is packed first, by k_fp8_pack);
  // an operand the tensor map cannot describe (misaligned) takes tile 0
  const bool fuse = tile == 1 && fp8_fusable(a) && fp8::first_operand_map(&g.tma_a, a);

  fp8::PackArgs pk;
  std::memset(&pk, 0, sizeof(pk));
  pk.gr[0] = a.gm;
  pk.gr[1] = a.gn;
  pk.gk = a.gk;
  pk.in[0] = static_cast<const float*>(a.A);
  pk.in[1] = static_cast<const float*>(a.B);
  pk.q[0] = w + L.off_qa;
  pk.q[1] = w + L.off_qb;
  pk.sf[0] = w + L.off_sa;
  pk.sf[1] = w + L.off_sb;
  pk.rows[0] = a.M;
  pk.rows[1] = a.N;
  pk.K = a.K;
  pk.tiles[0] = (int32_t)L.tiles_m;
  pk.tiles[1] = (int32_t)L.tiles_n;
  pk.nkb = (int32_t)L.nkb;
  pk.ngroups = (int32_t)L.ngroups;
  pk.nblocks0 = fuse ? 0 : L.tiles_m * L.nkb;  // 0: operand B only
  pk.rows_fast[0] = a.a_contig == CONTIG_MN;
  pk.rows_fast[1] = a.b_contig == CONTIG_MN;
  const int64_t nblocks = pk.nblocks0 + L.tiles_n * L.nkb;
  if (nblocks > 0x7fffffffll) return TC_ERR_UNSUPPORTED;
  fp8::k_fp8_pack<<<(unsigned)nblocks, fp8::kPackThreads, fp8::kPackSmem, s>>>(pk);
  if (cudaGetLastError() != cudaSuccess) return TC_ERR_CUDA;

  g.gm = a.gm;
  g.gn = a.gn;
  g.qa = pk.q[0];
  g.qb = pk.q[1];
  g.sfa = pk.sf[0];
  g.sfb = pk.sf[1];
  g.C = static_cast<float*>(a.C);
  g.M = a.M;
  g.N = a.N;
  g.tiles_p = (int32_t)((L.tiles_n + 1) / 2);
  g.ntiles = L.tiles_m * g.tiles_p;
  g.alpha = (float)a.alpha;
  g.beta = (float)a.beta;
  g.tiles_m = (int32_t)L.tiles_m;
  g.tiles_n = (int32_t)L.tiles_n;
  g.nkb = (int32_t)L.nkb;
  g.ngroups = (int32_t)L.ngroups;
  g.raster = a.raster;
  if (tile == 2) {
    // CTA pairs over 256 x 256 tiles, as many pairs as run at once
    const int pairs_max = fp8::max_pairs();
    if (pairs_max <= 0) return TC_ERR_CUDA;
    g.ntiles = ((L.tiles_m + 1) / 2) * g.tiles_p;
    if (!fp8::packed_map(&g.tma_qa, g.qa, (size_t)L.tiles_m * L.nkb * fp8::CHUNK) ||
        !fp8::packed_map(&g.tma_qb, g.qb, (size_t)L.tiles_n * L.nkb * fp8::CHUNK))
      return TC_ERR_CUDA;
    const int pairs = (int)std::min<int64_t>(g.ntiles, pairs_max);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(fp8::kThreads, 1, 1);
    cfg.dynamicSmemBytes = fp8::CfgP8::BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fp8::k_gemm_fp8p, g) == cudaSuccess ? TC_OK : TC_ERR_CUDA;
  }
  const int grid = (int)std::min<int64_t>(g.ntiles, sms);
  if (!fuse) {
    fp8::k_gemm_fp8<false><<<grid, fp8::Cfg<false>::THREADS, fp8::Cfg<false>::BYTES, s>>>(g);
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
  }
  // pack units in groups of the tiles of A one wave of GEMM tiles covers
  // (all of them when m-tiles run fastest)
  g.next_unit = reinterpret_cast<uint32_t*>(w + L.off_ready);
  g.ready = reinterpret_cast<uint32_t*>(w + L.off_ready + 16);
  g.units = L.tiles_m * L.nkb * 2;
  g.group_tiles = g.raster ? (int32_t)std::min<int64_t>(
                                 L.tiles_m, (grid + g.tiles_p - 1) / g.tiles_p + 1)
                           : (int32_t)L.tiles_m;
  // the pack counts start at zero, and so do A's scale-cell records (the pack
  // warps OR their bytes into them)
  if (cudaMemsetAsync(w + L.off_ready, 0, L.ready_bytes, s) != cudaSuccess ||
      cudaMemsetAsync(w + L.off_sa, 0, (size_t)L.tiles_m * L.ngroups * 512, s) != cudaSuccess)
    return TC_ERR_CUDA;
  fp8::k_gemm_fp8<true><<<grid, fp8::Cfg<true>::THREADS, fp8::Cfg<true>::BYTES, s>>>(g);
  return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status tc_fp8_read_status(int* h, void* stream) {
  return read_clear_status(h, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TC_OK
                                                                                : TC_ERR_CUDA;
}

}  // namespace tc
