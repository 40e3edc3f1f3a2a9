// tc_internal.h -- plan structures shared by the host planner and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <vector_types.h>  // float2

#include "tc.h"

namespace tc {

constexpr int kGroupMax = TC_MAX_ORDER;

// A multi-index group: labels enumerated column-major (first label fastest).
// st[0], st[1], st[2] are the element strides of each label in the kernel's
// first operand ("A"), second operand ("B") and in C; 0 where a label is absent.
struct Group {
  int32_t n;
  int32_t pad_;
  int64_t ext[kGroupMax];
  int64_t st[3][kGroupMax];
  // Division by ext[i] as a multiply and a shift (Granlund and Montgomery,
  // "Division by invariant integers using multiplication", 1994, with a
  // 31-bit dividend): for idx < 2^31, idx / ext[i] = (idx * dmul[i]) >> dsh[i].
  // dmul[i] == 0: divide (the group has 2^31 or more elements).
  uint32_t dmul[kGroupMax];
  uint32_t dsh[kGroupMax];
};


enum Kernel : int32_t {
  K_NONE = 0,
  K_GEMM_SIMT = 1,
  K_GEMM_TC = 2,
  K_GEMV = 3,
  K_DOT = 4,
  K_GEMM_FP8 = 5,
  K_GER = 6
};

// Operand contiguity (how the loader can coalesce):
//   0 = generic gather, 1 = contiguous along the M/N group's first label,
//   2 = contiguous along the K group's first label.
enum Contig : int32_t { CONTIG_NONE = 0, CONTIG_MN = 1, CONTIG_K = 2 };

// Kernel arguments of every GEMM-like kernel (passed by value).
//   C[m, n, b] = alpha * sum_k A[m, k, b] * B[k, n, b] + beta * C[m, n, b]
// with m, n, k, b multi-indices of the groups gm, gn, gk, gb.
struct GemmArgs {
  Group gm, gn, gk, gb;
  int64_t M, N, K, nbatch;
  const void* A;
  const void* B;
  void* C;
  double alpha, beta;
  int32_t a_contig, b_contig;  // Contig of A along (M | K), of B along (N | K)
  int32_t c_contig_m;          // 1 when C's stride along the first M label is 1
  int32_t math;                // tc_math
  int32_t raster;              // tensor-core GEMM: 1 = n-tiles fastest in launch order
  int32_t chunk_kb;            // tensor-core GEMM: K blocks per FP32 accumulation chunk
  int32_t swapped;             // batched items: the kernel's first operand is B
  int32_t ksplit;              // FP64 CUDA-core GEMM: K ranges per tile (1: tiles write C)
  void* ws;                    // workspace (DOT partials; split-K partial tiles)
  int64_t ws_elems;
};

// Dense permutation (COPY): out[col-major over g, in g's label order] =
// in[sum idx * st[0]].  st[2] holds the output strides.
struct PermArgs {
  Group g;
  int64_t total;
  const void* in;
  void* out;
};

struct Plan {
  // decisions reported through tc_plan_info
  tc_plan_info info;
  tc_dtype dtype;
  tc_math math;
  int32_t mapping;
  int32_t kernel;
  int32_t tile;
  bool swapped;
  // GEMM view (operands already swapped when `swapped`)
  GemmArgs args;
  // COPY+GEMM: permutation of one operand into workspace (0 none, 1 X, 2 Y)
  int copy_which;
  PermArgs perm;
  int64_t copy_elems;
  // empty output / empty contraction shortcuts
  bool empty_out;
  bool empty_k;
  int64_t c_elems_span;  // C's element span (for beta-only scaling)
  Group gc;              // C's own labels (for beta-only scaling)
  size_t workspace;
  float features[TC_SELECTOR_FEATURES];  // descriptor features (selector input)
  tc_layout_advice advice;               // storage-layout advice (Sec. 3.3)
};

size_t elem_size(tc_dtype dt);

// Host forward pass of a loaded selector: predicted log2 runtime of each of
// its candidates (returns false when no selector applies to dtype/math or a
// feature lies outside the training range).
bool selector_predict(const float* features, tc_dtype dtype, tc_math math, int32_t* cand,
                      float* pred, int32_t* n_cand);

// Kernel launchers (k_simt.cu); `stream` is a cudaStream_t.
tc_status launch_gemm_simt(const GemmArgs& a, tc_dtype dt, int tile, void* stream);
// FP64 CUDA-core GEMM split-K: K ranges per tile for tile configuration
// `tile`, and the bytes of their partial tiles (part of the workspace).
int simt_ksplit(const GemmArgs& a, tc_dtype dt, int tile);
size_t simt_part_bytes(const GemmArgs& a, tc_dtype dt, int tile);
tc_status launch_gemv(const GemmArgs& a, tc_dtype dt, int tile, void* stream);
tc_status launch_dot(const GemmArgs& a, tc_dtype dt, int tile, void* stream);
tc_status launch_ger(const GemmArgs& a, tc_dtype dt, void* stream);
tc_status launch_perm(const PermArgs& a, tc_dtype dt, void* stream);
tc_status launch_scale(const Group& gc, void* C, double beta, tc_dtype dt, int64_t total,
                       void* stream);
tc_status launch_gemm_tc(const GemmArgs& a, int math, void* stream);
int dot_partials(const GemmArgs& a, int tile);
// The scalar (Class 1) DOT: one FP64 partial per CTA into part[0 ..
// dot_partials()), then their ordered sum, alpha and beta.
tc_status launch_dot_scalar(const GemmArgs& a, tc_dtype dt, double* part, void* stream);
int num_tiles_tc();
// Enqueue a read-and-clear of the tensor-core kernels' timeout flag into *h.
tc_status tc_gemm_read_status(int* h, void* stream);
int tc_chunk_kb(int math, int tile);

// FP8 form: workspace layout of the packed operands (byte offsets).
struct Fp8Layout {
  int64_t tiles_m, tiles_n, nkb, ngroups;
  size_t off_qa, off_qb, off_sa, off_sb;
  size_t off_ready, ready_bytes;  // in-kernel packing: claim counter, per-block counts
  size_t bytes;
};
Fp8Layout fp8_layout(const GemmArgs& a);
// Tile configurations of the FP8 GEMM: 0 packs both operands in a pass of
// their own first, then multiplies on 128 x 256 tiles; 1 packs the second
// operand first and the first operand inside the GEMM launch, overlapped with
// the multiplications (needs fp8_fusable; slower on GB300 for the shapes
// measured: the pack warps' loads and the GEMM's operand copies share each
// SM's bandwidth); 2 (the default when M and N both span two 128-row tiles)
// packs as 0 and multiplies on CTA pairs over 256 x 256 tiles.
constexpr int kFp8Tiles = 3;
bool fp8_fusable(const GemmArgs& a);
// Pack the operands into `ws` (16-byte aligned) and run the FP8 GEMM.
tc_status launch_gemm_fp8(const GemmArgs& a, int tile, void* ws, void* stream);
tc_status tc_fp8_read_status(int* h, void* stream);

// Split-BF16 forms with packed operands (tile configuration kTilePacked of
// the tensor-core GEMM): workspace layout and launcher.
constexpr int kTilePacked = 3;
// Packed operands on 128 x 256 tiles with one FP32 accumulator per tile (the
// BF16, FP16 and BF16x3 forms).
constexpr int kTilePackedWide = 4;
// Packed operands on 256 x 256 tiles shared by a pair of SMs (a cluster of
// two CTAs on tcgen05.mma.cta_group::2), same arithmetic as tile 4.
constexpr int kTilePackedPair = 5;
struct PkLayout {
  int64_t tiles_m, tiles_n, nkb;
  size_t off_qa, off_qb, bytes;
};
PkLayout pk_layout(const GemmArgs& a, int math);
// K ranges of a packed GEMM (split-K when there are fewer tiles than SMs),
// and the bytes of its partial sums (part of the plan's workspace).
int pk_ksplit(const GemmArgs& a);
int pk_ksplit_w(const GemmArgs& a);
int pk_ksplit_p(const GemmArgs& a);
int pk_tail_split_p(const GemmArgs& a, int64_t* nfull);
int pk_ksplit_p6(const GemmArgs& a);
size_t pk_part_bytes(const GemmArgs& a, int tile);
// 32-K blocks per ring stage of the packed GEMM for a math form: every
// accumulation chunk must hold a multiple of them.
int pk_stage_blocks(int math);
tc_status launch_gemm_tc_packed(const GemmArgs& a, int math, tc_dtype dt, int tile, void* ws,
                                void* stream);
tc_status tc_pk_read_status(int* h, void* stream);

// One GEMM on packed operands as the packed kernel sees it.
struct PkItem {
  Group gm, gn;          // C offsets (slot 2) of the GEMM's rows and columns
  const uint8_t* qa;     // packed terms of the first and second operand
  const uint8_t* qb;
  int64_t M, N;
  int32_t tiles_m, tiles_n, nkb, chunk_kb, raster;
  int32_t ksplit;        // K ranges per tile (1: the tile writes C)
  float2* part;          // ksplit > 1: compensated partial sums [split][tile][col][row]
  // CTA pairs: the tiles of a last, partial round of work entries split K
  // (tsplit > 1): entries [0, nfull) are whole tiles, then each tail tile
  // t >= nfull is tsplit entries whose partial sums are
  // part[split][t - nfull][quarter][col][row]
  int64_t nfull;
  int32_t tsplit;
};
// Tensor-core route of a batch on packed operands (device tables owned by
// the batch): the pack entries (item, operand, row tile, 128-K chunk; int32
// x 4) and the GEMM's (item, tile) entries (int32 x 2).
struct PkBatch {
  const GemmArgs* items;
  const PkItem* pk;
  const int32_t* pack_work;
  int64_t n_pack;
  const int32_t* work;  // (item, tile, K range) per entry
  int64_t n_work;
  const int32_t* red;   // split-K reductions: (item, tile) per entry
  int64_t n_red;
};
tc_status launch_gemm_tc_packed_batch(const PkBatch& b, const void* const* A,
                                      const void* const* B, void* const* C, const double* alpha,
                                      const double* beta, int math, void* stream);
int num_tiles_simt(tc_dtype dt);
// Read and clear the peak probes' timeout flag into *h (k_peak.cu).
tc_status peak_read_status(int* h, void* stream);
int num_tiles_gemv();

}  // namespace tc
