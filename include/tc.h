/*
 * tc.h -- binary dense tensor contraction on one GB300 GPU (sm_103a).
 *
 * The operation (Sec. 2.1 "c_ij = sum_h a_ih b_hj", generalised to tensors of
 * any order in Sec. 2.3 and the Appendix): given tensors A and B whose indices
 * carry labels, every label present in both A and B is contracted (summed over
 * its range) and the remaining labels index the result,
 *
 *     C[free_A u free_B] = alpha * sum_{contracted} A * B  +  beta * C.
 *
 * Storage (Sec. 2.1 "stride", Sec. 2.4): each tensor is described by its
 * labels, extents and strides counted in elements; NULL strides mean
 * column-major (first index stride 1).  Any positive strides are accepted for
 * A and B; C's strides must not alias (no two index tuples may share an
 * element).
 *
 * The library sorts each contraction into the paper's classes by index
 * placement and strides (Sec. 3.2: Class 1 = DOT, Class 2 = GEMV, Class 3.1 =
 * COPY+GEMM, Class 3.2 = GEMM) and maps it onto its own CUDA kernels.  All
 * device buffers and streams belong to the caller; plans are host objects.
 *
 * Errors: every function returns a tc_status; nothing aborts.  Invalid input
 * is rejected before any launch.  Device-side waits are bounded: a wait that
 * runs out records TC_ERR_TIMEOUT in a device flag, reported by
 * tc_device_status().
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TC_MAX_ORDER 12   /* indices per tensor */

typedef enum {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,     /* null pointer, negative extent, order out of range */
  TC_ERR_LABEL = 2,           /* repeated label, label of C in neither operand,
                                 label of A/B in neither C nor the other operand */
  TC_ERR_EXTENT_MISMATCH = 3, /* a label has different extents in two tensors */
  TC_ERR_STRIDE = 4,          /* non-positive stride (extent > 1) or aliasing output */
  TC_ERR_UNSUPPORTED = 5,     /* dtype/math/mapping/tile combination */
  TC_ERR_WORKSPACE = 6,       /* workspace missing or smaller than tc_plan_info.workspace */
  TC_ERR_CUDA = 7,            /* a CUDA call failed */
  TC_ERR_TIMEOUT = 8,         /* a bounded device wait ran out */
  TC_ERR_NO_SELECTOR = 9      /* no selector weights loaded */
} tc_status;

/* Storage type of A, B and C (all three share it; Sec. 2.1 stores tensors of
 * one type).  The paper computes in FP64 (Sec. 4); the other types are for
 * callers whose tensors are FP32, BF16 or FP16 already.  Math forms each
 * storage type takes (else TC_ERR_UNSUPPORTED):
 *   TC_F64   TC_MATH_FP64
 *   TC_F32   TC_MATH_FP32, _BF16, _BF16X3, _BF16X6, _FP8, _FP16
 *   TC_BF16  TC_MATH_FP32 (CUDA cores), TC_MATH_BF16 (tensor cores)
 *   TC_F16   TC_MATH_FP32 (CUDA cores), TC_MATH_FP16 (tensor cores)
 * BF16 and FP16 elements are read exactly; results are computed in FP32 (FP64
 * where a kernel sums in FP64) and rounded to the storage type to nearest,
 * ties to even, when C is written. */
typedef enum { TC_F64 = 0, TC_F32 = 1, TC_BF16 = 2, TC_F16 = 3 } tc_dtype;

/* Arithmetic of the contraction.
 *   TC_MATH_FP64     FP64 inputs, FP64 multiply-add (the plain path; the paper
 *                    computes in double precision, Sec. 4).
 *   TC_MATH_FP32     FP32 multiply-add on the CUDA cores (FP32, BF16 or FP16
 *                    storage).
 *   TC_MATH_BF16     FP32 inputs rounded to BF16 (BF16 inputs as stored),
 *                    tensor-core products, FP32 accumulation.
 *   TC_MATH_BF16X3   FP32 inputs split into 2 BF16 terms; the 3 products of
 *                    order <= 1 on tensor cores.
 *   TC_MATH_BF16X6   FP32 inputs split into 3 BF16 terms; the 6 products of
 *                    order <= 2 on tensor cores (FP32-class accuracy).
 *   TC_MATH_FP8      FP32 inputs rounded to FP8-E4M3 with one power-of-two
 *                    scale per operand row and block of 128 consecutive
 *                    contracted elements (contracted indices enumerated in
 *                    ascending order of their strides in A, the first one
 *                    fastest; a row is one value of the operand's free
 *                    indices); the scale 2^e of a block is the smallest with
 *                    max |x| / 2^e <= 448, e >= -126.  Products on tensor
 *                    cores, each block summed in FP32 and scaled, blocks
 *                    added in FP32.  Class 3 contractions only, mapping AUTO,
 *                    RECIPE or FUSED_GEMM (one GEMM).  The paper has no
 *                    reduced-precision form; this one trades accuracy (about
 *                    2^-5 relative per product) for tensor-core throughput.
 *   TC_MATH_FP16     FP32 inputs rounded to IEEE binary16 (to nearest, ties to
 *                    even; magnitudes from 65520 on become infinite), FP16
 *                    inputs as stored; tensor-core products (exact in FP32),
 *                    FP32 accumulation.  Class 3 GEMM mappings run one GEMM on
 *                    packed operands (no batch labels); Class 1 and 2 and the
 *                    GER mapping compute on the CUDA cores in FP32. */
typedef enum {
  TC_MATH_FP64 = 0,
  TC_MATH_FP32 = 1,
  TC_MATH_BF16 = 2,
  TC_MATH_BF16X3 = 3,
  TC_MATH_BF16X6 = 4,
  TC_MATH_FP8 = 5,
  TC_MATH_FP16 = 6
} tc_math;

/* How the contraction is mapped onto kernels.
 *   TC_MAP_AUTO        the selector if weights are loaded, else TC_MAP_RECIPE.
 *   TC_MAP_RECIPE      the paper's class -> kernel family (Sec. 3.2 recipes):
 *                      Class 3 -> GEMM (fused loader, so Class 3.1 needs no copy),
 *                      Class 2 -> GEMV, Class 1 -> DOT.
 *   TC_MAP_SLICE_GEMM  the Class 3 recipe's slicing literally: the two stride-1
 *                      indices and one free index per operand stay unsliced, every
 *                      other free index becomes a batch of GEMMs, every other
 *                      contracted index is accumulated (Sec. 3.1 R1-R3, Sec. 3.2.3).
 *   TC_MAP_FUSED_GEMM  one GEMM: M = all free indices of A, N = all free
 *                      indices of B, K = all contracted indices, gathered by the
 *                      kernel's loader (no copy pass).
 *   TC_MAP_COPY_GEMM   explicit COPY+GEMM (Sec. 3.1 F1): the operand whose stride-1
 *                      index is sliced is first permuted into workspace.
 *   TC_MAP_GEMV        matrix-vector products (Sec. 3.2.2); for Class 3 one GEMV per
 *                      value of B's free indices (slicing (c) of Sec. 2.4).
 *   TC_MAP_DOT         one inner product per output element (Sec. 3.2.1, F3).
 *   TC_MAP_GER         rank-K update for tiny contracted ranges, the sum-of-GERs
 *                      slicing of Sec. 2.2 done in one pass: every output's K
 *                      products are summed in registers and C is written once;
 *                      K <= TC_GER_MAX_K (else TC_ERR_UNSUPPORTED).  Computes in
 *                      the storage precision (FP64, or FP32 for FP32 storage
 *                      whatever the math form; FP8 has only the fused mapping). */
typedef enum {
  TC_MAP_AUTO = 0,
  TC_MAP_RECIPE = 1,
  TC_MAP_SLICE_GEMM = 2,
  TC_MAP_FUSED_GEMM = 3,
  TC_MAP_COPY_GEMM = 4,
  TC_MAP_GEMV = 5,
  TC_MAP_DOT = 6,
  TC_MAP_GER = 7
} tc_mapping;
#define TC_GER_MAX_K 32

/* A tensor: `order` indices with labels (distinct int32 values), extents
 * (>= 0) and strides in elements (NULL = column-major).  The arrays are read
 * during tc_plan only. */
typedef struct {
  int32_t order;
  const int32_t* labels;
  const int64_t* extents;
  const int64_t* strides;
} tc_tensor_desc;

typedef struct tc_plan_s* tc_plan_t;

/* What tc_plan decided.  Slicing vectors (Sec. 2.4): bit i of slice_a is 1 when
 * index i of A is sliced (looped over) in the recipe's slicing; indices of
 * extent 1 are reported as sliced. */
typedef struct {
  int32_t cls;           /* 1, 2, 31 (Class 3.1) or 32 (Class 3.2) (Sec. 3.2) */
  int32_t p;             /* number of contracted indices of extent > 1 */
  int32_t delta_a;       /* Delta(A) = N(A) - p, indices of extent > 1 (Sec. 3.2) */
  int32_t delta_b;
  int32_t stride1_a;     /* label of A's stride-1 index, -1 if none */
  int32_t stride1_b;
  uint32_t slice_a;      /* recipe slicing vector s(A) */
  uint32_t slice_b;      /* recipe slicing vector s(B) */
  int32_t mapping;       /* tc_mapping in use (never AUTO or RECIPE) */
  int32_t kernel;        /* kernel family: 1 GEMM-SIMT, 2 GEMM-tcgen05, 3 GEMV, 4 DOT,
                            5 GEMM-tcgen05 FP8 (pack pass + GEMM), 6 GER */
  int32_t tile;          /* tile configuration index of that kernel */
  int32_t swapped;       /* 1 when the kernel's first operand is B */
  int64_t M, N, K, batch;   /* GEMM view after mode merging */
  double flops;          /* 2 * product of all extents */
  double min_bytes;      /* |A| + |B| + |C| (+|C| if beta may be non-zero) in bytes */
  size_t workspace;      /* bytes of device workspace tc_contract needs */
} tc_plan_info;

/* Build a plan (host only; no device work).  `mapping` forces a mapping
 * (TC_ERR_UNSUPPORTED if it cannot compute this contraction); `tile` forces a
 * tile configuration, -1 = default.  On success *out owns a new plan.
 * A label in A, B and C is a batch (Hadamard) label, beyond the paper's
 * definition: A, B and C are indexed by the same value, and the plan is one
 * contraction per value (the GEMM view's batch group).  The class and the
 * slicing vectors are those of one batch slice (batch labels count as sliced);
 * the FP8 form and the COPY+GEMM mapping do not take batch labels. */
tc_status tc_plan(tc_plan_t* out, const tc_tensor_desc* A, const tc_tensor_desc* B,
                  const tc_tensor_desc* C, tc_dtype dtype, tc_math math,
                  tc_mapping mapping, int32_t tile);

/* Copy the plan's decisions into *info. */
tc_status tc_plan_get_info(tc_plan_t plan, tc_plan_info* info);

/* Free a plan (NULL is allowed). */
tc_status tc_plan_destroy(tc_plan_t plan);

/* Storage-layout advice (the guideline of Sec. 3.3: store tensors so that no
 * stride-1 index is contracted).  For a Class 3.1 contraction, the operand to
 * re-store once (the smaller; B on a tie) and the storage order that gives it
 * a free stride-1 index (its largest free index first, then its other indices
 * in their present stride order, column-major in that order), which makes the
 * contraction Class 3.2; for any other class, operand 0 (keep the layouts).
 * The paper has no such report; it states the guideline. */
typedef struct {
  int32_t operand;                        /* 0 keep, 1 re-store A, 2 re-store B */
  int32_t order;                          /* entries of storage_order */
  int32_t storage_order[TC_MAX_ORDER];    /* index positions of that operand, fastest first */
  int32_t cls_after;                      /* class after re-storing (32), else the class */
  double copy_bytes;                      /* one-time re-layout traffic: read + write */
} tc_layout_advice;

tc_status tc_plan_layout_advice(tc_plan_t plan, tc_layout_advice* out);

/* ---- Free-index sharding -------------------------------------------------
 * Slicing a free index of C splits a contraction into independent ones (Sec.
 * 2.4), which can run on different devices with no data exchanged.  For n
 * shards, tc_shard_free_index picks C's largest free index (ties: the larger
 * stride in C) and gives shard `shard` the balanced index range
 * [begin, end) = [shard * E / n, (shard + 1) * E / n) of it.  The shard's slab
 * is the same contraction with that label's extent end - begin in every
 * tensor holding it, the tensors' strides unchanged (pass them explicitly),
 * and its buffers starting offset_a, offset_b, offset_c elements into A, B
 * and C; plan it with tc_plan and run it with tc_contract.  A shard whose
 * range is empty has nothing to do.  An order-0 C has no free index: label
 * -1, shard 0 computes the whole contraction (end = 1), the others nothing
 * (end = 0).  Host only; the descriptors are read, not kept.  Errors as
 * tc_plan's descriptor checks; TC_ERR_INVALID_ARG for n_shards < 1 or shard
 * outside [0, n_shards). */
typedef struct {
  int32_t label;                          /* the split label of C, -1 for an order-0 C */
  int32_t pos_a, pos_b, pos_c;            /* its index position in A, B, C; -1 where absent */
  int64_t begin, end;                     /* this shard's index range of that label */
  int64_t offset_a, offset_b, offset_c;   /* element offsets of the slab in A, B, C */
} tc_shard;

tc_status tc_shard_free_index(const tc_tensor_desc* A, const tc_tensor_desc* B,
                              const tc_tensor_desc* C, int32_t n_shards, int32_t shard,
                              tc_shard* out);

/* Run the contraction asynchronously on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  A, B, C are device pointers to elements of the
 * plan's dtype laid out as described at tc_plan time; C is read only when
 * beta != 0.  `workspace` is device memory of at least
 * tc_plan_info.workspace bytes (may be NULL when that is 0); with
 * TC_MATH_FP8 it must be 16-byte aligned (else TC_ERR_INVALID_ARG) and holds
 * the packed E4M3 operands and their scales.  Allocates nothing; may be
 * captured in a CUDA graph. */
tc_status tc_contract(tc_plan_t plan, double alpha, const void* A, const void* B, double beta,
                      void* C, void* workspace, size_t workspace_bytes, void* stream);

/* ---- Batched contractions in one submission ------------------------------
 * Many independent contractions (e.g. the products of a coupled-cluster
 * iteration, Sec. 4.2) run as one submission.  A batch is built once from
 * plans (FP32 storage, one tensor-core math form shared by all plans, any
 * mapping but COPY_GEMM); it owns device tables of the plans' index groups,
 * its work lists and a workspace for partial sums, so the plans may be
 * destroyed afterwards.  Each contraction is routed by its GEMM view:
 *   - M and N both >= the route threshold (64 by default): its 128x128 output
 *     tiles join the work list of one persistent tensor-core launch (one CTA
 *     per SM, longest K first); a tile with more K than half of one SM's
 *     share is split into K ranges, added afterwards in range order;
 *   - otherwise (the BLAS-1/2 cases of Sec. 3.2.1-3.2.2 and skinny GEMMs):
 *     CUDA-core kernels sum K segments -- short runs of FP32 products by
 *     fused multiply-adds, the runs added with Neumaier compensation; 32x32
 *     output tiles with operand blocks in shared memory where min(M, N) >= 16,
 *     a thread (or, below 256 outputs, a warp) per output otherwise -- and a
 *     last kernel adds each output's segments in order (FP64). */
typedef struct tc_batch_s* tc_batch_t;

typedef struct {
  int32_t n_items;
  int32_t math;          /* tc_math shared by every item */
  int64_t n_tiles;       /* tensor-core work-list entries */
  double flops;          /* sum over items of 2 * product of all extents */
  double min_bytes;      /* sum over items of |A| + |B| + |C| bytes */
  int32_t n_tc_items;    /* items on the tensor-core route */
  int32_t n_simt_items;  /* items on the CUDA-core route */
  int64_t n_simt_work;   /* CUDA-core partial-sum work entries, per output */
  int64_t n_simt_tiles;  /* CUDA-core partial-sum work entries, 32x32 tiles */
  int64_t n_tc_split;    /* tensor-core tiles whose K is split into ranges */
} tc_batch_info;

/* Route threshold used by later tc_batch_plan calls (process-wide): a
 * contraction goes to the tensor cores when its M and N are both >= tc_min_mn. */
tc_status tc_batch_set_route(int32_t tc_min_mn);

/* Build a batch from n plans (host and device allocation; synchronous).
 * TC_ERR_UNSUPPORTED if a plan's math is not TC_MATH_BF16, _BF16X3 or
 * _BF16X6 (FP32 storage), if the plans use different math forms, if a plan
 * copies an operand (COPY_GEMM), or if a plan has an empty output or an empty
 * contracted range (run those with tc_contract).  n == 0 gives an empty batch,
 * whose launch does nothing.  The batch packs the operands of its
 * tensor-core items into device memory of its own (a plan's workspace is not
 * used); plans with a batch group (the slicing mapping) take the CUDA-core
 * route. */
tc_status tc_batch_plan(tc_batch_t* out, const tc_plan_t* plans, int32_t n);

/* tc_batch_plan with a route per plan (routes may be NULL: all -1):
 *   -1  the threshold rule of tc_batch_set_route,
 *    0  the CUDA-core route, its shape by the rule (32x32 tiles where
 *       min(M, N) >= 16, else a thread or a warp per output),
 *    1  the tensor-core route, 128x128 tiles (TC_ERR_UNSUPPORTED for a plan
 *       with a batch group),
 *    2  the CUDA-core route on 32x32 output tiles,
 *    3  the CUDA-core route with a thread (a warp below 256 outputs) per output;
 * any other value is TC_ERR_INVALID_ARG.  An autotuner
 * (paper_1307_2100_gb300/autotune.py) picks a route and shape per size
 * bucket by timing. */
tc_status tc_batch_plan_routes(tc_batch_t* out, const tc_plan_t* plans, const int32_t* routes,
                               int32_t n);

tc_status tc_batch_get_info(tc_batch_t batch, tc_batch_info* info);

/* Run every contraction of the batch asynchronously on `stream` (at most six
 * kernel launches: pack, tensor-core GEMM, its split-K sums, CUDA-core
 * partial sums per output and per 32x32 tile, final sums).  When both routes have work, the CUDA-core
 * kernels run on a stream the batch owns, forked from `stream` and joined
 * back to it by events, so that the two routes overlap; work queued on
 * `stream` afterwards still sees every result.  A, B, C, alpha, beta are
 * DEVICE arrays of n entries (item i uses A[i], B[i], C[i], alpha[i],
 * beta[i], with the layouts of plan i).  Nothing is allocated or copied by
 * the call, so it may be captured in a CUDA graph; a replay reads the pointer
 * and scalar arrays at replay time.  Launches of one batch must not overlap
 * one another (they share its partial-sum workspace).  The five arrays and
 * every buffer they point to must stay allocated until the launch has
 * completed: the kernels read them on the device and cannot check them. */
tc_status tc_contract_batched(tc_batch_t batch, const void* const* A, const void* const* B,
                              void* const* C, const double* alpha, const double* beta,
                              void* stream);

/* Free a batch (NULL is allowed).  The batch must not be in use on the GPU. */
tc_status tc_batch_destroy(tc_batch_t batch);

/* Reads and clears the device error flag of the current device after
 * synchronising `stream`: TC_ERR_TIMEOUT if a bounded device wait ran out
 * since the last call, else TC_OK. */
tc_status tc_device_status(void* stream);

/* ---- The learned mapping selector -----------------------------------------
 * tc_plan_features() describes a planned contraction by TC_SELECTOR_FEATURES
 * numbers (log2 sizes of the fused GEMM view, index counts, the class of
 * Sec. 3.2, where the stride-1 indices sit, the extents the recipe leaves
 * unsliced, flops and bytes).  A selector file, written by the training
 * driver (paper_1307_2100_gb300/selector.py), holds a network that predicts
 * the log2 runtime of each candidate from them.  A candidate is a mapping
 * and, optionally, a tile configuration, encoded as
 * TC_SELECTOR_CANDIDATE(mapping, tile) (tile -1: the plan's default).  Once
 * loaded, tc_plan with TC_MAP_AUTO runs the network on the host and uses the
 * candidate with the smallest prediction among those able to compute the
 * contraction (its tile too, unless tc_plan was given one); with no selector
 * loaded, for another dtype/math, or when a feature lies outside the range
 * seen in training, AUTO falls back to the paper's recipe. */
#define TC_SELECTOR_FEATURES 23
#define TC_SELECTOR_CANDIDATE(mapping, tile) ((int32_t)(mapping) | (((int32_t)(tile) + 1) << 8))

tc_status tc_plan_features(tc_plan_t plan, float* out, int32_t n);
/* Load a selector file or unload every selector.  A file holds the network of
 * one storage type and math form; loading replaces the selector loaded for
 * that form, if any, and keeps those of other forms (up to eight forms, else
 * TC_ERR_UNSUPPORTED).  tc_plan(AUTO) consults the selector of the plan's own
 * storage type and math form.  tc_selector_load returns TC_ERR_INVALID_ARG
 * for a malformed file. */
tc_status tc_selector_load(const char* path);
tc_status tc_selector_unload(void);
/* Host prediction, with the most recently loaded selector, for n feature
 * vectors (n x TC_SELECTOR_FEATURES floats): out is n x n_cand log2 runtimes,
 * cand receives the candidates (TC_SELECTOR_CANDIDATE values, array of at
 * least 16).  TC_ERR_NO_SELECTOR if none is loaded. */
tc_status tc_selector_predict(const float* features, int32_t n, float* out, int32_t* cand,
                              int32_t* n_cand);

/* ---- The mapping selector's network ---------------------------------------
 * A 3-layer perceptron (in -> hidden -> hidden -> out, ReLU) that predicts the
 * log2 runtime of every candidate mapping from a descriptor's features
 * (tc_plan_features), trained and run by the library's own kernels: the
 * forward pass, the masked mean-squared-error backward pass and Adam.
 * Parameters are one flat FP32 vector W1[h][in], b1, W2[h][h], b2, W3[out][h],
 * b3 (the master copy); forward and backward use its FP16 rounding (the
 * working copy).  All pointers below are device pointers unless stated; X is
 * [batch][in], T and mask are [batch][out] row-major FP32.  The paper's recipe
 * (Sec. 3.2) is the fallback whenever no trained network is loaded. */
typedef struct tc_mlp_s* tc_mlp_t;

/* Allocates the network (parameters zero) for batches up to max_batch. */
tc_status tc_mlp_create(tc_mlp_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                        int32_t max_batch);
tc_status tc_mlp_destroy(tc_mlp_t net);
tc_status tc_mlp_num_params(tc_mlp_t net, int64_t* n);
/* Host array of n FP32 parameters -> master copy (and its FP16 working copy);
 * resets the Adam moments.  Synchronous. */
tc_status tc_mlp_set_params(tc_mlp_t net, const float* host, int64_t n);
/* Master copy (working == 0) or FP16 working copy (working != 0) -> host. */
tc_status tc_mlp_get_params(tc_mlp_t net, float* host, int64_t n, int32_t working);
/* Y[batch][out] = network(X) with the working copy. */
tc_status tc_mlp_forward(tc_mlp_t net, const float* X, float* Y, int32_t batch, void* stream);
/* loss (device scalar) = sum(mask * (Y - T)^2) / sum(mask) and its gradient
 * with respect to the working parameters (device array of n_params). */
tc_status tc_mlp_loss_grad(tc_mlp_t net, const float* X, const float* T, const float* mask,
                           int32_t batch, float* loss, float* grad, void* stream);
/* One bias-corrected Adam step (step number t >= 1) on the master copy. */
tc_status tc_mlp_adam_step(tc_mlp_t net, const float* grad, float lr, float beta1, float beta2,
                           float eps, int32_t t, void* stream);

/* ---- Scalar contraction without a workspace -------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that
 * cannot allocate device memory when they contract: runtimes that reserve all
 * device memory for their own pool up front, plug-ins handed only input and
 * output pointers, and latency-critical loops that cannot afford the device
 * synchronisation cudaMalloc / cudaFree may imply.  It runs a plan whose
 * result is a single element (Class 1 mapped to DOT, the one kernel that needs
 * scratch space, for its per-block partial sums) with the same kernels as
 * tc_contract, but keeps the partial sums in a fixed scratch array built into
 * the library instead of a workspace:
 *   - the array holds TC_NOALLOC_SCRATCH_BYTES on every GPU that loads the
 *     library, until the process exits; the DOT kernel's partial sums (608
 *     doubles, 4.9 KB, whatever the contraction's size) fit in it; should a
 *     plan ever need more, the call returns TC_ERR_WORKSPACE;
 *   - all calls share the array: calls that overlap on the GPU race; calls
 *     ordered on one stream are fine; the array keeps the last call's
 *     contents, none of which a later call relies on;
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it; make that
 *     first call before any stream capture; a cudaDeviceReset of the device
 *     invalidates the kept address, so do not call this entry point on a
 *     device after resetting it in the same process;
 *   - devices numbered 64 or above return TC_ERR_UNSUPPORTED.
 * Other plans return TC_ERR_UNSUPPORTED.  Calls no allocating routine. */
#define TC_NOALLOC_SCRATCH_BYTES (16 * 1024)
tc_status tc_contract_dot_noalloc(tc_plan_t plan, double alpha, const void* A, const void* B,
                                  double beta, void* C, void* stream);

/* Self-test of the bounded device waits: launches one warp that waits on an
 * mbarrier nothing ever arrives on.  The wait gives up after `timeout_ns`
 * nanoseconds, records the timeout in the device flag and returns, so a
 * following tc_device_status() reports TC_ERR_TIMEOUT.  No fault, no hang. */
tc_status tc_selftest_wait_timeout(int64_t timeout_ns, void* stream);

/* ---- Peak-rate probes (measurement support) -------------------------------
 * The roofline of each kernel is its arithmetic's peak rate on this GPU,
 * measured in the same process: one launch of a probe kernel that keeps
 * every SM busy with one kind of arithmetic and no memory traffic (operands
 * in registers, or a zero tile in shared memory that each MMA re-reads).
 * tc_peak_probe enqueues it on `stream` (a cudaStream_t) and stores the
 * floating-point operations the launch performs in *flops (host pointer);
 * time the launch with events on the same stream.  `iters` >= 1 sets the
 * length: per thread (CUDA-core kinds) or per issuing thread (tensor-core
 * kinds).  The paper has no counterpart (its peaks are the CPUs' nominal
 * figures, Sec. 4). */
typedef enum {
  TC_PEAK_DFMA = 0,       /* FP64 fused multiply-add, CUDA cores */
  TC_PEAK_DMMA = 1,       /* FP64 mma.sync m8n8k4 */
  TC_PEAK_FFMA = 2,       /* FP32 fused multiply-add, CUDA cores */
  TC_PEAK_BF16 = 3,       /* tcgen05.mma kind::f16 BF16, 128 x 128 x 16 */
  TC_PEAK_BF16_N256 = 4,  /* tcgen05.mma kind::f16 BF16, 128 x 256 x 16 */
  TC_PEAK_FP8 = 5         /* tcgen05.mma kind::mxf8f6f4 E4M3 block-scaled, 128 x 128 x 32 */
} tc_peak_kind;
tc_status tc_peak_probe(int32_t kind, int64_t iters, double* flops, void* stream);

/* Static description of a status code. */
const char* tc_status_string(tc_status s);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
