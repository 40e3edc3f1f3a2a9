/*
 * tco.h -- CPU FP64 oracle for binary tensor contractions.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference
 * the GPU library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product library neither
 * includes this header nor links this code, and this code includes nothing of
 * the product library.
 *
 * What it computes (Sec. 2.1 c_ij = sum_h a_ih b_hj generalised in Sec. 2.3 and
 * the Appendix): every label appearing in both A and B is summed over its full
 * range; the remaining labels of A and of B index the result C.
 *
 *     C[c] = alpha * sum_k A[a(c,k)] * B[b(c,k)]  +  beta * C[c]
 *
 * beta == 0 means C is write-only (its old contents, NaN included, are never
 * read).  Summation runs over the contracted multi-index with the contracted
 * labels sorted by ascending label value, the smallest label varying fastest,
 * so the rounding order depends only on the labels (not on storage order).
 */
#ifndef TCO_H
#define TCO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t order;           /* number of indices (0 = scalar) */
  const int32_t* labels;   /* order labels, distinct within the tensor */
  const int64_t* extents;  /* order extents (>= 0) */
  const int64_t* strides;  /* order strides in elements, or NULL = column-major */
} tco_desc;

/* Status: 0 ok; 1 bad argument; 2 label error (repeated label, label of C not
 * found in exactly one operand, label of A/B missing from C and from the other
 * operand, label in both operands and in C); 3 extent mismatch. */
int tco_contract_f64(const tco_desc* A, const double* a, const tco_desc* B, const double* b,
                     const tco_desc* C, double* c, double alpha, double beta, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
