/*
 * tco.c -- CPU FP64 oracle for binary tensor contractions (test infrastructure).
 *
 * Parity: pinned.  The pins (naive matrix/vector loops, integer exactness,
 * closed forms, invariances, brute force on tiny extents) live in the tests.
 *
 * The oracle is the definition written out (Sec. 2.1, Sec. 2.3 Einstein
 * convention, Appendix "index contraction"): for every output multi-index,
 * a plain loop over every contracted multi-index accumulating A*B in double.
 * A label of A, B and C (a batch, or Hadamard, index; beyond the paper's
 * definition, which pairs every label) is an output label that indexes both
 * operands: the output loop supplies its value to A, B and C.
 * Compiled with -O2 -ffp-contract=off so each step is a separate multiply
 * and add.  Parallelism (optional OpenMP) is over output elements only; each
 * output is summed by one thread in a fixed order, so the result does not
 * depend on the thread count.
 */
#include "tco.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TCO_MAX 32

typedef struct {
  int n;                 /* number of labels in the group */
  int64_t ext[TCO_MAX];
  int64_t sa[TCO_MAX];   /* stride in A (0 if absent) */
  int64_t sb[TCO_MAX];   /* stride in B (0 if absent) */
  int64_t sc[TCO_MAX];   /* stride in C (0 if absent) */
} group_t;

static int find(const tco_desc* t, int32_t label) {
  for (int i = 0; i < t->order; ++i)
    if (t->labels[i] == label) return i;
  return -1;
}

static int64_t stride_of(const tco_desc* t, int pos) {
  if (t->strides) return t->strides[pos];
  int64_t s = 1;
  for (int i = 0; i < pos; ++i) s *= t->extents[i];
  return s;
}

static int check_desc(const tco_desc* t) {
  if (!t || t->order < 0 || t->order > TCO_MAX) return 1;
  if (t->order > 0 && (!t->labels || !t->extents)) return 1;
  for (int i = 0; i < t->order; ++i) {
    if (t->extents[i] < 0) return 1;
    for (int j = 0; j < i; ++j)
      if (t->labels[i] == t->labels[j]) return 2;
  }
  return 0;
}

int tco_contract_f64(const tco_desc* A, const double* a, const tco_desc* B, const double* b,
                     const tco_desc* C, double* c, double alpha, double beta, int nthreads) {
  int st;
  if ((st = check_desc(A)) || (st = check_desc(B)) || (st = check_desc(C))) return st;

  /* Output labels: each comes from one operand, or from both (a batch label),
   * with equal extents. */
  group_t out;
  memset(&out, 0, sizeof(out));
  out.n = C->order;
  for (int i = 0; i < C->order; ++i) {
    int32_t l = C->labels[i];
    int pa = find(A, l), pb = find(B, l);
    if (pa < 0 && pb < 0) return 2;
    int64_t e = C->extents[i];
    if (pa >= 0 && A->extents[pa] != e) return 3;
    if (pb >= 0 && B->extents[pb] != e) return 3;
    out.ext[i] = e;
    out.sc[i] = stride_of(C, i);
    out.sa[i] = pa >= 0 ? stride_of(A, pa) : 0;
    out.sb[i] = pb >= 0 ? stride_of(B, pb) : 0;
  }

  /* Contracted labels: in both A and B, not in C.  Every label of A (or B)
   * must be either contracted or an output label. */
  group_t con;
  memset(&con, 0, sizeof(con));
  int32_t cl[TCO_MAX];
  int nc = 0;
  for (int i = 0; i < A->order; ++i) {
    int32_t l = A->labels[i];
    int pb = find(B, l), pc = find(C, l);
    if (pb < 0 && pc < 0) return 2;
    if (pb >= 0 && pc < 0) {
      if (A->extents[i] != B->extents[pb]) return 3;
      cl[nc++] = l;
    }
  }
  for (int i = 0; i < B->order; ++i) {
    int32_t l = B->labels[i];
    if (find(A, l) < 0 && find(C, l) < 0) return 2;
  }
  /* canonical order: ascending label value, first = fastest */
  for (int i = 1; i < nc; ++i)
    for (int j = i; j > 0 && cl[j - 1] > cl[j]; --j) {
      int32_t t = cl[j]; cl[j] = cl[j - 1]; cl[j - 1] = t;
    }
  con.n = nc;
  for (int i = 0; i < nc; ++i) {
    int pa = find(A, cl[i]), pb = find(B, cl[i]);
    con.ext[i] = A->extents[pa];
    con.sa[i] = stride_of(A, pa);
    con.sb[i] = stride_of(B, pb);
  }

  int64_t nout = 1, ncon = 1;
  for (int i = 0; i < out.n; ++i) nout *= out.ext[i];
  for (int i = 0; i < con.n; ++i) ncon *= con.ext[i];
  if (nout > 0 && !c) return 1;
  if (nout > 0 && ncon > 0 && (!a || !b)) return 1;

#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#else
  (void)nthreads;
#endif
  for (int64_t q = 0; q < nout; ++q) {
    /* column-major decomposition of the output linear index */
    int64_t rem = q, oa = 0, ob = 0, oc = 0;
    for (int i = 0; i < out.n; ++i) {
      int64_t idx = rem % out.ext[i];
      rem /= out.ext[i];
      oa += idx * out.sa[i];
      ob += idx * out.sb[i];
      oc += idx * out.sc[i];
    }
    double s = 0.0;
    int64_t kidx[TCO_MAX];
    for (int i = 0; i < con.n; ++i) kidx[i] = 0;
    int64_t ka = 0, kb = 0;
    for (int64_t k = 0; k < ncon; ++k) {
      double prod = a[oa + ka] * b[ob + kb];
      s = s + prod;
      /* advance the contracted multi-index, first label fastest */
      for (int i = 0; i < con.n; ++i) {
        kidx[i] += 1;
        ka += con.sa[i];
        kb += con.sb[i];
        if (kidx[i] < con.ext[i]) break;
        ka -= con.sa[i] * con.ext[i];
        kb -= con.sb[i] * con.ext[i];
        kidx[i] = 0;
      }
    }
    double r = alpha * s;
    if (beta != 0.0) r = r + beta * c[oc];
    c[oc] = r;
  }
  return 0;
}
