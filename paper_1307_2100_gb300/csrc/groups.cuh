// groups.cuh -- device-side address arithmetic of index groups.
//
// A group index is split column-major into the group's labels (first label
// fastest) and each label adds index * stride of the tensor slot asked for
// (0 = the kernel's first operand, 1 = its second operand, 2 = C).  Groups
// hold fewer than 2^31 elements, so the splits use 32-bit division, done as a
// multiply and a shift by each extent's precomputed constants.
#pragma once
#include <cstdint>

#include "tc_internal.h"

namespace tc {

// idx / ext[i] of a group index (idx < 2^31 whenever dmul[i] is set).
__device__ __forceinline__ uint32_t gdiv(const Group& g, int i, uint32_t idx) {
  const uint32_t m = g.dmul[i];
  return m ? (uint32_t)(((uint64_t)idx * m) >> g.dsh[i]) : idx / (uint32_t)g.ext[i];
}

// Offset of group index `idx` in tensor slot `t` (0 = first operand, 1 =
// second operand, 2 = C).  Groups are < 2^31 elements, so 32-bit division.
__device__ __forceinline__ int64_t goff(const Group& g, int t, uint32_t idx) {
  if (g.n == 1) return (int64_t)idx * g.st[t][0];
  int64_t off = 0;
  for (int i = 0; i < g.n; ++i) {
    uint32_t e = (uint32_t)g.ext[i];
    uint32_t q = gdiv(g, i, idx);
    off += (int64_t)(idx - q * e) * g.st[t][i];
    idx = q;
  }
  return off;
}

// goff for a group of 2^31 or more elements (a whole operand or a whole C,
// as the COPY baseline and the beta-only scaling walk them): the index is
// split with 64-bit division, so no part of it wraps.
__device__ __forceinline__ int64_t goff_wide(const Group& g, int t, uint64_t idx) {
  int64_t off = 0;
  for (int i = 0; i < g.n; ++i) {
    const uint64_t e = (uint64_t)g.ext[i];
    const uint64_t q = idx / e;
    off += (int64_t)(idx - q * e) * g.st[t][i];
    idx = q;
  }
  return off;
}

// Two offsets of one group index at once (first operand and C, etc.).
__device__ __forceinline__ void goff2(const Group& g, int t0, int t1, uint32_t idx, int64_t& o0,
                                      int64_t& o1) {
  o0 = 0;
  o1 = 0;
  for (int i = 0; i < g.n; ++i) {
    uint32_t e = (uint32_t)g.ext[i];
    uint32_t q = gdiv(g, i, idx);
    uint32_t r = idx - q * e;
    o0 += (int64_t)r * g.st[t0][i];
    o1 += (int64_t)r * g.st[t1][i];
    idx = q;
  }
}

__device__ __forceinline__ void goff3(const Group& g, uint32_t idx, int64_t& o0, int64_t& o1,
                                      int64_t& o2) {
  o0 = o1 = o2 = 0;
  for (int i = 0; i < g.n; ++i) {
    uint32_t e = (uint32_t)g.ext[i];
    uint32_t q = gdiv(g, i, idx);
    uint32_t r = idx - q * e;
    o0 += (int64_t)r * g.st[0][i];
    o1 += (int64_t)r * g.st[1][i];
    o2 += (int64_t)r * g.st[2][i];
    idx = q;
  }
}

}  // namespace tc
