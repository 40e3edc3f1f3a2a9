// plan.cpp -- descriptor analysis, classification and plan building (host only).
//
// Steps (Sec. 3 of the paper, adapted to one GPU):
//   1. read and validate the three descriptors;
//   2. split labels into contracted (in A and B), free of A, free of B;
//   3. classify by Delta(t) = N(t) - p and the stride-1 indices (Sec. 3.2);
//   4. derive the recipe's slicing vectors (Sec. 3.2 recipes, R1-R3 of Sec. 3.1);
//   5. build the GEMM view for the chosen mapping: groups M, N, K, batch with
//      per-operand strides, after merging index runs that are linear in every
//      tensor.
// Readings where the paper is silent: indices of extent 1 are ignored by the
// classification; the stride-1 index is the index with stride 1 and extent > 1
// (none: the operand cannot satisfy R1 and a Class 3 contraction is 3.1);
// largest-extent ties go to the smaller stride in C (free) or in the operand
// (contracted), then to the earlier position; in Class 3.1 the operand whose
// stride-1 index is larger keeps it (ties: A).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "tc_internal.h"

namespace tc {

size_t elem_size(tc_dtype dt) { return dt == TC_F64 ? 8 : dt == TC_F32 ? 4 : 2; }

namespace {

struct Tens {
  std::vector<int32_t> lab;
  std::vector<int64_t> ext;
  std::vector<int64_t> st;
  int find(int32_t l) const {
    for (size_t i = 0; i < lab.size(); ++i)
      if (lab[i] == l) return (int)i;
    return -1;
  }
  int64_t numel() const {
    int64_t n = 1;
    for (auto e : ext) n *= e;
    return n;
  }
  int32_t stride1() const {
    for (size_t i = 0; i < lab.size(); ++i)
      if (ext[i] > 1 && st[i] == 1) return lab[i];
    return -1;
  }
  int64_t stride_of(int32_t l) const {
    int p = find(l);
    return p < 0 ? 0 : st[p];
  }
};

tc_status read_desc(const tc_tensor_desc* d, Tens& t) {
  if (!d) return TC_ERR_INVALID_ARG;
  if (d->order < 0 || d->order > TC_MAX_ORDER) return TC_ERR_INVALID_ARG;
  if (d->order > 0 && (!d->labels || !d->extents)) return TC_ERR_INVALID_ARG;
  int64_t acc = 1;
  for (int i = 0; i < d->order; ++i) {
    int64_t e = d->extents[i];
    if (e < 0) return TC_ERR_INVALID_ARG;
    int64_t s = d->strides ? d->strides[i] : acc;
    acc *= (e > 0 ? e : 1);
    if (e > 1 && s <= 0) return TC_ERR_STRIDE;
    for (int j = 0; j < i; ++j)
      if (d->labels[j] == d->labels[i]) return TC_ERR_LABEL;
    t.lab.push_back(d->labels[i]);
    t.ext.push_back(e);
    t.st.push_back(e > 1 ? s : 0);
  }
  return TC_OK;
}

// C must not alias: sorted by stride, each stride covers the previous span.
bool output_aliases(const Tens& c) {
  std::vector<std::pair<int64_t, int64_t>> v;
  for (size_t i = 0; i < c.lab.size(); ++i)
    if (c.ext[i] > 1) v.push_back({c.st[i], c.ext[i]});
  std::sort(v.begin(), v.end());
  for (size_t i = 1; i < v.size(); ++i)
    if (v[i].first < v[i - 1].first * v[i - 1].second) return true;
  return false;
}

struct Analysis {
  std::vector<int32_t> con, fa, fb;  // contracted, free of A, free of B (all extents)
  std::vector<int32_t> bat;          // batch labels: in A, B and C
  std::map<int32_t, int64_t> ext;
  int cls = 0;
  int p = 0, da = 0, db = 0;
  int32_t s1a = -1, s1b = -1;
  std::vector<int32_t> keep_a, keep_b;  // recipe: unsliced labels
  char copied = 0;                      // 'A' or 'B' (Class 3.1)
};

bool contains(const std::vector<int32_t>& v, int32_t l) {
  return std::find(v.begin(), v.end(), l) != v.end();
}

// Largest extent, ties by (key1, key2) ascending.
template <class F>
int32_t pick_largest(const std::vector<int32_t>& cands, const std::map<int32_t, int64_t>& ext,
                     F key) {
  int32_t best = -1;
  for (int32_t l : cands) {
    if (best < 0) { best = l; continue; }
    int64_t eb = ext.at(best), el = ext.at(l);
    if (el > eb || (el == eb && key(l) < key(best))) best = l;
  }
  return best;
}

void classify(const Tens& A, const Tens& B, const Tens& C, Analysis& an) {
  auto big = [&](const std::vector<int32_t>& v) {
    std::vector<int32_t> r;
    for (auto l : v)
      if (an.ext[l] > 1) r.push_back(l);
    return r;
  };
  std::vector<int32_t> K = big(an.con), FA = big(an.fa), FB = big(an.fb);
  an.p = (int)K.size();
  an.da = (int)FA.size();
  an.db = (int)FB.size();
  an.s1a = A.stride1();
  an.s1b = B.stride1();
  const int32_t s1a = an.s1a, s1b = an.s1b;

  auto free_key = [&](const Tens& T) {
    return [&C, &T](int32_t l) {
      return std::make_pair(C.stride_of(l), (int64_t)T.find(l));
    };
  };
  auto con_key = [](const Tens& T) {
    return [&T](int32_t l) { return std::make_pair(T.stride_of(l), (int64_t)T.find(l)); };
  };
  auto pick_free = [&](const std::vector<int32_t>& c, const Tens& T) {
    return pick_largest(c, an.ext, free_key(T));
  };
  auto pick_con = [&](const std::vector<int32_t>& c, const Tens& T) {
    return c.empty() ? -1 : pick_largest(c, an.ext, con_key(T));
  };
  auto in = [](const std::vector<int32_t>& v, int32_t l) { return l >= 0 && contains(v, l); };

  std::vector<int32_t> ka, kb;
  if (an.da == 0 && an.db == 0) {
    an.cls = 1;
    if (!K.empty()) {
      int32_t k = in(K, s1a) ? s1a : pick_con(K, A);
      ka = {k};
      kb = {k};
    }
  } else if (an.da == 0 || an.db == 0) {
    an.cls = 2;
    const bool t1_is_a = an.da >= 1;
    const Tens& T1 = t1_is_a ? A : B;
    const std::vector<int32_t>& F1 = t1_is_a ? FA : FB;
    const int32_t s1 = t1_is_a ? s1a : s1b;
    int32_t kf, kc;
    if (in(K, s1)) {           // stride-1 index contracted: keep it and one free index
      kc = s1;
      kf = pick_free(F1, T1);
    } else if (in(F1, s1)) {   // stride-1 index free: keep it and one contracted index
      kf = s1;
      kc = pick_con(K, T1);
    } else {
      kf = pick_free(F1, T1);
      kc = pick_con(K, T1);
    }
    std::vector<int32_t> t1 = {kf}, t2;
    if (kc >= 0) {
      t1.push_back(kc);
      t2.push_back(kc);
    }
    if (t1_is_a) { ka = t1; kb = t2; } else { ka = t2; kb = t1; }
  } else {
    const bool both_con = in(K, s1a) && in(K, s1b);
    if (s1a < 0 || s1b < 0 || (s1a != s1b && both_con)) {
      an.cls = 31;
      bool keep_first_a = (s1a >= 0 && s1b >= 0) ? an.ext[s1a] >= an.ext[s1b] : (s1a >= 0);
      int32_t k;
      if (keep_first_a && in(K, s1a)) {
        k = s1a;
        an.copied = 'B';
      } else if (!keep_first_a && in(K, s1b)) {
        k = s1b;
        an.copied = 'A';
      } else {
        k = pick_con(K, A);
        an.copied = keep_first_a ? 'B' : 'A';
      }
      int32_t fa = in(FA, s1a) ? s1a : pick_free(FA, A);
      int32_t fb = in(FB, s1b) ? s1b : pick_free(FB, B);
      ka = {fa};
      kb = {fb};
      if (k >= 0) { ka.push_back(k); kb.push_back(k); }
    } else {
      an.cls = 32;
      int32_t k, fa, fb;
      if (in(K, s1a) && in(K, s1b)) {
        k = s1a;
        fa = pick_free(FA, A);
        fb = pick_free(FB, B);
      } else if (in(K, s1a)) {
        k = s1a; fb = s1b; fa = pick_free(FA, A);
      } else if (in(K, s1b)) {
        k = s1b; fa = s1a; fb = pick_free(FB, B);
      } else {
        fa = s1a; fb = s1b; k = pick_con(K, A);
      }
      ka = {fa};
      kb = {fb};
      if (k >= 0) { ka.push_back(k); kb.push_back(k); }
    }
  }
  an.keep_a = ka;
  an.keep_b = kb;
}

uint32_t slice_bits(const Tens& T, const std::vector<int32_t>& keep) {
  uint32_t bits = 0;
  for (size_t i = 0; i < T.lab.size(); ++i)
    if (!contains(keep, T.lab[i])) bits |= (1u << i);
  return bits;
}

// With d in [1, 2^31), l = ceil(log2 d) and m = ceil(2^(31+l) / d):
// 2^(31+l) <= m d < 2^(31+l) + 2^l, so floor(n / d) = floor(n m / 2^(31+l))
// for every n < 2^31 (Granlund and Montgomery 1994, Theorem 4.2), and
// m < 2^32.  Groups of 2^31 or more elements keep the division.
void group_divisors(Group& g, int64_t total) {
  for (int i = 0; i < kGroupMax; ++i) g.dmul[i] = g.dsh[i] = 0;
  if (total <= 0 || total >= ((int64_t)1 << 31)) return;
  for (int i = 0; i < g.n; ++i) {
    const uint64_t d = (uint64_t)g.ext[i];
    if (d == 0) continue;
    uint32_t l = 0;
    while (((uint64_t)1 << l) < d) ++l;
    g.dmul[i] = (uint32_t)((((uint64_t)1 << (31 + l)) + d - 1) / d);
    g.dsh[i] = 31 + l;
  }
}

// Build a group from labels in the given order: strides from X, Y, C; drop
// extent-1 labels; merge runs linear in every tensor.
bool make_group(const std::vector<int32_t>& labels, const std::map<int32_t, int64_t>& ext,
                const Tens* X, const Tens* Y, const Tens* Cc, Group& g, int64_t& total) {
  std::memset(&g, 0, sizeof(g));
  total = 1;
  const Tens* ts[3] = {X, Y, Cc};
  for (int32_t l : labels) {
    int64_t e = ext.at(l);
    total *= e;
    if (e == 1) continue;
    int64_t s[3];
    for (int t = 0; t < 3; ++t) s[t] = ts[t] ? ts[t]->stride_of(l) : 0;
    if (g.n > 0) {
      int q = g.n - 1;
      bool lin = true;
      for (int t = 0; t < 3; ++t)
        if (s[t] != g.st[t][q] * g.ext[q]) lin = false;
      if (lin) {
        g.ext[q] *= e;
        continue;
      }
    }
    if (g.n >= kGroupMax) return false;
    g.ext[g.n] = e;
    for (int t = 0; t < 3; ++t) g.st[t][g.n] = s[t];
    g.n++;
  }
  if (total == 0) {  // empty group: keep one zero-extent entry
    g.n = 1;
    g.ext[0] = 0;
  }
  group_divisors(g, total);
  return true;
}

std::vector<int32_t> sorted_by(std::vector<int32_t> v, const Tens& T) {
  std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) {
    return T.stride_of(x) < T.stride_of(y);
  });
  return v;
}

}  // namespace

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_plan(tc_plan_t* out, const tc_tensor_desc* Ad, const tc_tensor_desc* Bd,
                             const tc_tensor_desc* Cd, tc_dtype dtype, tc_math math,
                             tc_mapping mapping, int32_t tile) {
  if (!out) return TC_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype < TC_F64 || dtype > TC_F16) return TC_ERR_INVALID_ARG;
  if (math < TC_MATH_FP64 || math > TC_MATH_FP16) return TC_ERR_INVALID_ARG;
  if (mapping < TC_MAP_AUTO || mapping > TC_MAP_GER) return TC_ERR_INVALID_ARG;
  if ((math == TC_MATH_FP64) != (dtype == TC_F64)) return TC_ERR_UNSUPPORTED;
  // BF16 / FP16 storage: FP32 arithmetic on the CUDA cores, or the tensor
  // cores' products of the stored values (exact)
  if (dtype == TC_BF16 && math != TC_MATH_FP32 && math != TC_MATH_BF16) return TC_ERR_UNSUPPORTED;
  if (dtype == TC_F16 && math != TC_MATH_FP32 && math != TC_MATH_FP16) return TC_ERR_UNSUPPORTED;

  Tens A, B, C;
  tc_status st;
  if ((st = read_desc(Ad, A)) != TC_OK) return st;
  if ((st = read_desc(Bd, B)) != TC_OK) return st;
  if ((st = read_desc(Cd, C)) != TC_OK) return st;

  Analysis an;
  for (size_t i = 0; i < C.lab.size(); ++i) {
    int32_t l = C.lab[i];
    int pa = A.find(l), pb = B.find(l);
    if (pa < 0 && pb < 0) return TC_ERR_LABEL;
    int64_t e = C.ext[i];
    if ((pa >= 0 && A.ext[pa] != e) || (pb >= 0 && B.ext[pb] != e)) return TC_ERR_EXTENT_MISMATCH;
    if (pa >= 0 && pb >= 0) an.bat.push_back(l);  // batch (Hadamard) label
    an.ext[l] = e;
  }
  for (size_t i = 0; i < A.lab.size(); ++i) {
    int32_t l = A.lab[i];
    int pb = B.find(l), pc = C.find(l);
    if (pb < 0 && pc < 0) return TC_ERR_LABEL;
    if (pb >= 0 && pc < 0) {
      if (A.ext[i] != B.ext[pb]) return TC_ERR_EXTENT_MISMATCH;
      an.con.push_back(l);
    } else if (pb < 0) {
      an.fa.push_back(l);
    }
    an.ext[l] = A.ext[i];
  }
  for (size_t i = 0; i < B.lab.size(); ++i) {
    int32_t l = B.lab[i];
    if (A.find(l) < 0) {
      if (C.find(l) < 0) return TC_ERR_LABEL;
      an.fb.push_back(l);
    }
    an.ext[l] = B.ext[i];
  }
  if (output_aliases(C)) return TC_ERR_STRIDE;

  // the class is that of one batch slice: batch labels are left out
  if (an.bat.empty()) {
    classify(A, B, C, an);
  } else {
    auto drop = [&](const Tens& T) {
      Tens R;
      for (size_t i = 0; i < T.lab.size(); ++i)
        if (!contains(an.bat, T.lab[i])) {
          R.lab.push_back(T.lab[i]);
          R.ext.push_back(T.ext[i]);
          R.st.push_back(T.st[i]);
        }
      return R;
    };
    classify(drop(A), drop(B), drop(C), an);
  }

  Plan* P = new (std::nothrow) Plan();
  if (!P) return TC_ERR_INVALID_ARG;
  std::memset(&P->info, 0, sizeof(P->info));
  P->dtype = dtype;
  P->math = math;
  tc_plan_info& info = P->info;
  info.cls = an.cls;
  info.p = an.p;
  info.delta_a = an.da;
  info.delta_b = an.db;
  info.stride1_a = an.s1a;
  info.stride1_b = an.s1b;
  info.slice_a = slice_bits(A, an.keep_a);
  info.slice_b = slice_bits(B, an.keep_b);
  double flops = 2.0;
  for (auto& kv : an.ext) flops *= (double)kv.second;
  info.flops = flops;
  const size_t es = elem_size(dtype);
  info.min_bytes = (double)(A.numel() + B.numel() + C.numel()) * (double)es;

  // ---- storage-layout advice (Sec. 3.3): give the smaller operand of a
  // Class 3.1 contraction a free stride-1 index
  {
    tc_layout_advice& adv = P->advice;
    std::memset(&adv, 0, sizeof(adv));
    adv.cls_after = an.cls;
    if (an.cls == 31) {
      const bool re_a = A.numel() < B.numel();
      const Tens& T = re_a ? A : B;
      const std::vector<int32_t>& fr = re_a ? an.fa : an.fb;
      int32_t first = -1;
      for (auto l : fr)
        if (an.ext[l] > 1 && (first < 0 || an.ext[l] > an.ext[first])) first = l;
      if (first >= 0) {
        std::vector<int> pos(T.lab.size());
        for (size_t i = 0; i < pos.size(); ++i) pos[i] = (int)i;
        std::stable_sort(pos.begin(), pos.end(), [&](int x, int y) {
          const bool fx = T.lab[x] == first, fy = T.lab[y] == first;
          if (fx != fy) return fx;
          return T.st[x] < T.st[y];
        });
        adv.operand = re_a ? 1 : 2;
        adv.order = (int32_t)pos.size();
        for (size_t i = 0; i < pos.size(); ++i) adv.storage_order[i] = pos[i];
        adv.cls_after = 32;
        adv.copy_bytes = 2.0 * (double)T.numel() * (double)elem_size(dtype);
      }
    }
  }

  // ---- mapping
  // ---- descriptor features (the selector's input; computed for every plan)
  {
    float* f = P->features;
    for (int i = 0; i < TC_SELECTOR_FEATURES; ++i) f[i] = 0.0f;
    auto lg = [](double x) { return (float)(std::log2(std::max(x, 1.0))); };
    auto prod = [&](const std::vector<int32_t>& v) {
      double t = 1.0;
      for (auto l : v) t *= (double)an.ext[l];
      return t;
    };
    auto nbig = [&](const std::vector<int32_t>& v) {
      int c = 0;
      for (auto l : v) c += an.ext[l] > 1;
      return (float)c;
    };
    f[0] = lg(prod(an.fa)) / 16;
    f[1] = lg(prod(an.fb)) / 16;
    f[2] = lg(prod(an.con)) / 16;
    f[3] = nbig(an.fa) / 8;
    f[4] = nbig(an.fb) / 8;
    f[5] = nbig(an.con) / 8;
    f[6] = an.cls == 1;
    f[7] = an.cls == 2;
    f[8] = an.cls == 31;
    f[9] = an.cls == 32;
    f[10] = an.s1a >= 0 && contains(an.con, an.s1a);
    f[11] = an.s1a >= 0 && contains(an.fa, an.s1a);
    f[12] = an.s1b >= 0 && contains(an.con, an.s1b);
    f[13] = an.s1b >= 0 && contains(an.fb, an.s1b);
    const int32_t s1c = C.stride1();
    f[14] = s1c >= 0 && contains(an.fa, s1c);
    f[15] = s1c >= 0 && contains(an.fb, s1c);
    int32_t kf = -1, kc = -1, kb = -1;
    for (auto l : an.keep_a) (contains(an.con, l) ? kc : kf) = l;
    for (auto l : an.keep_b)
      if (!contains(an.con, l)) kb = l;
    f[16] = kf >= 0 ? lg((double)an.ext[kf]) / 16 : 0.0f;
    f[17] = kb >= 0 ? lg((double)an.ext[kb]) / 16 : 0.0f;
    f[18] = kc >= 0 ? lg((double)an.ext[kc]) / 16 : 0.0f;
    f[19] = lg(info.flops) / 48;
    f[20] = lg(info.min_bytes) / 40;
    // fragmentation of the fused view: labels left after mode merging
    Group ga, gb, gk;
    int64_t t0, t1, t2;
    int merged = 0;
    if (make_group(sorted_by(an.fa, A), an.ext, &A, nullptr, &C, ga, t0)) merged += ga.n;
    if (make_group(sorted_by(an.fb, B), an.ext, nullptr, &B, &C, gb, t1)) merged += gb.n;
    if (make_group(sorted_by(an.con, A), an.ext, &A, &B, nullptr, gk, t2)) merged += gk.n;
    f[21] = (float)merged / 12;
    f[22] = (float)(A.lab.size() + B.lab.size()) / 12;
  }

  int32_t map = mapping;
  int32_t sel_tile = -1;  // tile configuration of the selector's candidate
  if (map == TC_MAP_AUTO) {
    int32_t cand[16], nc = 0;
    float pred[16];
    map = TC_MAP_RECIPE;
    if (selector_predict(P->features, dtype, math, cand, pred, &nc)) {
      const bool class3 = an.cls == 31 || an.cls == 32;
      double kprod = 1.0;
      for (auto l : an.con) kprod *= (double)an.ext[l];
      float best = 0;
      bool found = false;
      for (int i = 0; i < nc; ++i) {
        const int32_t cm = cand[i] & 0xFF, ct = (cand[i] >> 8) - 1;
        const bool feasible =
            cm >= TC_MAP_SLICE_GEMM && cm <= TC_MAP_GER &&
            (class3 || (cm != TC_MAP_SLICE_GEMM && cm != TC_MAP_COPY_GEMM)) &&
            (cm != TC_MAP_COPY_GEMM || an.bat.empty()) &&
            (cm != TC_MAP_GER || kprod <= TC_GER_MAX_K);
        if (feasible && (!found || pred[i] < best)) {
          map = cm;
          sel_tile = ct;
          best = pred[i];
          found = true;
        }
      }
    }
  }
  if (map == TC_MAP_RECIPE)
    map = (an.cls == 1) ? TC_MAP_DOT : (an.cls == 2) ? TC_MAP_GEMV : TC_MAP_FUSED_GEMM;
  const bool is3 = an.cls == 31 || an.cls == 32;
  const bool fp8 = math == TC_MATH_FP8;
  if ((fp8 && (!is3 || map != TC_MAP_FUSED_GEMM || !an.bat.empty())) ||
      (map == TC_MAP_COPY_GEMM && !an.bat.empty())) {
    // the FP8 form is one block-scaled GEMM: Class 3, fused mapping, no batch
    // labels; the COPY baseline's dense copy has no batch labels either
    delete P;
    return TC_ERR_UNSUPPORTED;
  }
  if ((map == TC_MAP_SLICE_GEMM || map == TC_MAP_COPY_GEMM) && !is3) {
    delete P;
    return TC_ERR_UNSUPPORTED;
  }
  const bool gemm_family =
      map == TC_MAP_SLICE_GEMM || map == TC_MAP_FUSED_GEMM || map == TC_MAP_COPY_GEMM;
  const bool tensor_core = math == TC_MATH_BF16 || math == TC_MATH_BF16X3 ||
                           math == TC_MATH_BF16X6 || math == TC_MATH_FP16;
  int32_t kernel = fp8 ? K_GEMM_FP8
                 : gemm_family ? (tensor_core ? K_GEMM_TC : K_GEMM_SIMT)
                 : map == TC_MAP_GER ? K_GER
                               : (map == TC_MAP_GEMV ? K_GEMV : K_DOT);

  // ---- operand roles: the kernel's first operand X provides M
  bool swap = false;
  if (an.cls == 2) {
    swap = an.da == 0;
  } else if (is3) {
    int32_t s1c = C.stride1();
    swap = s1c >= 0 && contains(an.fb, s1c);
  }
  const Tens& X = swap ? B : A;
  const Tens& Y = swap ? A : B;
  const std::vector<int32_t>& fx = swap ? an.fb : an.fa;
  const std::vector<int32_t>& fy = swap ? an.fa : an.fb;
  const std::vector<int32_t>& keep_x = swap ? an.keep_b : an.keep_a;
  const std::vector<int32_t>& keep_y = swap ? an.keep_a : an.keep_b;

  std::vector<int32_t> lm, ln, lk, lb;
  if (map == TC_MAP_SLICE_GEMM) {
    // unsliced free index of each operand -> M, N; the other free indices -> batch;
    // every contracted index is accumulated, the unsliced one varying fastest.
    int32_t mx = -1, ny = -1, kk = -1;
    for (auto l : keep_x) (contains(an.con, l) ? kk : mx) = l;
    for (auto l : keep_y)
      if (!contains(an.con, l)) ny = l;
    if (mx >= 0) lm.push_back(mx);
    if (ny >= 0) ln.push_back(ny);
    for (auto l : fx)
      if (l != mx) lb.push_back(l);
    for (auto l : fy)
      if (l != ny) lb.push_back(l);
    for (auto l : an.bat) lb.push_back(l);
    lb = sorted_by(lb, C);
    if (kk >= 0) lk.push_back(kk);
    for (auto l : sorted_by(an.con, X))
      if (l != kk) lk.push_back(l);
  } else {
    lm = sorted_by(fx, X);
    ln = sorted_by(fy, Y);
    // the FP8 form's scale blocks follow A's strides, whichever operand is first
    lk = sorted_by(an.con, fp8 ? A : X);
    lb = sorted_by(an.bat, C);  // batch labels: one GEMM per value
  }

  // COPY+GEMM: permute the copied operand (the one whose stride-1 index the
  // recipe slices; B when the contraction is Class 3.2) into a dense layout
  // [contracted labels in the GEMM's K order..., its free labels in M/N order].
  Tens Xc, Yc;
  const Tens* Xp = &X;
  const Tens* Yp = &Y;
  P->copy_which = 0;
  if (map == TC_MAP_COPY_GEMM) {
    const char copied = an.copied ? an.copied : 'B';
    const bool copy_y = (copied == 'B') != swap;
    const Tens& src = copy_y ? Y : X;
    if (!copy_y) lk = sorted_by(an.con, Y);  // K order follows the operand left in place
    std::vector<int32_t> order = lk;
    const std::vector<int32_t>& fr = copy_y ? ln : lm;
    order.insert(order.end(), fr.begin(), fr.end());
    Tens& dst = copy_y ? Yc : Xc;
    int64_t acc = 1;
    for (auto l : order) {
      dst.lab.push_back(l);
      dst.ext.push_back(an.ext[l]);
      dst.st.push_back(an.ext[l] > 1 ? acc : 0);
      acc *= std::max<int64_t>(an.ext[l], 1);
    }
    int64_t tot;
    if (!make_group(order, an.ext, &src, nullptr, &dst, P->perm.g, tot)) {
      delete P;
      return TC_ERR_UNSUPPORTED;
    }
    P->perm.total = tot;
    P->perm.in = nullptr;
    P->perm.out = nullptr;
    P->copy_elems = tot;
    P->copy_which = copy_y ? 2 : 1;
    if (copy_y) Yp = &Yc; else Xp = &Xc;
  }

  GemmArgs& g = P->args;
  int64_t M, N, Kt, Bt;
  bool ok = make_group(lm, an.ext, Xp, nullptr, &C, g.gm, M) &&
            make_group(ln, an.ext, nullptr, Yp, &C, g.gn, N) &&
            make_group(lk, an.ext, Xp, Yp, nullptr, g.gk, Kt) &&
            make_group(lb, an.ext, Xp, Yp, &C, g.gb, Bt);
  if (!ok || M > INT_MAX || N > INT_MAX || Kt > INT_MAX || Bt > INT_MAX ||
      (kernel == K_GER && Kt > TC_GER_MAX_K)) {
    delete P;
    return TC_ERR_UNSUPPORTED;
  }
  // group strides must be in the kernel's operand slots: gm uses st[0] (X) and st[2] (C),
  // gn uses st[1] (Y) and st[2], gk uses st[0] and st[1]; batch uses all three.
  g.M = M;
  g.N = N;
  g.K = Kt;
  g.nbatch = Bt;
  g.math = math;
  g.a_contig = (g.gm.n > 0 && g.gm.ext[0] > 1 && g.gm.st[0][0] == 1) ? CONTIG_MN
               : (g.gk.n > 0 && g.gk.ext[0] > 1 && g.gk.st[0][0] == 1) ? CONTIG_K
                                                                       : CONTIG_NONE;
  g.b_contig = (g.gn.n > 0 && g.gn.ext[0] > 1 && g.gn.st[1][0] == 1) ? CONTIG_MN
               : (g.gk.n > 0 && g.gk.ext[0] > 1 && g.gk.st[1][0] == 1) ? CONTIG_K
                                                                       : CONTIG_NONE;
  g.c_contig_m = (g.gm.n > 0 && g.gm.st[2][0] == 1) ? 1 : 0;

  P->mapping = map;
  P->kernel = kernel;
  P->swapped = swap;
  P->empty_out = C.numel() == 0;
  P->empty_k = Kt == 0;
  {
    int64_t tc_;
    std::vector<int32_t> cl = C.lab;
    make_group(cl, an.ext, nullptr, nullptr, &C, P->gc, tc_);
    P->c_elems_span = tc_;
  }

  // ---- tiles and workspace
  int ntiles = kernel == K_GEMM_SIMT ? num_tiles_simt(dtype)
               : kernel == K_GEMM_TC ? num_tiles_tc()
               : kernel == K_GEMM_FP8 ? kFp8Tiles
               : kernel == K_GEMV    ? num_tiles_gemv()
                                     : 1;
  if (tile >= ntiles) {
    delete P;
    return TC_ERR_UNSUPPORTED;
  }
  // packed operands (split once, moved by bulk copies) suit one GEMM unless
  // padding a skinny operand to 128-row tiles would more than double its
  // packed size (beyond 64 MB of slack)
  bool packed_ok = false;
  if (kernel == K_GEMM_TC && Bt == 1) {
    const double terms = (math == TC_MATH_BF16 || math == TC_MATH_FP16) ? 1
                         : math == TC_MATH_BF16X3 ? 2 : 3;
    const double dense = 2.0 * terms * 2.0 * (double)(M + N) * (double)Kt;
    packed_ok = (double)pk_layout(g, math).bytes <= 2.0 * dense + 64.0 * (1 << 20);
  }
  // the selector's tile configuration, where it applies: it was timed with
  // exactly that tile (packed operands too, whatever their padding costs, up
  // to the 2 GB of workspace the timing allowed)
  const bool packed_sel = Bt == 1 && kernel == K_GEMM_TC &&
                          pk_layout(g, math).bytes <= ((size_t)2 << 30);
  if (tile < 0 && sel_tile >= 0 &&
      ((kernel == K_GEMM_TC && (sel_tile != kTilePacked || packed_sel)) ||
       (kernel == K_GEMM_SIMT && sel_tile < num_tiles_simt(dtype))))
    tile = sel_tile;
  const bool packed_tile =
      tile == kTilePacked || tile == kTilePackedWide || tile == kTilePackedPair;
  if (kernel == K_GEMM_TC && packed_tile && Bt > 1) {
    delete P;  // packed operands: one GEMM, no batch group
    return TC_ERR_UNSUPPORTED;
  }
  if (kernel == K_GEMM_TC && tile == kTilePackedWide && math == TC_MATH_BF16X6) {
    delete P;  // wide tiles keep one accumulator: not the FP32-class form
    return TC_ERR_UNSUPPORTED;
  }
  // BF16 / FP16 storage and the FP16 form run only on packed operands (the
  // gathering kernel stages 4-byte elements); a batch of GEMMs of BF16 or FP16
  // data computes on the CUDA cores instead, in FP32 (the products of the
  // stored values are exact there too)
  if (kernel == K_GEMM_TC && (dtype == TC_BF16 || dtype == TC_F16 || math == TC_MATH_FP16)) {
    if (Bt > 1 && dtype != TC_F32 && tile < 0) {
      kernel = K_GEMM_SIMT;
      P->kernel = kernel;
    } else if (Bt > 1 || (tile >= 0 && tile != kTilePacked && tile != kTilePackedWide &&
                          tile != kTilePackedPair)) {
      delete P;
      return TC_ERR_UNSUPPORTED;
    } else if (tile < 0) {
      tile = (M > 128 && N > 128) ? kTilePackedPair : kTilePacked;
    }
  }
  if (tile < 0) {
    if (kernel == K_GEMM_SIMT) {
      // enough 64x64 tiles to fill the GPU twice, else 32x32 tiles; FP64
      // with a long K keeps the 64x64 tile and splits K instead (the 16x16
      // tile, half-filled warps, is left to the selector, which times it)
      int64_t t64 = ((M + 63) / 64) * ((N + 63) / 64) * std::max<int64_t>(Bt, 1);
      tile = t64 >= 2 * 152 ? 0 : 1;
      g.ksplit = 1;
      if (tile == 1 && simt_ksplit(g, dtype, 0) > 1) tile = 0;
    } else if (kernel == K_GEMM_TC) {
      // the gathering kernel for a batch of GEMMs (the slicing mapping) and
      // for skinny operands
      // the one-accumulator forms (BF16, FP16, BF16x3) on CTA pairs when both
      // M and N span two tiles or more (a third fewer operand bytes per SM),
      // BF16x3 on 128 x 256 tiles when only N does
      const bool one_acc = math == TC_MATH_BF16 || math == TC_MATH_FP16 || math == TC_MATH_BF16X3;
      tile = !packed_ok ? 0
             : (one_acc && M > 128 && N > 128) ? kTilePackedPair
             : (math == TC_MATH_BF16X6 && M > 128) ? kTilePackedPair
             : (math == TC_MATH_BF16X3 && N > 128) ? kTilePackedWide : kTilePacked;
    } else if (kernel == K_GEMM_FP8) {
      tile = (M > 128 && N > 128) ? 2 : 0;  // CTA pairs when both span two tiles
    } else {
      tile = 0;
    }
  }
  if (kernel == K_GEMM_FP8 && tile == 1 && !fp8_fusable(g)) {
    delete P;  // in-kernel packing needs a plain first operand, M contiguous
    return TC_ERR_UNSUPPORTED;
  }
  P->tile = tile;
  if (kernel == K_GEMM_TC || kernel == K_GEMM_FP8) {
    if (kernel == K_GEMM_TC) g.chunk_kb = tc_chunk_kb(math, tile);
    // n-tiles fastest when there are few of them: the CTAs that share a panel
    // of the first operand then run at the same time and read it once from HBM
    g.raster = ((N + 127) / 128) <= 16 ? 1 : 0;
  }
  size_t ws = 0;
  if (kernel == K_DOT && M * N * Bt == 1) ws += (size_t)dot_partials(g, tile) * 8;
  ws = (ws + 255) & ~(size_t)255;
  if (P->copy_which) ws += ((size_t)P->copy_elems * es + 255) & ~(size_t)255;
  if (kernel == K_GEMM_FP8) ws += fp8_layout(g).bytes;
  if (kernel == K_GEMM_TC &&
      (tile == kTilePacked || tile == kTilePackedWide || tile == kTilePackedPair))
    ws += pk_layout(g, math).bytes + pk_part_bytes(g, tile);  // packed terms, split-K partials
  if (kernel == K_GEMM_SIMT) {
    g.ksplit = simt_ksplit(g, dtype, tile);
    ws += simt_part_bytes(g, dtype, tile);               // FP64 split-K partial tiles
  }
  P->workspace = ws;

  info.mapping = map;
  info.kernel = kernel;
  info.tile = tile;
  info.swapped = swap ? 1 : 0;
  info.M = M;
  info.N = N;
  info.K = Kt;
  info.batch = Bt;
  info.workspace = ws;
  *out = reinterpret_cast<tc_plan_t>(P);
  return TC_OK;
}

extern "C" tc_status tc_plan_features(tc_plan_t plan, float* out, int32_t n) {
  if (!plan || !out || n < 0) return TC_ERR_INVALID_ARG;
  const Plan* P = reinterpret_cast<const Plan*>(plan);
  for (int32_t i = 0; i < n && i < TC_SELECTOR_FEATURES; ++i) out[i] = P->features[i];
  return TC_OK;
}

extern "C" tc_status tc_plan_layout_advice(tc_plan_t plan, tc_layout_advice* out) {
  if (!plan || !out) return TC_ERR_INVALID_ARG;
  *out = reinterpret_cast<Plan*>(plan)->advice;
  return TC_OK;
}

extern "C" tc_status tc_plan_get_info(tc_plan_t plan, tc_plan_info* info) {
  if (!plan || !info) return TC_ERR_INVALID_ARG;
  *info = reinterpret_cast<Plan*>(plan)->info;
  return TC_OK;
}

extern "C" tc_status tc_plan_destroy(tc_plan_t plan) {
  delete reinterpret_cast<Plan*>(plan);
  return TC_OK;
}

extern "C" const char* tc_status_string(tc_status s) {
  switch (s) {
    case TC_OK: return "ok";
    case TC_ERR_INVALID_ARG: return "invalid argument";
    case TC_ERR_LABEL: return "invalid label set";
    case TC_ERR_EXTENT_MISMATCH: return "extent mismatch";
    case TC_ERR_STRIDE: return "invalid stride";
    case TC_ERR_UNSUPPORTED: return "unsupported";
    case TC_ERR_WORKSPACE: return "workspace too small";
    case TC_ERR_CUDA: return "CUDA error";
    case TC_ERR_TIMEOUT: return "device wait timed out";
    case TC_ERR_NO_SELECTOR: return "no selector loaded";
  }
  return "unknown status";
}

// ---------------------------------------------------------------------------
// Free-index sharding (Sec. 2.4: slicing a free index of C gives independent
// contractions, one per slice).  C's largest free index is split into n
// balanced ranges; shard r contracts the slab of A, B and C where that index
// lies in its range.  No data crosses shards.
// ---------------------------------------------------------------------------
extern "C" tc_status tc_shard_free_index(const tc_tensor_desc* Ad, const tc_tensor_desc* Bd,
                                         const tc_tensor_desc* Cd, int32_t n_shards,
                                         int32_t shard, tc_shard* out) {
  if (!out || n_shards < 1 || shard < 0 || shard >= n_shards) return TC_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  Tens A, B, C;
  tc_status st;
  if ((st = read_desc(Ad, A)) != TC_OK) return st;
  if ((st = read_desc(Bd, B)) != TC_OK) return st;
  if ((st = read_desc(Cd, C)) != TC_OK) return st;
  for (size_t i = 0; i < A.lab.size(); ++i) {  // contracted labels agree too
    const int pb = B.find(A.lab[i]);
    if (pb >= 0 && A.ext[i] != B.ext[pb]) return TC_ERR_EXTENT_MISMATCH;
  }
  int pick = -1;
  for (size_t i = 0; i < C.lab.size(); ++i) {
    const int32_t l = C.lab[i];
    const int pa = A.find(l), pb = B.find(l);
    if (pa < 0 && pb < 0) return TC_ERR_LABEL;
    if ((pa >= 0 && A.ext[pa] != C.ext[i]) || (pb >= 0 && B.ext[pb] != C.ext[i]))
      return TC_ERR_EXTENT_MISMATCH;
    // the largest extent; ties go to the larger stride in C, so that a
    // column-major C is cut into contiguous slabs
    if (pick < 0 || C.ext[i] > C.ext[pick] || (C.ext[i] == C.ext[pick] && C.st[i] > C.st[pick]))
      pick = (int)i;
  }
  if (pick < 0) {  // an order-0 C has no free index: shard 0 computes it
    out->label = -1;
    out->pos_a = out->pos_b = out->pos_c = -1;
    out->begin = 0;
    out->end = shard == 0 ? 1 : 0;
    return TC_OK;
  }
  const int32_t l = C.lab[pick];
  const int64_t E = C.ext[pick];
  out->label = l;
  out->pos_a = A.find(l);
  out->pos_b = B.find(l);
  out->pos_c = pick;
  out->begin = (int64_t)((__int128)shard * E / n_shards);
  out->end = (int64_t)((__int128)(shard + 1) * E / n_shards);
  out->offset_a = out->pos_a >= 0 ? out->begin * A.st[out->pos_a] : 0;
  out->offset_b = out->pos_b >= 0 ? out->begin * B.st[out->pos_b] : 0;
  out->offset_c = out->begin * C.st[pick];
  return TC_OK;
}
