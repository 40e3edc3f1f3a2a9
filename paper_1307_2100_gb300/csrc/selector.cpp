// selector.cpp -- the learned mapping selector on the host: loading a trained
// network and predicting each candidate's log2 runtime for tc_plan(AUTO).
//
// File layout (little-endian), written by paper_1307_2100_gb300/selector.py:
//   char   magic[8]  = "TCSEL01\0"
//   int32  n_in, n_hidden, n_out, dtype, math
//   int32  cand[n_out]                 tc_mapping of each output
//   float  lo[n_in], hi[n_in]          feature range seen in training
//   float  mean[n_in], scale[n_in]     x_net = (x - mean) * scale
//   float  y_mean, y_scale             log2 time = y_net * y_scale + y_mean
//   uint16 params[n]                   FP16 W1, b1, W2, b2, W3, b3 (row-major)
// The forward pass uses the FP16 weights widened to FP32 with FP32
// accumulation, the arithmetic of the library's network kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "tc_internal.h"

namespace tc {
namespace {

struct Selector {
  int32_t n_in = 0, n_hidden = 0, n_out = 0, dtype = 0, math = 0;
  std::vector<int32_t> cand;
  std::vector<float> lo, hi, mean, scale;
  float y_mean = 0, y_scale = 1;
  std::vector<float> W1, b1, W2, b2, W3, b3;
};

// One selector per (storage type, math form); the most recently loaded one
// answers tc_selector_predict.
std::mutex g_mu;
constexpr int kMaxSelectors = 8;
Selector* g_sels[kMaxSelectors] = {};
Selector* g_last = nullptr;

Selector* find(int32_t dtype, int32_t math) {
  for (Selector* s : g_sels)
    if (s && s->dtype == dtype && s->math == math) return s;
  return nullptr;
}

float half_to_float(uint16_t h) {
  const uint32_t sign = (uint32_t)(h & 0x8000u) << 16;
  const uint32_t exp = (h >> 10) & 0x1Fu;
  const uint32_t man = h & 0x3FFu;
  float v;
  if (exp == 0) {
    v = std::ldexp((float)man, -24);  // subnormal (or zero)
  } else if (exp == 31) {
    v = man ? NAN : INFINITY;
  } else {
    v = std::ldexp((float)(man | 0x400u), (int)exp - 25);
  }
  uint32_t bits;
  std::memcpy(&bits, &v, 4);
  bits |= sign;
  std::memcpy(&v, &bits, 4);
  return v;
}

template <class T>
bool rd(FILE* f, T* p, size_t n) {
  return std::fread(p, sizeof(T), n, f) == n;
}

void forward(const Selector& S, const float* x, float* y) {
  const int F = S.n_in, H = S.n_hidden, C = S.n_out;
  std::vector<float> xn(F), h1(H), h2(H);
  for (int i = 0; i < F; ++i) xn[i] = (x[i] - S.mean[i]) * S.scale[i];
  for (int o = 0; o < H; ++o) {
    float s = S.b1[o];
    for (int i = 0; i < F; ++i) s = std::fma(xn[i], S.W1[(size_t)o * F + i], s);
    h1[o] = s > 0 ? s : 0;
  }
  for (int o = 0; o < H; ++o) {
    float s = S.b2[o];
    for (int i = 0; i < H; ++i) s = std::fma(h1[i], S.W2[(size_t)o * H + i], s);
    h2[o] = s > 0 ? s : 0;
  }
  for (int o = 0; o < C; ++o) {
    float s = S.b3[o];
    for (int i = 0; i < H; ++i) s = std::fma(h2[i], S.W3[(size_t)o * H + i], s);
    y[o] = s * S.y_scale + S.y_mean;
  }
}

}  // namespace

bool selector_predict(const float* features, tc_dtype dtype, tc_math math, int32_t* cand,
                      float* pred, int32_t* n_cand) {
  std::lock_guard<std::mutex> lock(g_mu);
  const Selector* sp = find(dtype, math);
  if (!sp) return false;
  const Selector& S = *sp;
  if (S.n_in != TC_SELECTOR_FEATURES || S.n_out > 16) return false;
  for (int i = 0; i < S.n_in; ++i) {
    const float margin = 0.05f * (S.hi[i] - S.lo[i]) + 1e-6f;
    if (features[i] < S.lo[i] - margin || features[i] > S.hi[i] + margin) return false;
  }
  forward(S, features, pred);
  for (int i = 0; i < S.n_out; ++i) cand[i] = S.cand[i];
  *n_cand = S.n_out;
  return true;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_selector_load(const char* path) {
  if (!path) return TC_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return TC_ERR_INVALID_ARG;
  Selector* S = new Selector();
  char magic[8];
  bool ok = rd(f, magic, 8) && std::memcmp(magic, "TCSEL01", 8) == 0 && rd(f, &S->n_in, 1) &&
            rd(f, &S->n_hidden, 1) && rd(f, &S->n_out, 1) && rd(f, &S->dtype, 1) &&
            rd(f, &S->math, 1);
  ok = ok && S->n_in > 0 && S->n_in <= 4096 && S->n_hidden > 0 && S->n_hidden <= 4096 &&
       S->n_out > 0 && S->n_out <= 16;
  if (ok) {
    const int F = S->n_in, H = S->n_hidden, C = S->n_out;
    S->cand.resize(C);
    S->lo.resize(F);
    S->hi.resize(F);
    S->mean.resize(F);
    S->scale.resize(F);
    ok = rd(f, S->cand.data(), C) && rd(f, S->lo.data(), F) && rd(f, S->hi.data(), F) &&
         rd(f, S->mean.data(), F) && rd(f, S->scale.data(), F) && rd(f, &S->y_mean, 1) &&
         rd(f, &S->y_scale, 1);
    const size_t sz[6] = {(size_t)H * F, (size_t)H, (size_t)H * H, (size_t)H, (size_t)C * H,
                          (size_t)C};
    std::vector<float>* dst[6] = {&S->W1, &S->b1, &S->W2, &S->b2, &S->W3, &S->b3};
    for (int i = 0; i < 6 && ok; ++i) {
      std::vector<uint16_t> h(sz[i]);
      ok = rd(f, h.data(), sz[i]);
      dst[i]->resize(sz[i]);
      for (size_t k = 0; k < sz[i] && ok; ++k) (*dst[i])[k] = half_to_float(h[k]);
    }
    for (int i = 0; i < C && ok; ++i) {  // TC_SELECTOR_CANDIDATE(mapping, tile), tile -1..14
      const int32_t m = S->cand[i] & 0xFF, t = S->cand[i] >> 8;
      ok = m >= TC_MAP_SLICE_GEMM && m <= TC_MAP_GER && t >= 0 && t <= 15;
    }
    uint8_t extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;  // nothing after the parameters
  }
  std::fclose(f);
  if (!ok) {
    delete S;
    return TC_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  int slot = -1;
  for (int i = 0; i < kMaxSelectors; ++i)
    if (g_sels[i] && g_sels[i]->dtype == S->dtype && g_sels[i]->math == S->math) slot = i;
  for (int i = 0; i < kMaxSelectors && slot < 0; ++i)
    if (!g_sels[i]) slot = i;
  if (slot < 0) {
    delete S;
    return TC_ERR_UNSUPPORTED;  // selectors for kMaxSelectors forms are loaded already
  }
  delete g_sels[slot];
  g_sels[slot] = S;
  g_last = S;
  return TC_OK;
}

extern "C" tc_status tc_selector_unload(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (Selector*& s : g_sels) {
    delete s;
    s = nullptr;
  }
  g_last = nullptr;
  return TC_OK;
}

extern "C" tc_status tc_selector_predict(const float* features, int32_t n, float* out,
                                         int32_t* cand, int32_t* n_cand) {
  if (!features || !out || !cand || !n_cand || n < 0) return TC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_last) return TC_ERR_NO_SELECTOR;
  const Selector& S = *g_last;
  for (int32_t i = 0; i < n; ++i) forward(S, features + (size_t)i * S.n_in, out + (size_t)i * S.n_out);
  for (int i = 0; i < S.n_out; ++i) cand[i] = S.cand[i];
  *n_cand = S.n_out;
  return TC_OK;
}
