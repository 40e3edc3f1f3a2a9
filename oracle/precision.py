"""Reduced-precision forms of the contraction -- TEST INFRASTRUCTURE ONLY.

Parity: pinned (tests/test_oracle_precision.py: exact reconstruction of FP32
values by three BF16 terms, hand-made rounding ties, the E4M3 and binary16
value tables; binary16 rounding against numpy's float16 cast; the FP8 and
FP16 forms exact on small integers, the FP8 form equivariant under
power-of-two scaling and its GEMM view reproducing the FP64 contraction).

The paper computes in FP64 only (Sec. 4); these forms come from the project's
goal of running the bulk of the multiply on BF16/FP8 tensor cores:

* BF16 rounding is round-to-nearest, ties to the even significand, written
  from that definition: the two BF16 neighbours of x are found by truncating
  and incrementing the 16 low bits of x's FP32 encoding, and the nearer one is
  kept (equal distance: the one whose last significand bit is 0).
* Split terms: x = t0 + t1 + t2 with t0 = bf16(x), t1 = bf16(x - t0),
  t2 = bf16(x - t0 - t1), residuals exact in FP32.
* Forms: BF16 uses t0*t0 only; BF16x3 keeps the three products of a 2-term
  split whose order is <= 1 (a0b0 + a0b1 + a1b0); BF16x6 keeps the six
  products of a 3-term split whose order is <= 2.
* FP8-E4M3 (1 sign, 4 exponent bits with bias 7, 3 significand bits, no
  infinities, largest finite 448): round to nearest, ties to even code,
  saturating to +-448.  Block scales are powers of two 2^e, e the smallest
  integer with amax / 2^e <= 448, but not below -126 (so that 2^e and 2^-e
  are normal FP32 numbers; blocks whose largest value is below about 2^-135
  then round to zero).
* FP16 (IEEE binary16: 1 sign, 5 exponent bits with bias 15, 10 significand
  bits, subnormals, infinities): round to nearest, ties to the even code;
  magnitudes from 65520 (the midpoint above 65504) on overflow to infinity.
  The FP16 form rounds both operands to binary16 and contracts exactly.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import contract

FORMS = {
    "bf16": [(0, 0)],
    "bf16x3": [(0, 0), (0, 1), (1, 0)],
    "bf16x6": [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)],
}
TERMS = {"bf16": 1, "bf16x3": 2, "bf16x6": 3}


def bf16_rne(x) -> np.ndarray:
    """Round float32 values to the nearest BF16 value (ties to even); returns
    float32 arrays holding BF16-representable values.  Finite inputs only."""
    x = np.asarray(x, dtype=np.float32)
    bits = x.view(np.uint32)
    lo_bits = bits & np.uint32(0xFFFF0000)          # truncation toward zero
    hi_bits = lo_bits + np.uint32(0x00010000)       # next BF16 value away from zero
    lo = lo_bits.view(np.float32).astype(np.float64)
    hi = hi_bits.view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    d_lo = np.abs(xd - lo)
    d_hi = np.abs(hi - xd)
    lo_even = (lo_bits & np.uint32(0x00010000)) == 0
    take_hi = (d_hi < d_lo) | ((d_hi == d_lo) & ~lo_even)
    out = np.where(take_hi, hi_bits, lo_bits).view(np.float32)
    return np.where(x == 0, x, out)


def split_bf16(x, nterms: int) -> List[np.ndarray]:
    """x = t0 + t1 + ... with each t a BF16 value; residuals are formed in FP64
    and are exact in FP32."""
    r = np.asarray(x, dtype=np.float32)
    terms = []
    for _ in range(nterms):
        t = bf16_rne(r)
        terms.append(t)
        r = (r.astype(np.float64) - t.astype(np.float64)).astype(np.float32)
    return terms


def contract_form(p, form: str, nthreads: int = 0) -> np.ndarray:
    """FP64 result of the split-product form: the selected term products are
    contracted exactly-rounded in FP64 (tco) and summed.  p.A, p.B hold FP32."""
    n = TERMS[form]
    ta = split_bf16(p.A.data, n)
    tb = split_bf16(p.B.data, n)
    acc = None
    import copy
    for i, j in FORMS[form]:
        A = copy.copy(p.A)
        B = copy.copy(p.B)
        A.data, B.data = ta[i], tb[j]
        r = contract(A, B, p.C, 1.0, 0.0, nthreads=nthreads)
        acc = r if acc is None else acc + r
    C = copy.copy(p.C)
    out = p.alpha * acc
    if p.beta != 0:
        out = out + p.beta * np.asarray(p.C.data, np.float64)
    return out


# ---------------------------------------------------------------- FP8 E4M3

def e4m3_values() -> Tuple[np.ndarray, np.ndarray]:
    """All non-negative finite E4M3 values with their 7-bit codes, sorted."""
    codes, vals = [], []
    for code in range(0x7F):              # 0x7F is NaN
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0:
            v = (m / 8.0) * 2.0 ** (-6)
        else:
            v = (1.0 + m / 8.0) * 2.0 ** (e - 7)
        codes.append(code)
        vals.append(v)
    order = np.argsort(vals, kind="stable")
    return np.asarray(vals)[order], np.asarray(codes)[order]


_E4M3_VALS, _E4M3_CODES = e4m3_values()
E4M3_MAX = 448.0


def e4m3_rne(x) -> np.ndarray:
    """Round to the nearest E4M3 value, ties to the even code, saturating."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.minimum(np.abs(x), E4M3_MAX)
    vals, codes = _E4M3_VALS, _E4M3_CODES
    hi_i = np.clip(np.searchsorted(vals, ax, side="left"), 0, len(vals) - 1)
    lo_i = np.clip(hi_i - 1, 0, len(vals) - 1)
    lo, hi = vals[lo_i], vals[hi_i]
    d_lo, d_hi = ax - lo, hi - ax
    even_hi = (codes[hi_i] & 1) == 0
    take_hi = (d_hi < d_lo) | ((d_hi == d_lo) & even_hi)
    q = np.where(take_hi, hi, lo)
    q = np.where(ax == vals[hi_i], vals[hi_i], q)
    return np.copysign(q, x)


E_MIN = -126   # scales stay normal FP32 numbers (2^-126 .. 2^120)


def pow2_scale_exponent(amax) -> np.ndarray:
    """Smallest integer e >= -126 with amax / 2^e <= 448 (-126 for amax == 0)."""
    amax = np.asarray(amax, dtype=np.float64)
    e = np.ceil(np.log2(np.where(amax > 0, amax, 1.0) / E4M3_MAX)).astype(np.int64)
    # correct possible off-by-one of log2 at exact powers of two
    e = np.where(amax / np.exp2(e - 1) <= E4M3_MAX, e - 1, e)
    e = np.where(amax / np.exp2(e) > E4M3_MAX, e + 1, e)
    return np.maximum(np.where(amax > 0, e, E_MIN), E_MIN)


def quantize_rows_e4m3(mat: np.ndarray, block: int = 128):
    """Quantise a [rows, K] matrix with one power-of-two scale per (row, block
    of `block` consecutive K).  Returns (dequantised values, exponents)."""
    rows, K = mat.shape
    nb = (K + block - 1) // block
    out = np.zeros_like(mat, dtype=np.float64)
    exps = np.zeros((rows, nb), dtype=np.int64)
    for bi in range(nb):
        blk = mat[:, bi * block:(bi + 1) * block].astype(np.float64)
        e = pow2_scale_exponent(np.max(np.abs(blk), axis=1))
        s = np.exp2(e.astype(np.float64))[:, None]
        out[:, bi * block:(bi + 1) * block] = e4m3_rne(blk / s) * s
        exps[:, bi] = e
    return out, exps


# ------------------------------------------------ FP8 form of a contraction

def k_order(p):
    """Contracted labels in the order that defines the FP8 form's K blocks:
    ascending stride in A, ties kept in A's label order."""
    A, B = p.A, p.B
    con = [l for l in A.labels if l in B.labels]
    sa = dict(zip(A.labels, A.strides))
    pos = {l: k for k, l in enumerate(A.labels)}
    return sorted(con, key=lambda l: (sa[l], pos[l]))


def gemm_view(p):
    """Dense matrices of the contraction's GEMM view: A_mat [M, K], B_mat [K, N]
    with rows m enumerated column-major over A's free labels (A's order), rows
    n over B's free labels (B's order), and K column-major over the contracted
    labels sorted by ascending stride in A (ties: position in A).  Returns
    (A_mat, B_mat, m_labels, n_labels, k_labels)."""
    A, B = p.A, p.B
    fa = [l for l in A.labels if l not in B.labels]
    fb = [l for l in B.labels if l not in A.labels]
    kl = k_order(p)
    ext = dict(zip(A.labels, A.extents))
    ext.update(zip(B.labels, B.extents))

    def offsets(t, labels):
        st = dict(zip(t.labels, t.strides))
        if not labels:
            return np.zeros(1, dtype=np.int64)
        grids = np.meshgrid(*[np.arange(ext[l], dtype=np.int64) * st[l] for l in labels],
                            indexing="ij")
        return np.asarray(sum(grids)).reshape(-1, order="F")

    am = offsets(A, fa)[:, None] + offsets(A, kl)[None, :]
    bm = offsets(B, kl)[:, None] + offsets(B, fb)[None, :]
    return (np.asarray(A.data, np.float64)[am], np.asarray(B.data, np.float64)[bm], fa, fb, kl)


def contract_fp8(p, block: int = 128):
    """FP64 result of the FP8 form: each operand row (a free multi-index) is
    cut into blocks of `block` consecutive K (in the gemm_view order), scaled by
    the block's power of two 2^e (smallest e with amax / 2^e <= 448) and
    rounded to E4M3; the dequantised products are summed exactly (FP64).
    Returns a buffer laid out like p.C."""
    Am, Bm, fa, fb, kl = gemm_view(p)
    qa, _ = quantize_rows_e4m3(Am, block)
    qb, _ = quantize_rows_e4m3(Bm.T.copy(), block)
    Cm = qa @ qb.T                                    # [M, N], FP64
    C = p.C
    ext = dict(zip(p.A.labels, p.A.extents))
    ext.update(zip(p.B.labels, p.B.extents))
    st = dict(zip(C.labels, C.strides))

    def offs(labels):
        if not labels:
            return np.zeros(1, dtype=np.int64)
        grids = np.meshgrid(*[np.arange(ext[l], dtype=np.int64) * st[l] for l in labels],
                            indexing="ij")
        return np.asarray(sum(grids)).reshape(-1, order="F")

    idx = offs(fa)[:, None] + offs(fb)[None, :]
    out = np.array(np.asarray(C.data, np.float64), copy=True)
    val = p.alpha * Cm
    if p.beta != 0:
        val = val + p.beta * out[idx]
    out[idx] = val
    return out


# ------------------------------------------------------- FP16 (IEEE binary16)

def f16_values() -> Tuple[np.ndarray, np.ndarray]:
    """All non-negative finite binary16 values with their 15-bit codes, in
    increasing order: 1 sign bit, 5 exponent bits with bias 15, 10 significand
    bits; exponent field 0 holds the subnormals (m / 2^10) 2^-14, field 31 the
    infinities and NaNs (left out)."""
    codes = np.arange(0x7C00, dtype=np.int64)
    e = codes >> 10
    m = (codes & 0x3FF).astype(np.float64)
    vals = np.where(e == 0, m / 1024.0 * 2.0 ** (-14),
                    (1.0 + m / 1024.0) * np.exp2((e - 15).astype(np.float64)))
    return vals, codes


_F16_VALS, _F16_CODES = f16_values()
F16_MAX = 65504.0
F16_OVERFLOW = 65520.0   # midpoint of 65504 and 2^16: from here on, infinity


def f16_rne(x) -> np.ndarray:
    """Round to the nearest binary16 value, ties to the even code (IEEE 754
    round-to-nearest-even).  Magnitudes of F16_OVERFLOW or more become
    infinite: that midpoint is a tie between the odd code of 65504 and the
    even code of infinity.  Returns float64 values."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    vals, codes = _F16_VALS, _F16_CODES
    hi_i = np.clip(np.searchsorted(vals, ax, side="left"), 0, len(vals) - 1)
    lo_i = np.clip(hi_i - 1, 0, len(vals) - 1)
    lo, hi = vals[lo_i], vals[hi_i]
    d_lo, d_hi = ax - lo, hi - ax
    even_hi = (codes[hi_i] & 1) == 0
    take_hi = (d_hi < d_lo) | ((d_hi == d_lo) & even_hi)
    q = np.where(take_hi, hi, lo)
    q = np.where(ax == vals[hi_i], vals[hi_i], q)
    q = np.where(ax > F16_MAX, np.where(ax >= F16_OVERFLOW, np.inf, F16_MAX), q)
    return np.copysign(q, x)


def contract_f16(p, nthreads: int = 0) -> np.ndarray:
    """FP64 result of the FP16 form: every element of A and B rounded to
    binary16 (f16_rne), the rounded operands contracted exactly-rounded in
    FP64.  The tensor cores then only add accumulation error: a product of
    two binary16 values (11-bit significands) is exact in FP32."""
    import copy
    A, B = copy.copy(p.A), copy.copy(p.B)
    A.data = f16_rne(p.A.data)
    B.data = f16_rne(p.B.data)
    return contract(A, B, p.C, p.alpha, p.beta, nthreads=nthreads)
