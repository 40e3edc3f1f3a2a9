"""Helpers of the GPU parity tests: run a tcsynth.Problem through the C ABI and
compute sampled oracle outputs for problems too large for the full oracle."""
from __future__ import annotations

import copy
import itertools

import numpy as np

import oracle
import tcsynth as ts

TOL_FP64 = 1e-12        # relative Frobenius, FP64 path


def addressed_index(t) -> np.ndarray:
    """Flat buffer positions of every element of tensor t, column-major order."""
    if t.order == 0:
        return np.zeros(1, dtype=np.int64)
    grids = np.meshgrid(*[np.arange(e, dtype=np.int64) * s for e, s in zip(t.extents, t.strides)],
                        indexing="ij")
    tot = sum(grids)
    return np.asarray(tot).reshape(-1, order="F")


def run(p, math="fp64", mapping="auto", tile=-1, alpha=None, beta=None, stream=None,
        plan_out=None):
    """Run problem p on cuda:0; returns the full C buffer (float64 copy)."""
    import torch
    from paper_1307_2100_gb300 import Contraction
    dt = "f64" if p.A.data.dtype == np.float64 else "f32"
    alpha = p.alpha if alpha is None else alpha
    beta = p.beta if beta is None else beta
    plan = Contraction((p.A.labels, p.A.extents, p.A.strides),
                       (p.B.labels, p.B.extents, p.B.strides),
                       (p.C.labels, p.C.extents, p.C.strides), dt, math, mapping, tile)
    if plan_out is not None:
        plan_out.append(plan.info.as_dict())
    dev = torch.device("cuda:0")
    A = torch.from_numpy(np.ascontiguousarray(p.A.data)).to(dev)
    B = torch.from_numpy(np.ascontiguousarray(p.B.data)).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(p.C.data)).to(dev)
    if A.numel() == 0:
        A = torch.zeros(1, dtype=C.dtype, device=dev)
    if B.numel() == 0:
        B = torch.zeros(1, dtype=C.dtype, device=dev)
    if C.numel() == 0:
        C = torch.zeros(1, dtype=A.dtype, device=dev)
    plan(A, B, C, alpha, beta, stream)
    torch.cuda.synchronize()
    out = C.cpu().numpy().astype(np.float64)
    return out[: p.C.data.size] if p.C.data.size else out[:0]


def _sub_operand(t, fix, con):
    """The contracted sub-tensor of operand t at fixed free-label values,
    gathered into a compact column-major array (labels, extents, strides, data)."""
    off = sum(fix[l] * s for l, s in zip(t.labels, t.strides) if l in fix)
    keep = [k for k, l in enumerate(t.labels) if l in con]
    labels = [t.labels[k] for k in keep]
    ext = [int(t.extents[k]) for k in keep]
    st = [int(t.strides[k]) for k in keep]
    if ext:
        grids = np.meshgrid(*[np.arange(e, dtype=np.int64) * s for e, s in zip(ext, st)],
                            indexing="ij")
        idx = (off + sum(grids)).reshape(-1, order="F")
    else:
        idx = np.array([off], dtype=np.int64)
    return labels, ext, ts.col_major(ext), np.asarray(t.data[idx], np.float64)


def oracle_full(p, **kw):
    return oracle.contract_problem(p, **kw)


def compare(got, ref, C):
    """Relative Frobenius error over the addressed elements of C."""
    idx = addressed_index(C) if C.numel else np.zeros(0, dtype=np.int64)
    return oracle.rel_fro(got[idx], ref[idx])


def sample_outputs(p, samples):
    """Oracle values of selected output elements: for each output multi-index
    the free labels are fixed, the operands' contracted sub-tensors gathered,
    and the oracle contracts them into a scalar."""
    con = [l for l in p.A.labels if l in p.B.labels]
    vals = []
    for cidx in samples:
        fix = dict(zip(p.C.labels, cidx))
        (la, ea, sa, a) = _sub_operand(p.A, fix, con)
        (lb, eb, sb, b) = _sub_operand(p.B, fix, con)
        c = np.zeros(1)
        if p.beta != 0:
            c[0] = float(p.C.data[sum(i * s for i, s in zip(cidx, p.C.strides))])
        oracle.contract_raw(la, ea, sa, a, lb, eb, sb, b, [], [], [], c, p.alpha, p.beta)
        vals.append(c[0])
    return np.array(vals)


def random_output_indices(p, n, seed=0):
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(0, e)) for e in p.C.extents) for _ in range(n)]


def gather(buf, C, samples):
    return np.array([buf[sum(i * s for i, s in zip(cidx, C.strides))] for cidx in samples])


def sample_outputs_form(p, samples, form):
    """Oracle values of selected outputs for a split-product form: each
    sample's gathered operand sub-tensors are split into BF16 terms
    (oracle.precision) and the form's term products are contracted in FP64
    and summed."""
    from oracle import precision as op
    con = [l for l in p.A.labels if l in p.B.labels]
    nt = op.TERMS[form]
    vals = []
    for cidx in samples:
        fix = dict(zip(p.C.labels, cidx))
        la, ea, sa, a = _sub_operand(p.A, fix, con)
        lb, eb, sb, b = _sub_operand(p.B, fix, con)
        ta = op.split_bf16(a.astype(np.float32), nt)
        tb = op.split_bf16(b.astype(np.float32), nt)
        acc = 0.0
        for i, j in op.FORMS[form]:
            c = np.zeros(1)
            oracle.contract_raw(la, ea, sa, ta[i], lb, eb, sb, tb[j], [], [], [], c, 1.0, 0.0)
            acc += c[0]
        v = p.alpha * acc
        if p.beta != 0:
            v += p.beta * float(p.C.data[sum(i * s for i, s in zip(cidx, p.C.strides))])
        vals.append(v)
    return np.array(vals)


NPROD = {"bf16": 1, "bf16x3": 3, "bf16x6": 6}
SPLIT_ERR = {"bf16": 2.0 ** -8, "bf16x3": 3 * 2.0 ** -18, "bf16x6": 4 * 2.0 ** -26}


def magnitude(p):
    """Oracle contraction of |A| and |B|: the elementwise scale sum |a||b| that
    worst-case rounding bounds are proportional to."""
    import copy
    A, B = copy.copy(p.A), copy.copy(p.B)
    A.data = np.abs(np.asarray(p.A.data, np.float64))
    B.data = np.abs(np.asarray(p.B.data, np.float64))
    C = copy.copy(p.C)
    return oracle.contract(A, B, C, abs(p.alpha), 0.0)


def tc_bounds(p, form, chunk_k=256, single=False):
    """(accumulation bound, total bound) as multiples of sum |a||b| for the
    tensor-core forms.  The tensor cores add each 16-product block into FP32
    with an error of at most one unit of the running sum (2^-23 relative):
    the main product is summed over one K-chunk, the correction products
    (2^-8 smaller) over all of K; BF16 keeps one accumulator over all of K.
    The split error of the form adds to that: 2^-8 (BF16), 3*2^-18 (the
    missing a1*b1 and the 2-term residuals, BF16x3), 4*2^-26 (products of
    order >= 3, BF16x6).  single: every product of every block goes into one
    accumulator over all of K (the wide-tile kernel), (K/16) NPROD + 1 units."""
    K = 1
    for l, e in zip(p.A.labels, p.A.extents):
        if l in p.B.labels:
            K *= int(e)
    u = 2.0 ** -23
    if single:
        acc = (K / 16 * NPROD[form] + 1) * u
    elif form == "bf16":
        acc = (K / 16 + 1) * u
    else:
        acc = (min(K, chunk_k) / 16 + 1) * u + (K / 16 + 1) * (NPROD[form] - 1) * u * 2.0 ** -8
    return acc, acc + SPLIT_ERR[form]


def within(got, ref, mag, C, c):
    """||got - ref||_F <= c * ||sum |a||b| ||_F over the addressed elements of C."""
    idx = addressed_index(C) if C.numel else np.zeros(0, dtype=np.int64)
    d = np.linalg.norm((np.asarray(got)[idx] - np.asarray(ref)[idx]).ravel())
    return d <= c * np.linalg.norm(np.asarray(mag)[idx].ravel()) + 1e-300, d


def _k_row(t, fix, kl, ext):
    """Operand t's values along the contracted labels kl (first fastest) at
    fixed free-label values."""
    st = dict(zip(t.labels, t.strides))
    off = sum(fix[l] * st[l] for l in t.labels if l in fix)
    if not kl:
        return np.asarray([t.data[off]], np.float64)
    grids = np.meshgrid(*[np.arange(ext[l], dtype=np.int64) * st[l] for l in kl], indexing="ij")
    idx = (off + sum(grids)).reshape(-1, order="F")
    return np.asarray(t.data[idx], np.float64)


def sample_outputs_fp8(p, samples, block=128):
    """Oracle values of selected outputs of the FP8 form: the sample's row of A
    and column of B along the K order are quantised per block
    (oracle.precision) and their dequantised products summed in FP64."""
    from oracle import precision as op
    kl = op.k_order(p)
    ext = dict(zip(p.A.labels, p.A.extents))
    ext.update(zip(p.B.labels, p.B.extents))
    vals = []
    for cidx in samples:
        fix = dict(zip(p.C.labels, cidx))
        a = _k_row(p.A, fix, kl, ext)
        b = _k_row(p.B, fix, kl, ext)
        qa, _ = op.quantize_rows_e4m3(a[None, :], block)
        qb, _ = op.quantize_rows_e4m3(b[None, :], block)
        v = p.alpha * float(qa[0] @ qb[0])
        if p.beta != 0:
            v += p.beta * float(p.C.data[sum(i * s for i, s in zip(cidx, p.C.strides))])
        vals.append(v)
    return np.array(vals)


def fp8_bound(p, block=128):
    """Accumulation bound of the FP8 kernel against the FP8 oracle, as a
    multiple of sum |qa||qb| (<= 1.13 sum |a||b|, E4M3 rounding being <= 2^-4
    relative).  The scaled products are exact; the block-scaled tensor cores
    add each K = 32 step into one FP32 accumulator over all of K (allowed two
    units of the running sum, 2^-22, per step), then alpha/beta round once."""
    K = 1
    for l, e in zip(p.A.labels, p.A.extents):
        if l in p.B.labels:
            K *= int(e)
    return 1.13 * ((K / 32 + 1) * 2.0 ** -22 + 2.0 ** -23)
