"""Seeded synthetic inputs for binary tensor contractions.

This module is shared by the oracle's tests, the GPU parity tests and the
benchmark.  It only builds descriptors (labels, extents, strides) and fills
buffers with seeded random numbers; it performs no contraction arithmetic.

Conventions (Sec. 2.4 of the paper): a tensor is a list of labelled indices,
each with an extent, stored with per-index strides counted in elements.  The
default storage is column-major: the first index has stride 1 and each later
stride is the previous stride times the previous extent.  Labels are small
non-negative integers; the helpers accept one-character strings and map them
with ord().
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

BASE_SEED = 20130708


def lab(s) -> List[int]:
    """Map 'aibc' or ['a', 'i'] or [97, 105] to a list of integer labels."""
    if isinstance(s, str):
        return [ord(ch) for ch in s]
    return [ord(x) if isinstance(x, str) else int(x) for x in s]


def col_major(extents: Sequence[int]) -> List[int]:
    """Column-major element strides: stride[0] = 1, stride[k+1] = stride[k]*extent[k]."""
    st, acc = [], 1
    for e in extents:
        st.append(acc)
        acc *= max(int(e), 1)
    return st


def storage_strides(extents: Sequence[int], order: Sequence[int]) -> List[int]:
    """Strides of a dense tensor whose storage visits index positions in `order`
    (order[0] fastest).  order = range(n) is column-major."""
    st = [0] * len(extents)
    acc = 1
    for pos in order:
        st[pos] = acc
        acc *= max(int(extents[pos]), 1)
    return st


def span(extents: Sequence[int], strides: Sequence[int]) -> int:
    """Number of elements a buffer needs to hold every addressed element."""
    if any(int(e) == 0 for e in extents):
        return 0
    return 1 + sum((int(e) - 1) * int(s) for e, s in zip(extents, strides))


@dataclass
class Tensor:
    labels: List[int]
    extents: List[int]
    strides: List[int]
    data: np.ndarray  # flat buffer of span(extents, strides) elements

    @property
    def order(self) -> int:
        return len(self.labels)

    @property
    def numel(self) -> int:
        n = 1
        for e in self.extents:
            n *= int(e)
        return n


@dataclass
class Problem:
    """C[labels_c] = alpha * sum_contracted A[labels_a] * B[labels_b] + beta * C."""
    name: str
    A: Tensor
    B: Tensor
    C: Tensor
    alpha: float = 1.0
    beta: float = 0.0
    meta: Dict = field(default_factory=dict)

    def flops(self) -> float:
        ext = {}
        for t in (self.A, self.B, self.C):
            for l, e in zip(t.labels, t.extents):
                ext[l] = int(e)
        f = 2.0
        for e in ext.values():
            f *= e
        return f

    def min_bytes(self) -> float:
        esz = self.A.data.dtype.itemsize
        n = self.A.numel + self.B.numel + self.C.numel * (2 if self.beta != 0 else 1)
        return float(n * esz)


def fill(rng: np.random.Generator, n: int, dist: str = "uniform", dtype=np.float64,
         lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    if dist == "uniform":
        x = rng.uniform(lo, hi, size=n)
    elif dist == "normal":
        x = rng.standard_normal(size=n)
    elif dist == "int":
        x = rng.integers(int(lo), int(hi) + 1, size=n).astype(np.float64)
    elif dist == "ones":
        x = np.ones(n)
    else:
        raise ValueError(dist)
    return x.astype(dtype)


def make_tensor(rng, labels, extents: Dict[int, int], order=None, dist="uniform",
                dtype=np.float64, lo=-1.0, hi=1.0, strides=None) -> Tensor:
    labels = lab(labels)
    ext = [int(extents[l]) for l in labels]
    if strides is None:
        strides = col_major(ext) if order is None else storage_strides(ext, order)
    n = span(ext, strides)
    return Tensor(labels, ext, list(strides), fill(rng, n, dist, dtype, lo, hi))


def empty_output(labels, extents: Dict[int, int], dtype=np.float64, strides=None,
                 fill_value=np.nan) -> Tensor:
    labels = lab(labels)
    ext = [int(extents[l]) for l in labels]
    if strides is None:
        strides = col_major(ext)
    n = span(ext, strides)
    return Tensor(labels, ext, list(strides), np.full(n, fill_value, dtype=dtype))


def problem(name, la, lb, lc, extents, seed, dist="uniform", dtype=np.float64,
            order_a=None, order_b=None, order_c=None, lo=-1.0, hi=1.0) -> Problem:
    """Build a seeded problem; `extents` maps one-character labels to sizes."""
    ext = {lab(k)[0] if isinstance(k, str) else int(k): int(v) for k, v in extents.items()}
    rng = np.random.Generator(np.random.PCG64(seed))
    A = make_tensor(rng, la, ext, order_a, dist, dtype, lo, hi)
    B = make_tensor(rng, lb, ext, order_b, dist, dtype, lo, hi)
    lcl = lab(lc)
    cext = [ext[l] for l in lcl]
    cst = col_major(cext) if order_c is None else storage_strides(cext, order_c)
    C = empty_output(lcl, ext, dtype, cst)
    return Problem(name, A, B, C, meta={"seed": seed, "dist": dist})


# ---------------------------------------------------------------------------
# The workloads.  Shapes follow the paper's examples: the single contraction of
# case (iii) in Eq. (tenscases), the two double contractions of Eq. (xy) and a
# Class 2 contraction; the CCD-shaped precision workload follows Sec. 4.2.
# ---------------------------------------------------------------------------

def slice_gemm_48(seed=BASE_SEED + 0, dist="uniform") -> Problem:
    """C[a,b,c] = sum_i A[a,i,c] B[i,b], every extent 48 (case (iii) of Eq. tenscases)."""
    return problem("slice_gemm_48", "aic", "ib", "abc", dict(a=48, b=48, c=48, i=48), seed, dist)


def direct_gemm_64(seed=BASE_SEED + 1, n=64, dist="uniform") -> Problem:
    """C[a,b,c,d] = sum_{i,j} A[a,i,j,b] B[i,j,c,d], every extent 64 (Eq. xy (a) pattern, Class 3.2)."""
    return problem("direct_gemm_64", "aijb", "ijcd", "abcd",
                   dict(a=n, b=n, c=n, d=n, i=n, j=n), seed, dist)


def fused_permute_48(seed=BASE_SEED + 1, n=48, dist="uniform") -> Problem:
    """C[a,b,c,d] = sum_{i,j} A[i,a,j,b] B[j,c,i,d], every extent 48 (Eq. xy (b), Class 3.1)."""
    return problem("fused_permute_48", "iajb", "jcid", "abcd",
                   dict(a=n, b=n, c=n, d=n, i=n, j=n), seed + 100, dist)


def gemv_1024(seed=BASE_SEED + 1, a=1024, b=1024, i=2048, dist="uniform") -> Problem:
    """C[a,b] = sum_i A[a,i,b] B[i] with a=b=1024, i=2048 (Class 2)."""
    return problem("gemv_1024", "aib", "i", "ab", dict(a=a, b=b, i=i), seed + 200, dist)


def precision_ccd(seed=BASE_SEED + 2, v=128, o=32, dtype=np.float32) -> Problem:
    """C[a,b,i,j] = sum_{e,f} A[a,b,e,f] B[e,f,i,j]; a=b=e=f=v, i=j=o.

    A = N(0,1) / (1 + |a - e|) (0-based indices), B = N(0,1): decaying
    magnitudes across the virtual index pair as in CCD amplitudes (Sec. 4.2).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ext = dict(zip(lab("abefij"), [v, v, v, v, o, o]))
    A = make_tensor(rng, "abef", ext, dist="normal", dtype=np.float64)
    a_idx = np.arange(v)
    scale = 1.0 / (1.0 + np.abs(a_idx[:, None] - a_idx[None, :]))  # [a, e]
    Av = A.data.reshape(v, v, v, v, order="F") * scale[:, None, :, None]
    A.data = np.asfortranarray(Av).reshape(-1, order="F").astype(dtype)
    B = make_tensor(rng, "efij", ext, dist="normal", dtype=dtype)
    C = empty_output("abij", ext, dtype)
    return Problem("precision_ccd", A, B, C, meta={"seed": seed, "dist": "normal/decay"})


def random_problem(rng: np.random.Generator, max_order=4, max_ext=3, min_ext=1,
                   max_p=3, dist="uniform", dtype=np.float64, permute=True,
                   allow_outer=True, label_pool=None) -> Problem:
    """A random valid binary contraction: orders, contracted count, extents and
    storage permutations drawn from `rng`."""
    while True:
        na = int(rng.integers(0, max_order + 1))
        nb = int(rng.integers(0, max_order + 1))
        pmax = min(max_p, na, nb)
        p = int(rng.integers(0 if allow_outer else min(1, pmax), pmax + 1))
        if na - p + nb - p > 8:
            continue
        break
    pool = list(label_pool) if label_pool is not None else list(range(1, 60))
    perm = rng.permutation(len(pool))
    names = [pool[k] for k in perm[: na + nb - p]]
    contracted = names[:p]
    fa = names[p:na]
    fb = names[na:na + nb - p]
    la = contracted + fa
    lb = contracted + fb
    la = [la[k] for k in rng.permutation(len(la))]
    lb = [lb[k] for k in rng.permutation(len(lb))]
    lc = fa + fb
    lc = [lc[k] for k in rng.permutation(len(lc))]
    ext = {l: int(rng.integers(min_ext, max_ext + 1)) for l in names}

    def mk(labels, out=False):
        e = [ext[l] for l in labels]
        order = list(rng.permutation(len(labels))) if permute else list(range(len(labels)))
        st = storage_strides(e, order)
        if out:
            return empty_output(labels, ext, dtype, st)
        return make_tensor(rng, labels, ext, dist=dist, dtype=dtype, strides=st)

    A, B, C = mk(la), mk(lb), mk(lc, out=True)
    return Problem("random", A, B, C)


def log_uniform_int(rng, lo, hi) -> int:
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def batching_items(n=512, seed=BASE_SEED + 3, max_elems=1 << 22, max_flops=float(1 << 34),
                   lo=8, hi=192, dtype=np.float32, with_data=True) -> List[Problem]:
    """Items of the batched workload: orders 2..5, 1..3 contracted indices,
    extents log-uniform in [lo, hi], random storage permutations of both
    operands; an item is redrawn until |A|, |B|, |C| <= max_elems and its
    flops <= max_flops."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items = []
    while len(items) < n:
        na = int(rng.integers(2, 6))
        nb = int(rng.integers(2, 6))
        p = int(rng.integers(1, min(3, na, nb) + 1))
        names = list(range(1, 1 + na + nb - p))
        contracted = names[:p]
        fa = names[p:na]
        fb = names[na:]
        ext = {l: log_uniform_int(rng, lo, hi) for l in names}
        la = contracted + fa
        lb = contracted + fb
        la = [la[k] for k in rng.permutation(len(la))]
        lb = [lb[k] for k in rng.permutation(len(lb))]
        lc = fa + fb

        def numel(ls):
            v = 1
            for l in ls:
                v *= ext[l]
            return v

        flops = 2.0 * numel(names)
        if max(numel(la), numel(lb), numel(lc)) > max_elems or flops > max_flops:
            continue
        oa = list(rng.permutation(len(la)))
        ob = list(rng.permutation(len(lb)))
        if with_data:
            A = make_tensor(rng, la, ext, order=oa, dtype=dtype)
            B = make_tensor(rng, lb, ext, order=ob, dtype=dtype)
        else:
            ea = [ext[l] for l in la]
            eb = [ext[l] for l in lb]
            A = Tensor(la, ea, storage_strides(ea, oa), np.zeros(0, dtype))
            B = Tensor(lb, eb, storage_strides(eb, ob), np.zeros(0, dtype))
        C = empty_output(lc, ext, dtype) if with_data else Tensor(
            lc, [ext[l] for l in lc], col_major([ext[l] for l in lc]), np.zeros(0, dtype))
        items.append(Problem(f"batch{len(items)}", A, B, C))
    return items


_CHUNK = 1 << 24  # elements per independent stream; fixed so results do not depend on threads


def fill_uniform_parallel(seed: int, n: int, dtype=np.float64, lo=-1.0, hi=1.0,
                          nthreads: int = 0, out: Optional[np.ndarray] = None) -> np.ndarray:
    """n uniform[lo, hi) values; chunk c (of 2^24 elements) comes from
    PCG64(seed) jumped c+1 times, so element q depends only on (seed, q): a
    shorter fill is a prefix of a longer one."""
    import concurrent.futures as cf
    import os
    if out is None:
        out = np.empty(n, dtype=dtype)
    nchunks = (n + _CHUNK - 1) // _CHUNK
    base = np.random.PCG64(seed)

    def work(c):
        g = np.random.Generator(base.jumped(c + 1))
        view = out[c * _CHUNK:min(n, (c + 1) * _CHUNK)]
        if dtype == np.float64:
            g.random(out=view)
        else:
            view[:] = g.random(view.size)
        view *= (hi - lo)
        view += lo
        return c

    nt = nthreads or min(32, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=nt) as ex:
        list(ex.map(work, range(nchunks)))
    return out


def big_problem(name, la, lb, lc, extents, seed, dtype=np.float64, alloc=None) -> Problem:
    """Like `problem` with uniform[-1, 1) entries, filled by fill_uniform_parallel
    (for operands of many gigabytes).  `alloc(n, dtype)` may supply the buffers
    (e.g. pinned host memory)."""
    ext = {lab(k)[0]: int(v) for k, v in extents.items()}
    tens = []
    for t, ls in enumerate((la, lb)):
        ls = lab(ls)
        e = [ext[l] for l in ls]
        st = col_major(e)
        n = span(e, st)
        buf = alloc(n, dtype) if alloc is not None else None
        tens.append(Tensor(ls, e, st, fill_uniform_parallel(seed * 16 + t, n, dtype, out=buf)))
    C = empty_output(lc, ext, dtype)
    return Problem(name, tens[0], tens[1], C, meta={"seed": seed, "dist": "uniform"})


def gemv_1024_full(seed=BASE_SEED + 1, b=1024, alloc=None) -> Problem:
    """The Class 2 workload at full size: A is 2^31 FP64 values (17.2 GB).
    A smaller b gives the leading slab of the same tensor."""
    return big_problem("gemv_1024", "aib", "i", "ab", dict(a=1024, b=b, i=2048), seed + 200,
                       alloc=alloc)


def ccd_skewed(free: int, occ: int, beta: int = 8, seed: int = BASE_SEED + 5,
               dtype=np.float64, alloc=None) -> Problem:
    """R[a,b,c,d] = sum_{i,j} X[i,a,j,b] Y[i,c,j,d], the CCD contraction of
    Sec. 4.2 (X^{i alpha j beta} Y_{i gamma j delta}) with a = c = d = free,
    b = beta fixed and i = j = occ; column-major, uniform[-1, 1) entries.
    occ = 4 is the GR case of the same section."""
    return big_problem(f"ccd_f{free}_o{occ}", "iajb", "icjd", "abcd",
                       dict(i=occ, j=occ, a=free, b=beta, c=free, d=free), seed + free * 7 + occ,
                       dtype, alloc)


def selector_descriptors(n: int, seed: int = BASE_SEED + 4, lo: int = 4, hi: int = 256,
                         max_elems: int = 1 << 24, max_out: int = 1 << 24,
                         max_flops: float = float(1 << 35)):
    """Random contraction descriptors of the selector workload: orders 2-6,
    1-3 contracted labels, extents log-uniform in [lo, hi], random storage
    orders of A, B and C.  A draw is repeated until every tensor has at most
    max_elems elements, C at most max_out, and 2 * prod(extents) <= max_flops.
    Returns (A, B, C) descriptor triples of Tensor objects without data."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n:
        na = int(rng.integers(2, 7))
        nb = int(rng.integers(2, 7))
        p = int(rng.integers(1, min(3, na, nb) + 1))
        names = list(range(1, 1 + na + nb - p))
        con, fa, fb = names[:p], names[p:na], names[na:]
        ext = {l: log_uniform_int(rng, lo, hi) for l in names}

        def numel(ls):
            v = 1
            for l in ls:
                v *= ext[l]
            return v

        if (max(numel(con + fa), numel(con + fb)) > max_elems or numel(fa + fb) > max_out
                or 2.0 * numel(names) > max_flops):
            continue
        tens = []
        for ls in (con + fa, con + fb, fa + fb):
            ls = [ls[k] for k in rng.permutation(len(ls))]
            e = [ext[l] for l in ls]
            order = list(rng.permutation(len(ls)))
            tens.append(Tensor(ls, e, storage_strides(e, order), np.zeros(0, np.float32)))
        out.append(tuple(tens))
    return out
