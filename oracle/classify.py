"""The paper's contraction classification and slicing recipes, in plain Python.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Parity: pinned by the
paper's worked examples (tests/golden/classification_cases.json).

Definitions followed:
  * slicing vector s(T) in {0,1}^N(T), 1 = the index is looped over
    (Sec. 2.4; the printed equation is blank, the meaning is taken from the
    three examples (a) s=(0,1,0), (b) s=(1,0,0), (c) s=(1,1,0) that follow it);
  * requirements R1-R3 and failure modes F1-F3 (Sec. 3.1);
  * Delta(t) = N(t) - p, the number of free indices (Sec. 3.2);
  * Class 1: Delta(t1) = Delta(t2) = 0; Class 2: exactly one Delta is 0;
    Class 3: both >= 1, split into 3.1 (stride-1 indices of t1 and t2 distinct
    and both contracted) and 3.2 (otherwise) (Sec. 3.2.3 and the general rule
    stated after Table 1);
  * the recipes of Classes 1, 2, 3.1 and 3.2 (Sec. 3.2).

Readings where the paper is silent:
  * indices of extent 1 are ignored by the classification (slicing them is
    free) and are reported as sliced;
  * the stride-1 index of a tensor is its index with stride 1 and extent > 1;
    a tensor with no such index cannot satisfy R1 for any slicing, so a Class 3
    contraction involving it is put in Class 3.1 (it needs a copy);
  * "keep the index with the largest size unsliced": ties go to the index with
    the smaller stride in C (free indices) or in the tensor itself (contracted
    indices), then to the earlier position in the tensor;
  * Class 3.1: the operand whose stride-1 index has the larger extent keeps it
    (ties: A), so the other operand's stride-1 index is sliced and that operand
    is the one copied.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple


@dataclass
class Desc:
    labels: List[int]
    extents: List[int]
    strides: List[int]


def _mk(t) -> Desc:
    labels = list(t.labels)
    extents = [int(e) for e in t.extents]
    strides = getattr(t, "strides", None)
    if strides is None:
        strides, acc = [], 1
        for e in extents:
            strides.append(acc)
            acc *= max(e, 1)
    return Desc(labels, extents, [int(s) for s in strides])


@dataclass
class Classification:
    contracted: List[int]
    free_a: List[int]
    free_b: List[int]
    p: int
    delta_a: int
    delta_b: int
    cls: int                       # 1, 2, 31 or 32
    stride1_a: Optional[int]
    stride1_b: Optional[int]
    slice_a: Tuple[int, ...]       # s(A), one entry per index of A
    slice_b: Tuple[int, ...]       # s(B)
    family: str                    # DOT, GEMV, GEMM, COPY+GEMM
    copied: Optional[str] = None   # 'A' or 'B' for Class 3.1


def stride1(t: Desc) -> Optional[int]:
    for l, e, s in zip(t.labels, t.extents, t.strides):
        if e > 1 and s == 1:
            return l
    return None


def _pick_largest(cands: Sequence[int], ext: Dict[int, int], key2) -> int:
    """Largest extent; ties by key2 (ascending)."""
    return sorted(cands, key=lambda l: (-ext[l], key2(l)))[0]


def classify(A, B, C) -> Classification:
    A, B, C = _mk(A), _mk(B), _mk(C)
    ext: Dict[int, int] = {}
    for t in (A, B, C):
        for l, e in zip(t.labels, t.extents):
            ext[l] = e
    big = lambda ls: [l for l in ls if ext[l] > 1]
    contracted = [l for l in A.labels if l in B.labels]
    free_a = [l for l in A.labels if l not in B.labels]
    free_b = [l for l in B.labels if l not in A.labels]
    K = big(contracted)
    FA = big(free_a)
    FB = big(free_b)
    p = len(K)
    da, db = len(FA), len(FB)
    s1a, s1b = stride1(A), stride1(B)

    sa_of = dict(zip(A.labels, A.strides))
    sb_of = dict(zip(B.labels, B.strides))
    sc_of = dict(zip(C.labels, C.strides))
    pos_a = {l: k for k, l in enumerate(A.labels)}
    pos_b = {l: k for k, l in enumerate(B.labels)}

    def pick_free(cands, pos):
        return _pick_largest(cands, ext, lambda l: (sc_of.get(l, 0), pos.get(l, 0)))

    def pick_con(cands, strides, pos):
        return _pick_largest(cands, ext, lambda l: (strides[l], pos[l]))

    keep_a: List[int] = []
    keep_b: List[int] = []
    copied = None
    if da == 0 and db == 0:
        cls, family = 1, "DOT"
        if K:
            if s1a in K:
                k = s1a
            else:
                k = pick_con(K, sa_of, pos_a)
            keep_a, keep_b = [k], [k]
    elif da == 0 or db == 0:
        cls, family = 2, "GEMV"
        # t1 = the tensor with free indices
        if da >= 1:
            t1_free, s1, st1, pos1 = FA, s1a, sa_of, pos_a
        else:
            t1_free, s1, st1, pos1 = FB, s1b, sb_of, pos_b
        if s1 is not None and s1 in K:
            kc = s1
            kf = pick_free(t1_free, pos1)
        elif s1 is not None and s1 in t1_free:
            kf = s1
            kc = pick_con(K, st1, pos1) if K else None
        else:  # no stride-1 index: keep the largest of each kind
            kf = pick_free(t1_free, pos1)
            kc = pick_con(K, st1, pos1) if K else None
        t1_keep = [kf] + ([kc] if kc is not None else [])
        t2_keep = [kc] if kc is not None else []
        if da >= 1:
            keep_a, keep_b = t1_keep, t2_keep
        else:
            keep_a, keep_b = t2_keep, t1_keep
    else:
        both_con = (s1a in K) and (s1b in K)
        if s1a is None or s1b is None or (s1a != s1b and both_con):
            cls, family = 31, "COPY+GEMM"
            # keep the first (stride-1) index of one operand
            if s1a is not None and s1b is not None:
                keep_first_a = ext[s1a] >= ext[s1b]
            else:
                keep_first_a = s1a is not None
            if keep_first_a and s1a in K:
                k = s1a
                copied = "B"
            elif (not keep_first_a) and s1b in K:
                k = s1b
                copied = "A"
            else:
                k = pick_con(K, sa_of, pos_a) if K else None
                copied = "B" if keep_first_a else "A"
            fa = s1a if s1a in FA else pick_free(FA, pos_a)
            fb = s1b if s1b in FB else pick_free(FB, pos_b)
            keep_a = [fa] + ([k] if k is not None else [])
            keep_b = [fb] + ([k] if k is not None else [])
        else:
            cls, family = 32, "GEMM"
            # leave both stride-1 indices untouched
            if s1a in K and s1b in K:          # same contracted index
                k = s1a
                fa, fb = pick_free(FA, pos_a), pick_free(FB, pos_b)
            elif s1a in K:                     # s1b is free
                k, fb = s1a, s1b
                fa = pick_free(FA, pos_a)
            elif s1b in K:                     # s1a is free
                k, fa = s1b, s1a
                fb = pick_free(FB, pos_b)
            else:                              # both stride-1 indices free
                fa, fb = s1a, s1b
                k = pick_con(K, sa_of, pos_a) if K else None
            keep_a = [fa] + ([k] if k is not None else [])
            keep_b = [fb] + ([k] if k is not None else [])

    slice_a = tuple(0 if l in keep_a else 1 for l in A.labels)
    slice_b = tuple(0 if l in keep_b else 1 for l in B.labels)
    return Classification(K, FA, FB, p, da, db, cls, s1a, s1b, slice_a, slice_b, family, copied)


def requirements(A, B, sa: Sequence[int], sb: Sequence[int]) -> Dict[str, bool]:
    """Check R1-R3 (Sec. 3.1) for slicing vectors sa, sb over the indices of A, B
    (indices of extent 1 are ignored)."""
    A, B = _mk(A), _mk(B)
    ext = dict(zip(A.labels, A.extents))
    ext.update(zip(B.labels, B.extents))
    con = set(A.labels) & set(B.labels)
    # a contracted index is sliced in both tensors or in neither
    consistent = all(sa[A.labels.index(l)] == sb[B.labels.index(l)] for l in con)
    def unsliced(t, s):
        return [l for l, v in zip(t.labels, s) if v == 0 and ext[l] > 1]
    ua, ub = unsliced(A, sa), unsliced(B, sb)
    s1a, s1b = stride1(A), stride1(B)
    r1 = (s1a is None or s1a in ua) and (s1b is None or s1b in ub) and s1a is not None \
        and s1b is not None
    r2 = len(ua) == 2 and len(ub) == 2
    r3 = (len([l for l in ua if l in con]) == 1 and len([l for l in ua if l not in con]) == 1
          and len([l for l in ub if l in con]) == 1 and len([l for l in ub if l not in con]) == 1
          and set(l for l in ua if l in con) == set(l for l in ub if l in con))
    return {"consistent": consistent, "R1": bool(r1), "R2": r2, "R3": bool(r3)}


def slicing_kernel(A, B, sa: Sequence[int], sb: Sequence[int]) -> str:
    """The BLAS kernel a slicing leads to (Sec. 2.2, Sec. 2.4, Sec. 3.1 F1-F3):
    count the unsliced free (f) and contracted (k) indices of each slice.

      f=1,k=1 in both, sharing k   -> GEMM (COPY+GEMM if R1 fails, F1)
      one slice a matrix (f=1,k>=1), the other a vector of contracted (f=0) -> GEMV
      f=1,k=0 in both              -> GER (outer product)
      f=0 in both, k>=1            -> DOT (inner products summed, F3)
      anything else                -> NONE (element-wise, no BLAS)
    """
    A, B = _mk(A), _mk(B)
    ext = dict(zip(A.labels, A.extents))
    ext.update(zip(B.labels, B.extents))
    con = set(A.labels) & set(B.labels)

    def counts(t, s):
        u = [l for l, v in zip(t.labels, s) if v == 0 and ext[l] > 1]
        return len([l for l in u if l not in con]), len([l for l in u if l in con])

    fa, ka = counts(A, sa)
    fb, kb = counts(B, sb)
    if fa == 1 and ka == 1 and fb == 1 and kb == 1:
        return "GEMM" if requirements(A, B, sa, sb)["R1"] else "COPY+GEMM"
    if (fa == 1 and ka >= 1 and fb == 0 and kb >= 1) or (fb == 1 and kb >= 1 and fa == 0 and ka >= 1):
        return "GEMV"
    if fa == 1 and ka == 0 and fb == 1 and kb == 0:
        return "GER"
    if fa == 0 and fb == 0 and ka >= 1 and kb >= 1:
        return "DOT"
    return "NONE"
