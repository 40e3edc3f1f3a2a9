"""Free-index sharding of one contraction over ranks (one device each).

Slicing a free index of C gives independent contractions (Sec. 2.4).  Rank r
of n takes the slab that tc_shard_free_index assigns it (a balanced range of
C's largest free index), plans it with tc_plan and runs it on its own device
with tc_contract on its own buffers, offset to the slab.  No data crosses
ranks: each rank writes a disjoint part of C.  Marshalling only; the choice
of label and range is the library's.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

from . import tc
from .api import Contraction

Desc = Tuple[Sequence[int], Sequence[int], Optional[Sequence[int]]]


def col_major(extents: Sequence[int]):
    st, acc = [], 1
    for e in extents:
        st.append(acc)
        acc *= max(int(e), 1)
    return st


def _explicit(d: Desc) -> Desc:
    labels, extents, strides = d
    return (list(labels), list(extents), list(strides) if strides is not None
            else col_major(extents))


def slab(A: Desc, B: Desc, C: Desc, n: int, r: int):
    """(shard, (A', B', C')): the shard of rank r of n and its slab
    descriptors (the split label's extent replaced, strides explicit)."""
    A, B, C = _explicit(A), _explicit(B), _explicit(C)
    sh = tc.tc_shard_free_index(A, B, C, n, r)
    out = []
    for d, pos in ((A, sh.pos_a), (B, sh.pos_b), (C, sh.pos_c)):
        ext = list(d[1])
        if pos >= 0:
            ext[pos] = sh.end - sh.begin
        out.append((d[0], ext, d[2]))
    return sh, tuple(out)


def rank_and_world():
    """(rank, world size) of torch.distributed if initialised, else (0, 1)."""
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist.get_rank(), dist.get_world_size()
    except Exception:
        pass
    return 0, 1


class ShardedContraction:
    """This rank's part of C = alpha A.B + beta C, sharded over a free index.

    A, B, C: (labels, extents, strides-or-None) of the whole tensors; rank and
    world default to torch.distributed's.  Calling it with the whole tensors'
    device buffers (every rank holds them, or at least its slab of them at the
    same offsets) computes this rank's slab of C."""

    def __init__(self, A: Desc, B: Desc, C: Desc, dtype: str = "f64", math: str = "fp64",
                 mapping: str = "auto", rank: Optional[int] = None,
                 world: Optional[int] = None):
        r, w = rank_and_world()
        self.rank = r if rank is None else int(rank)
        self.world = w if world is None else int(world)
        self.shard, (sa, sb, sc) = slab(A, B, C, self.world, self.rank)
        self.empty = self.shard.end <= self.shard.begin
        self.plan = None if self.empty else Contraction(sa, sb, sc, dtype, math, mapping)
        self.esz = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[dtype]

    def __call__(self, A, B, C, alpha: float = 1.0, beta: float = 0.0, stream=None):
        if self.empty:
            return C
        import torch
        pl = self.plan
        ws = pl.workspace(C.device)
        s = stream if stream is not None else torch.cuda.current_stream(C.device)
        sh, e = self.shard, self.esz
        tc.tc_contract(pl.handle, alpha, A.data_ptr() + sh.offset_a * e,
                       B.data_ptr() + sh.offset_b * e, beta, C.data_ptr() + sh.offset_c * e,
                       ws.data_ptr() if ws is not None else 0,
                       ws.numel() if ws is not None else 0, s.cuda_stream)
        return C
