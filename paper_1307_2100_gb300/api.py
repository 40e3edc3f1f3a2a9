"""Convenience layer over the C ABI taking PyTorch tensors (memory and streams only)."""
from __future__ import annotations

from . import tc

class Contraction:
    """A planned contraction C = alpha * A.B + beta * C over labelled indices.

    Each operand is (labels, extents, strides-or-None); strides count
    elements.  `dtype` is one of tc.DTYPE ("f64", "f32", "bf16", "f16"),
    `math` one of tc.MATH, `mapping` one of tc.MAPPING.
    """

    def __init__(self, A, B, C, dtype: str = "f64", math: str = "fp64",
                 mapping: str = "auto", tile: int = -1):
        self.dtype = tc.DTYPE[dtype]
        self.handle = tc.tc_plan(A, B, C, self.dtype, tc.MATH[math], tc.MAPPING[mapping], tile)
        self.info = tc.tc_plan_get_info(self.handle)
        self._ws = None

    def workspace(self, device):
        import torch
        n = int(self.info.workspace)
        if n and (self._ws is None or self._ws.numel() < n or self._ws.device != device):
            self._ws = torch.empty(n, dtype=torch.uint8, device=device)
        return self._ws

    def __call__(self, A, B, C, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """A, B, C: CUDA tensors whose storage holds the described layouts."""
        import torch
        ws = self.workspace(C.device)
        s = stream if stream is not None else torch.cuda.current_stream(C.device)
        tc.tc_contract(self.handle, alpha, A.data_ptr(), B.data_ptr(), beta, C.data_ptr(),
                       ws.data_ptr() if ws is not None else 0,
                       ws.numel() if ws is not None else 0, s.cuda_stream)
        return C

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            tc.tc_plan_destroy(h)
            self.handle = None
