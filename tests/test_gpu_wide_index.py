"""Tensors of 2^32 or more elements through the kernels that walk a whole
tensor by one flat index: the COPY baseline's permute (Sec. 3.1 F1) and the
beta-only scaling of an empty contracted range (C = beta C).  A 32-bit split
of that index would wrap, write some elements twice and never reach the
tail; these tests check the tail and the whole tensor.

The inputs are small integers, so every output is exact in any summation
order and must equal the oracle's bit for bit."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

WIDE = (1 << 32) + 8


def _fill_int_pattern(buf, I):
    """buf[i + I*b] = ((7 i + b) mod 9) - 4, written in chunks on the device."""
    import torch
    n = buf.numel()
    step = 1 << 27
    for lo in range(0, n, step):
        hi = min(n, lo + step)
        q = torch.arange(lo, hi, dtype=torch.int64, device=buf.device)
        buf[lo:hi] = ((7 * (q % I) + q // I) % 9 - 4).to(buf.dtype)
        del q


def test_copy_gemm_operand_beyond_2_pow_32():
    """C[a,b] = sum_i A[a,i] B[i,b] with B of 8 x (2^29 + 1) = 2^32 + 8 FP32
    elements, mapping COPY_GEMM: B is permuted into the workspace by the flat
    permute kernel, then multiplied.  Sampled columns, the last ones included,
    against the oracle."""
    import torch
    from paper_1307_2100_gb300 import Contraction
    I, a_ext = 8, 2
    b_ext = WIDE // I
    assert I * b_ext == WIDE
    dev = torch.device("cuda:0")
    a, i, b = 0, 1, 2                                   # labels
    plan = Contraction(([a, i], [a_ext, I], None), ([i, b], [I, b_ext], None),
                       ([a, b], [a_ext, b_ext], None), "f32", "fp32", "copy_gemm")
    assert plan.info.workspace >= WIDE * 4          # B is the copied operand
    A_h = np.array([1, -4, -2, 1, 3, 0, 0, 2, 4, -2, -1, 3, 2, 1, -3, 1], np.float32)  # [a, i]
    A = torch.from_numpy(A_h).to(dev)
    B = torch.empty(WIDE, dtype=torch.float32, device=dev)
    _fill_int_pattern(B, I)
    C = torch.full((a_ext * b_ext,), float("nan"), dtype=torch.float32, device=dev)
    plan(A, B, C)
    torch.cuda.synchronize()
    cols = np.r_[0, 1, 12345, (1 << 28) + 3, b_ext - 8 + np.arange(8)]
    got = C.view(b_ext, a_ext)[torch.from_numpy(cols).to(dev)].cpu().numpy().T
    ii = np.arange(I)
    Bcols = np.stack([((7 * ii + c) % 9 - 4).astype(np.float64) for c in cols], axis=1)
    ref = np.zeros(a_ext * len(cols))
    oracle.contract_raw([a, i], [a_ext, I], [1, a_ext], A_h.astype(np.float64),
                        [i, b], [I, len(cols)], [1, I], Bcols.reshape(-1, order="F"),
                        [a, b], [a_ext, len(cols)], [1, a_ext], ref, 1.0, 0.0)
    ref = ref.reshape(a_ext, len(cols), order="F")
    np.testing.assert_array_equal(got.astype(np.float64), ref)
    assert not torch.isnan(C).any().item()
    del B, C, plan
    torch.cuda.empty_cache()


def test_beta_scaling_of_output_beyond_2_pow_32():
    """An empty contracted range gives C = beta C over C's own (row-major)
    layout: C[a,b] with a = 2^16 + 1, b = 2^16, strides (2^16, 1), FP32,
    2^32 + 2^16 elements.  Every element must be scaled exactly once."""
    import torch
    from paper_1307_2100_gb300 import Contraction
    a_ext, b_ext = (1 << 16) + 1, 1 << 16
    n = a_ext * b_ext
    dev = torch.device("cuda:0")
    a, k, b = 0, 1, 2                                   # labels
    plan = Contraction(([a, k], [a_ext, 0], None), ([k, b], [0, b_ext], None),
                       ([a, b], [a_ext, b_ext], [b_ext, 1]), "f32", "fp32", "auto")
    A = torch.zeros(1, dtype=torch.float32, device=dev)
    B = torch.zeros(1, dtype=torch.float32, device=dev)
    C = torch.full((n,), 1.5, dtype=torch.float32, device=dev)
    plan(A, B, C, 1.0, -2.0)
    torch.cuda.synchronize()
    assert bool((C == -3.0).all().item())
    del C
    torch.cuda.empty_cache()
