"""ctypes binding of libtc.so -- argument marshalling only.

Functions carry the C names (tc_plan, tc_contract, ...).  Device memory and
streams come from PyTorch; every computation runs in the library's kernels.
If the shared library is missing this module raises at import: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtc.so")

TC_OK = 0
TC_ERR_TIMEOUT = 8
STATUS = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_LABEL", 3: "TC_ERR_EXTENT_MISMATCH",
          4: "TC_ERR_STRIDE", 5: "TC_ERR_UNSUPPORTED", 6: "TC_ERR_WORKSPACE", 7: "TC_ERR_CUDA",
          8: "TC_ERR_TIMEOUT", 9: "TC_ERR_NO_SELECTOR"}
TC_F64, TC_F32, TC_BF16, TC_F16 = 0, 1, 2, 3
DTYPE = {"f64": TC_F64, "f32": TC_F32, "bf16": TC_BF16, "f16": TC_F16}
MATH = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16x3": 3, "bf16x6": 4, "fp8": 5, "fp16": 6}
MAPPING = {"auto": 0, "recipe": 1, "slice_gemm": 2, "fused_gemm": 3, "copy_gemm": 4, "gemv": 5,
           "dot": 6, "ger": 7}
MAPPING_NAME = {v: k for k, v in MAPPING.items()}
KERNEL_NAME = {0: "none", 1: "gemm_simt", 2: "gemm_tc", 3: "gemv", 4: "dot", 5: "gemm_fp8",
               6: "ger"}
MAX_ORDER = 12
N_FEATURES = 23


class TcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


class TensorDesc(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32),
                ("labels", ctypes.POINTER(ctypes.c_int32)),
                ("extents", ctypes.POINTER(ctypes.c_int64)),
                ("strides", ctypes.POINTER(ctypes.c_int64))]


class PlanInfo(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_int32), ("p", ctypes.c_int32), ("delta_a", ctypes.c_int32),
                ("delta_b", ctypes.c_int32), ("stride1_a", ctypes.c_int32),
                ("stride1_b", ctypes.c_int32), ("slice_a", ctypes.c_uint32),
                ("slice_b", ctypes.c_uint32), ("mapping", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("tile", ctypes.c_int32), ("swapped", ctypes.c_int32),
                ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("batch", ctypes.c_int64), ("flops", ctypes.c_double),
                ("min_bytes", ctypes.c_double), ("workspace", ctypes.c_size_t)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["mapping_name"] = MAPPING_NAME.get(self.mapping, "?")
        d["kernel_name"] = KERNEL_NAME.get(self.kernel, "?")
        return d


class LayoutAdvice(ctypes.Structure):
    _fields_ = [("operand", ctypes.c_int32), ("order", ctypes.c_int32),
                ("storage_order", ctypes.c_int32 * MAX_ORDER), ("cls_after", ctypes.c_int32),
                ("copy_bytes", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("math", ctypes.c_int32),
                ("n_tiles", ctypes.c_int64), ("flops", ctypes.c_double),
                ("min_bytes", ctypes.c_double), ("n_tc_items", ctypes.c_int32),
                ("n_simt_items", ctypes.c_int32), ("n_simt_work", ctypes.c_int64),
                ("n_simt_tiles", ctypes.c_int64), ("n_tc_split", ctypes.c_int64)]


class Shard(ctypes.Structure):
    _fields_ = [("label", ctypes.c_int32), ("pos_a", ctypes.c_int32), ("pos_b", ctypes.c_int32),
                ("pos_c", ctypes.c_int32), ("begin", ctypes.c_int64), ("end", ctypes.c_int64),
                ("offset_a", ctypes.c_int64), ("offset_b", ctypes.c_int64),
                ("offset_c", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1307_2100_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.tc_plan.restype = ctypes.c_int
    lib.tc_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(TensorDesc),
                            ctypes.POINTER(TensorDesc), ctypes.POINTER(TensorDesc), ctypes.c_int,
                            ctypes.c_int, ctypes.c_int, ctypes.c_int32]
    lib.tc_plan_get_info.restype = ctypes.c_int
    lib.tc_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.tc_plan_layout_advice.restype = ctypes.c_int
    lib.tc_plan_layout_advice.argtypes = [P, ctypes.POINTER(LayoutAdvice)]
    lib.tc_plan_destroy.restype = ctypes.c_int
    lib.tc_plan_destroy.argtypes = [P]
    lib.tc_contract.restype = ctypes.c_int
    lib.tc_contract.argtypes = [P, ctypes.c_double, P, P, ctypes.c_double, P, P, ctypes.c_size_t,
                                P]
    lib.tc_batch_set_route.restype = ctypes.c_int
    lib.tc_batch_set_route.argtypes = [ctypes.c_int32]
    lib.tc_batch_plan.restype = ctypes.c_int
    lib.tc_batch_plan.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int32]
    lib.tc_batch_plan_routes.restype = ctypes.c_int
    lib.tc_batch_plan_routes.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), P, ctypes.c_int32]
    lib.tc_batch_get_info.restype = ctypes.c_int
    lib.tc_batch_get_info.argtypes = [P, ctypes.POINTER(BatchInfo)]
    lib.tc_contract_batched.restype = ctypes.c_int
    lib.tc_contract_batched.argtypes = [P, P, P, P, P, P, P]
    lib.tc_batch_destroy.restype = ctypes.c_int
    lib.tc_batch_destroy.argtypes = [P]
    lib.tc_contract_dot_noalloc.restype = ctypes.c_int
    lib.tc_contract_dot_noalloc.argtypes = [P, ctypes.c_double, P, P, ctypes.c_double, P, P]
    lib.tc_mlp_create.restype = ctypes.c_int
    lib.tc_mlp_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_int32]
    lib.tc_mlp_destroy.restype = ctypes.c_int
    lib.tc_mlp_destroy.argtypes = [P]
    lib.tc_mlp_num_params.restype = ctypes.c_int
    lib.tc_mlp_num_params.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
    lib.tc_mlp_set_params.restype = ctypes.c_int
    lib.tc_mlp_set_params.argtypes = [P, P, ctypes.c_int64]
    lib.tc_mlp_get_params.restype = ctypes.c_int
    lib.tc_mlp_get_params.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32]
    lib.tc_mlp_forward.restype = ctypes.c_int
    lib.tc_mlp_forward.argtypes = [P, P, P, ctypes.c_int32, P]
    lib.tc_mlp_loss_grad.restype = ctypes.c_int
    lib.tc_mlp_loss_grad.argtypes = [P, P, P, P, ctypes.c_int32, P, P, P]
    lib.tc_mlp_adam_step.restype = ctypes.c_int
    lib.tc_mlp_adam_step.argtypes = [P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_int32, P]
    lib.tc_plan_features.restype = ctypes.c_int
    lib.tc_plan_features.argtypes = [P, P, ctypes.c_int32]
    lib.tc_selector_load.restype = ctypes.c_int
    lib.tc_selector_load.argtypes = [ctypes.c_char_p]
    lib.tc_selector_unload.restype = ctypes.c_int
    lib.tc_selector_unload.argtypes = []
    lib.tc_selector_predict.restype = ctypes.c_int
    lib.tc_selector_predict.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.tc_selftest_wait_timeout.restype = ctypes.c_int
    lib.tc_selftest_wait_timeout.argtypes = [ctypes.c_int64, P]
    lib.tc_device_status.restype = ctypes.c_int
    lib.tc_device_status.argtypes = [P]
    lib.tc_status_string.restype = ctypes.c_char_p
    lib.tc_status_string.argtypes = [ctypes.c_int]
    lib.tc_shard_free_index.restype = ctypes.c_int
    lib.tc_shard_free_index.argtypes = [ctypes.POINTER(TensorDesc), ctypes.POINTER(TensorDesc),
                                        ctypes.POINTER(TensorDesc), ctypes.c_int32,
                                        ctypes.c_int32, ctypes.POINTER(Shard)]
    lib.tc_peak_probe.restype = ctypes.c_int
    lib.tc_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                  P]
    return lib


lib = _load()


def make_desc(labels: Sequence[int], extents: Sequence[int],
              strides: Optional[Sequence[int]] = None):
    """A TensorDesc plus the ctypes arrays that keep its pointers alive."""
    n = len(labels)
    la = (ctypes.c_int32 * max(n, 1))(*[int(x) for x in labels])
    ex = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in extents])
    st = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in strides]) if strides is not None else None
    d = TensorDesc(n, la, ex, st if st is not None else ctypes.POINTER(ctypes.c_int64)())
    return d, (la, ex, st)


def tc_status_string(status: int) -> str:
    return lib.tc_status_string(int(status)).decode()


def tc_plan(A, B, C, dtype: int, math: int, mapping: int = 0, tile: int = -1) -> int:
    """A, B, C: (labels, extents, strides-or-None).  Returns the plan handle."""
    dA, kA = make_desc(*A)
    dB, kB = make_desc(*B)
    dC, kC = make_desc(*C)
    out = ctypes.c_void_p()
    st = lib.tc_plan(ctypes.byref(out), ctypes.byref(dA), ctypes.byref(dB), ctypes.byref(dC),
                     int(dtype), int(math), int(mapping), int(tile))
    if st != TC_OK:
        raise TcError(st, "tc_plan")
    return out.value


def tc_plan_status(A, B, C, dtype: int, math: int, mapping: int = 0, tile: int = -1) -> int:
    """tc_plan's status code only (the plan, if any, is destroyed)."""
    try:
        h = tc_plan(A, B, C, dtype, math, mapping, tile)
    except TcError as e:
        return e.status
    tc_plan_destroy(h)
    return TC_OK


def tc_shard_free_index(A, B, C, n_shards: int, shard: int) -> Shard:
    """A, B, C: (labels, extents, strides-or-None).  Shard `shard` of n."""
    dA, kA = make_desc(*A)
    dB, kB = make_desc(*B)
    dC, kC = make_desc(*C)
    out = Shard()
    _check(lib.tc_shard_free_index(ctypes.byref(dA), ctypes.byref(dB), ctypes.byref(dC),
                                   int(n_shards), int(shard), ctypes.byref(out)),
           "tc_shard_free_index")
    return out


def tc_plan_layout_advice(plan: int) -> LayoutAdvice:
    adv = LayoutAdvice()
    _check(lib.tc_plan_layout_advice(ctypes.c_void_p(plan), ctypes.byref(adv)),
           "tc_plan_layout_advice")
    return adv


def tc_plan_get_info(plan: int) -> PlanInfo:
    info = PlanInfo()
    st = lib.tc_plan_get_info(ctypes.c_void_p(plan), ctypes.byref(info))
    if st != TC_OK:
        raise TcError(st, "tc_plan_get_info")
    return info


def tc_plan_destroy(plan: int) -> None:
    lib.tc_plan_destroy(ctypes.c_void_p(plan))


def tc_contract(plan: int, alpha: float, A: int, B: int, beta: float, C: int, workspace: int = 0,
                workspace_bytes: int = 0, stream: int = 0) -> None:
    """Pointers are integer device addresses; stream is a cudaStream_t as int."""
    st = lib.tc_contract(ctypes.c_void_p(plan), float(alpha), ctypes.c_void_p(A),
                         ctypes.c_void_p(B), float(beta), ctypes.c_void_p(C),
                         ctypes.c_void_p(workspace), int(workspace_bytes),
                         ctypes.c_void_p(stream))
    if st != TC_OK:
        raise TcError(st, "tc_contract")


def tc_device_status(stream: int = 0) -> int:
    return lib.tc_device_status(ctypes.c_void_p(stream))


def tc_batch_plan(plans) -> int:
    arr = (ctypes.c_void_p * max(len(plans), 1))(*plans)
    out = ctypes.c_void_p()
    st = lib.tc_batch_plan(ctypes.byref(out), arr, len(plans))
    if st != TC_OK:
        raise TcError(st, "tc_batch_plan")
    return out.value


def tc_batch_plan_routes(plans, routes) -> int:
    """routes: one of -1 (threshold rule), 0 (CUDA cores), 1 (tensor cores) per plan."""
    import numpy as np
    arr = (ctypes.c_void_p * max(len(plans), 1))(*plans)
    r = np.ascontiguousarray(routes, np.int32)
    if len(r) != len(plans):
        raise ValueError("one route per plan")
    out = ctypes.c_void_p()
    st = lib.tc_batch_plan_routes(ctypes.byref(out), arr, ctypes.c_void_p(r.ctypes.data),
                                  len(plans))
    if st != TC_OK:
        raise TcError(st, "tc_batch_plan_routes")
    return out.value


def tc_batch_get_info(batch: int) -> BatchInfo:
    info = BatchInfo()
    st = lib.tc_batch_get_info(ctypes.c_void_p(batch), ctypes.byref(info))
    if st != TC_OK:
        raise TcError(st, "tc_batch_get_info")
    return info


def tc_contract_batched(batch: int, A: int, B: int, C: int, alpha: int, beta: int,
                        stream: int = 0) -> None:
    """A, B, C, alpha, beta: device addresses of arrays of n pointers / doubles."""
    st = lib.tc_contract_batched(ctypes.c_void_p(batch), ctypes.c_void_p(A), ctypes.c_void_p(B),
                                 ctypes.c_void_p(C), ctypes.c_void_p(alpha),
                                 ctypes.c_void_p(beta), ctypes.c_void_p(stream))
    if st != TC_OK:
        raise TcError(st, "tc_contract_batched")


def tc_batch_destroy(batch: int) -> None:
    lib.tc_batch_destroy(ctypes.c_void_p(batch))


def tc_selftest_wait_timeout(timeout_ns: int, stream: int = 0) -> None:
    st = lib.tc_selftest_wait_timeout(int(timeout_ns), ctypes.c_void_p(stream))
    if st != TC_OK:
        raise TcError(st, "tc_selftest_wait_timeout")


def tc_contract_dot_noalloc(plan: int, alpha: float, A: int, B: int, beta: float, C: int,
                            stream: int = 0) -> None:
    """Scalar (single-output) contraction using the library's built-in scratch
    array instead of a workspace; see include/tc.h."""
    st = lib.tc_contract_dot_noalloc(ctypes.c_void_p(plan), float(alpha), ctypes.c_void_p(A),
                                     ctypes.c_void_p(B), float(beta), ctypes.c_void_p(C),
                                     ctypes.c_void_p(stream))
    if st != TC_OK:
        raise TcError(st, "tc_contract_dot_noalloc")


PEAK = {"dfma": 0, "dmma": 1, "ffma": 2, "bf16": 3, "bf16_n256": 4, "fp8": 5}


def tc_peak_probe(kind: int, iters: int, stream: int = 0) -> float:
    """Enqueue one peak-rate probe launch; returns the FLOPs it performs."""
    f = ctypes.c_double(0.0)
    st = lib.tc_peak_probe(int(kind), int(iters), ctypes.byref(f), ctypes.c_void_p(stream))
    if st != TC_OK:
        raise TcError(st, "tc_peak_probe")
    return f.value


def tc_batch_set_route(tc_min_mn: int) -> None:
    st = lib.tc_batch_set_route(int(tc_min_mn))
    if st != TC_OK:
        raise TcError(st, "tc_batch_set_route")


def _check(st, where):
    if st != TC_OK:
        raise TcError(st, where)


def tc_mlp_create(n_in: int, n_hidden: int, n_out: int, max_batch: int) -> int:
    out = ctypes.c_void_p()
    _check(lib.tc_mlp_create(ctypes.byref(out), n_in, n_hidden, n_out, max_batch), "tc_mlp_create")
    return out.value


def tc_mlp_destroy(net: int) -> None:
    lib.tc_mlp_destroy(ctypes.c_void_p(net))


def tc_mlp_num_params(net: int) -> int:
    n = ctypes.c_int64()
    _check(lib.tc_mlp_num_params(ctypes.c_void_p(net), ctypes.byref(n)), "tc_mlp_num_params")
    return n.value


def tc_mlp_set_params(net: int, host_ptr: int, n: int) -> None:
    _check(lib.tc_mlp_set_params(ctypes.c_void_p(net), ctypes.c_void_p(host_ptr), n),
           "tc_mlp_set_params")


def tc_mlp_get_params(net: int, host_ptr: int, n: int, working: bool = False) -> None:
    _check(lib.tc_mlp_get_params(ctypes.c_void_p(net), ctypes.c_void_p(host_ptr), n,
                                 1 if working else 0), "tc_mlp_get_params")


def tc_mlp_forward(net: int, X: int, Y: int, batch: int, stream: int = 0) -> None:
    _check(lib.tc_mlp_forward(ctypes.c_void_p(net), ctypes.c_void_p(X), ctypes.c_void_p(Y),
                              batch, ctypes.c_void_p(stream)), "tc_mlp_forward")


def tc_mlp_loss_grad(net: int, X: int, T: int, mask: int, batch: int, loss: int, grad: int,
                     stream: int = 0) -> None:
    _check(lib.tc_mlp_loss_grad(ctypes.c_void_p(net), ctypes.c_void_p(X), ctypes.c_void_p(T),
                                ctypes.c_void_p(mask), batch, ctypes.c_void_p(loss),
                                ctypes.c_void_p(grad), ctypes.c_void_p(stream)), "tc_mlp_loss_grad")


def tc_mlp_adam_step(net: int, grad: int, lr: float, beta1: float, beta2: float, eps: float,
                     t: int, stream: int = 0) -> None:
    _check(lib.tc_mlp_adam_step(ctypes.c_void_p(net), ctypes.c_void_p(grad), lr, beta1, beta2,
                                eps, t, ctypes.c_void_p(stream)), "tc_mlp_adam_step")


def tc_plan_features(plan: int):
    import numpy as np
    out = np.zeros(N_FEATURES, np.float32)
    _check(lib.tc_plan_features(ctypes.c_void_p(plan), ctypes.c_void_p(out.ctypes.data),
                                N_FEATURES), "tc_plan_features")
    return out


def tc_selector_load(path: str) -> None:
    _check(lib.tc_selector_load(str(path).encode()), "tc_selector_load")


def tc_selector_unload() -> None:
    lib.tc_selector_unload()


def tc_selector_predict(features):
    """features: float32 array [n, N_FEATURES] -> (pred [n, n_cand], candidate mappings)."""
    import numpy as np
    X = np.ascontiguousarray(features, np.float32).reshape(-1, N_FEATURES)
    out = np.zeros((X.shape[0], 16), np.float32)
    cand = np.zeros(16, np.int32)
    nc = ctypes.c_int32()
    _check(lib.tc_selector_predict(ctypes.c_void_p(X.ctypes.data), X.shape[0],
                                   ctypes.c_void_p(out.ctypes.data),
                                   ctypes.c_void_p(cand.ctypes.data), ctypes.byref(nc)),
           "tc_selector_predict")
    n = nc.value
    return out.reshape(-1)[: X.shape[0] * n].reshape(X.shape[0], n), cand[:n]
