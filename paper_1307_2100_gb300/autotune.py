"""Autotuner of a batch's routes: for each size bucket of its contractions,
the tensor-core route (128 x 128 tiles on packed BF16 terms) or the CUDA-core
route (partial sums per output over K segments), chosen by timing
tc_contract_batched on the GPU.

Buckets group the plans by log2 of min(M, N) and of K of their GEMM views.
Starting from the threshold rule (tc_batch_set_route), the buckets are
visited in order of decreasing flops and each one's route is flipped; a flip
is kept when the whole batch gets faster by more than `gain` (relative).  The
visit repeats (up to `passes` times) while a pass keeps a flip, since a
bucket's best route depends on the load the others leave on each route.
Plans with a batch group (the slicing mapping) stay on the CUDA-core route.
"""
from __future__ import annotations

import math as _math

import numpy as np

from . import tc


def bucket_of(M: int, N: int, K: int) -> tuple:
    """Size bucket of a GEMM view: (log2 min(M, N), log2 K / 2), capped."""
    mn = max(1, min(int(M), int(N)))
    return (min(int(_math.log2(mn)), 10), min(int(_math.log2(max(1, int(K)))) // 2, 10))


def default_routes(infos, tc_min_mn: int = 64) -> np.ndarray:
    """Routes of the threshold rule, made explicit (1 tensor cores, 0 CUDA cores)."""
    r = np.zeros(len(infos), np.int32)
    for i, d in enumerate(infos):
        if d.batch == 1 and d.M >= tc_min_mn and d.N >= tc_min_mn:
            r[i] = 1
    return r


def time_routes(plans, routes, ptrs, stream, reps: int = 5) -> float:
    """Median ms of tc_contract_batched for the given routes (after a warm-up)."""
    import torch
    pa, pb, pc, al, be = ptrs
    batch = tc.tc_batch_plan_routes(plans, routes)
    try:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        run = lambda: tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(),
                                             al.data_ptr(), be.data_ptr(), stream.cuda_stream)
        with torch.cuda.stream(stream):
            run()
            ts = []
            for _ in range(reps):
                e0.record(stream)
                run()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))
    finally:
        tc.tc_batch_destroy(batch)


def tune_routes(plans, ptrs, stream, reps: int = 5, gain: float = 0.02, tc_min_mn: int = 64,
                passes: int = 3):
    """Routes per plan (int32 array) and a report.  `plans` are plan handles,
    `ptrs` the device arrays (A, B, C pointers; alpha, beta) that
    tc_contract_batched takes, `stream` a torch CUDA stream."""
    infos = [tc.tc_plan_get_info(h) for h in plans]
    routes = default_routes(infos, tc_min_mn)
    movable = np.array([d.batch == 1 for d in infos])
    buckets = {}
    for i, d in enumerate(infos):
        if movable[i]:
            buckets.setdefault(bucket_of(d.M, d.N, d.K), []).append(i)
    flops = {b: sum(infos[i].flops for i in idx) for b, idx in buckets.items()}
    t0 = best = time_routes(plans, routes, ptrs, stream, reps)
    decisions = []
    for ps in range(passes):
        kept = 0
        for b in sorted(buckets, key=lambda b: -flops[b]):
            idx = buckets[b]
            trial = routes.copy()
            # a bucket split by the rule moves as a whole to the minority's route
            trial[idx] = 0 if routes[idx].mean() >= 0.5 else 1
            t = time_routes(plans, trial, ptrs, stream, reps)
            keep = t < best * (1.0 - gain)
            decisions.append({"pass": ps, "bucket": list(b), "items": len(idx),
                              "route": int(trial[idx[0]]), "ms": t, "kept": bool(keep)})
            if keep:
                routes, best = trial, t
                kept += 1
        if kept == 0:
            break
    report = {"buckets": len(buckets), "default_ms": t0, "tuned_ms": best,
              "tensor_core_items": int(routes.sum()), "trials": decisions}
    return routes, report
