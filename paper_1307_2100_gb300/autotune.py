"""Autotuner of a batch's routes and tile shapes: for each size bucket of its
contractions one of three kernels and shapes, chosen by timing
tc_contract_batched on the GPU:
  1  tensor cores, 128 x 128 output tiles on packed BF16 terms;
  2  CUDA cores, 32 x 32 output tiles over K segments;
  3  CUDA cores, a thread (or, below 256 outputs, a warp) per output.

Buckets group the plans by log2 of min(M, N) and of K of their GEMM views.
Starting from the threshold rule (tc_batch_set_route), the buckets are
visited in order of decreasing flops and each one is tried on the two
shapes it does not have; a change is kept when the whole batch gets faster
by more than `gain` (relative).  The visit repeats (up to `passes` times)
while a pass keeps a change, since a bucket's best shape depends on the
load the others leave on each route.  Plans with a batch group (the slicing
mapping) stay on the CUDA-core route.
"""
from __future__ import annotations

import math as _math

import numpy as np

from . import tc


def bucket_of(M: int, N: int, K: int) -> tuple:
    """Size bucket of a GEMM view: (log2 min(M, N), log2 K / 2), capped."""
    mn = max(1, min(int(M), int(N)))
    return (min(int(_math.log2(mn)), 10), min(int(_math.log2(max(1, int(K)))) // 2, 10))


TILE_MIN = 16   # the batch's rule: CUDA-core tiles where min(M, N) >= 16


def default_routes(infos, tc_min_mn: int = 64) -> np.ndarray:
    """Routes and shapes of the threshold rule, made explicit (1 tensor cores,
    2 CUDA-core tiles, 3 CUDA cores per output)."""
    r = np.zeros(len(infos), np.int32)
    for i, d in enumerate(infos):
        if d.batch == 1 and d.M >= tc_min_mn and d.N >= tc_min_mn:
            r[i] = 1
        else:
            r[i] = 2 if min(d.M, d.N) >= TILE_MIN else 3
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
            # a bucket split by the rule is tried whole on each shape but its
            # most common one
            vals, counts = np.unique(routes[idx], return_counts=True)
            now = int(vals[np.argmax(counts)])
            best_trial = None
            for shape in (1, 2, 3):
                if shape == now and len(vals) == 1:
                    continue
                trial = routes.copy()
                trial[idx] = shape
                t = time_routes(plans, trial, ptrs, stream, reps)
                decisions.append({"pass": ps, "bucket": list(b), "items": len(idx),
                                  "route": shape, "ms": t, "kept": False})
                if t < best * (1.0 - gain) and (best_trial is None or t < best_trial[1]):
                    best_trial = (trial, t, len(decisions) - 1)
            if best_trial is not None:
                routes, best = best_trial[0], best_trial[1]
                decisions[best_trial[2]]["kept"] = True
                kept += 1
        if kept == 0:
            break
    report = {"buckets": len(buckets), "default_ms": t0, "tuned_ms": best,
              "tensor_core_items": int((routes == 1).sum()),
              "cuda_core_tile_items": int((routes == 2).sum()),
              "cuda_core_output_items": int((routes == 3).sum()), "trials": decisions}
    return routes, report
