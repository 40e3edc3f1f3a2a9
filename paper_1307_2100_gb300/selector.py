"""The learned mapping selector: timing dataset, training and evaluation.

    python -m paper_1307_2100_gb300.selector generate --n 20000 --out sel_data.npz [--kind fp64]
    python -m paper_1307_2100_gb300.selector fill --data sel_data.npz --out sel_data.npz
    python -m paper_1307_2100_gb300.selector train --data sel_data.npz --out selector.bin
    python -m paper_1307_2100_gb300.selector evaluate --data sel_data.npz --weights selector.bin

A selector serves one storage type and math form (a "kind"):
  bf16x6  FP32 storage, BF16x6 math (the FP32-class form); candidates are a
          mapping and, for the fused and COPY+GEMM mappings, the
          packed-operand or the gathering tensor-core kernel;
  fp64    FP64 storage and math (the paper's own arithmetic); candidates are
          the CUDA-core GEMM's four tile shapes (64x64, 32x32, 128x64, 16x16) for
          the fused mapping, the slicing and COPY+GEMM mappings, GEMV, DOT and
          GER.  Its descriptors are those of the bf16x6 kind with at most
          2^34 flops (a second at the FP64 rate), so that timing stays bounded.
Every descriptor is planned under each candidate and timed by CUDA events
(median of a few runs after a warm-up).  The network (libtc's tc_mlp_* kernels: forward,
masked-MSE backward, Adam; FP16 working weights) learns the log2 runtime of
every candidate from the plan's features (tc_plan_features).  Regret of a
choice is t(choice) / t(best) - 1 against the same exhaustive timing table;
the paper's class recipe (Sec. 3.2) is the method the network is compared
with and falls back to.
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import sys
import time

import numpy as np

from . import tc

# (name, mapping, tile configuration; -1 = the plan's default).  The fused and
# COPY+GEMM mappings run on packed operands (tile 3) or on the gathering
# tensor-core kernel (tile 0); the slicing mapping's batches on the latter;
# GER (K <= 32) on the CUDA cores in FP32.  New candidates go at the end (the
# timing tables keep their columns).
KINDS = {
    "bf16x6": {"dtype": tc.TC_F32, "math": "bf16x6", "max_flops": None, "candidates": [
        ("fused_gemm", "fused_gemm", 3),
        ("fused_gemm_gather", "fused_gemm", 0),
        ("slice_gemm", "slice_gemm", -1),
        ("copy_gemm", "copy_gemm", 3),
        ("copy_gemm_gather", "copy_gemm", 0),
        ("gemv", "gemv", -1),
        ("dot", "dot", -1),
        ("ger", "ger", -1),
    ]},
    "fp64": {"dtype": tc.TC_F64, "math": "fp64", "max_flops": 2.0 ** 34, "candidates": [
        ("fused_gemm_64x64", "fused_gemm", 0),
        ("fused_gemm_32x32", "fused_gemm", 1),
        ("fused_gemm_128x64", "fused_gemm", 2),
        ("slice_gemm", "slice_gemm", -1),
        ("copy_gemm", "copy_gemm", -1),
        ("gemv", "gemv", -1),
        ("dot", "dot", -1),
        ("ger", "ger", -1),
        ("fused_gemm_16x16", "fused_gemm", 3),
    ]},
}
CANDIDATE_SPECS = KINDS["bf16x6"]["candidates"]
CANDIDATES = [c[0] for c in CANDIDATE_SPECS]
MATH = "bf16x6"
HIDDEN = 128


def specs(kind):
    return KINDS[kind]["candidates"]


def cand_ids(kind):
    return [tc.MAPPING[m] | ((t + 1) << 8) for _, m, t in specs(kind)]


CAND_IDS = cand_ids("bf16x6")


def _flops(desc):
    ext = {}
    for t in desc:
        for l, e in zip(t.labels, t.extents):
            ext[l] = int(e)
    f = 2.0
    for e in ext.values():
        f *= e
    return f


def descriptors(kind, n, seed):
    """The n descriptors of a kind's dataset (seeded): the selector workload's
    descriptors, for fp64 only those with at most 2^34 flops."""
    import tcsynth as ts
    cap = KINDS[kind]["max_flops"]
    if cap is None:
        return ts.selector_descriptors(n, seed=seed)
    m = n + n // 32 + 64
    while True:   # the generator's first m descriptors do not depend on m
        d = [x for x in ts.selector_descriptors(m, seed=seed) if _flops(x) <= cap]
        if len(d) >= n:
            return d[:n]
        m *= 2


def _desc(t):
    return (t.labels, t.extents, t.strides)


def _span(t):
    if any(e == 0 for e in t.extents):
        return 0
    return 1 + sum((e - 1) * s for e, s in zip(t.extents, t.strides))


def _timer(ws_bytes, dtype=None):
    """Device buffers and a function timing one planned candidate (median of
    `reps` runs after a warm-up, ms; None if the workspace does not fit)."""
    import torch
    dev = torch.device("cuda", 0)
    tdt = torch.float64 if dtype == tc.TC_F64 else torch.float32
    state = {"big": 0, "arena": None, "cbuf": None}
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def ensure(big):
        if big > state["big"]:
            state["arena"] = [torch.rand(big, device=dev, dtype=tdt) * 2 - 1 for _ in range(2)]
            state["cbuf"] = torch.zeros(big, device=dev, dtype=tdt)
            state["big"] = big

    def time_plan(h, reps):
        w = tc.tc_plan_get_info(h).workspace
        if w > ws.numel():
            return None
        arena, cbuf = state["arena"], state["cbuf"]
        args = (h, 1.0, arena[0].data_ptr(), arena[1].data_ptr(), 0.0, cbuf.data_ptr(),
                ws.data_ptr(), ws.numel(), s.cuda_stream)
        tc.tc_contract(*args)                        # warm-up
        times = []
        for _ in range(reps):
            e0.record(s)
            tc.tc_contract(*args)
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if times[0] > 50.0:                       # long runs: one sample
                break
        return float(np.median(times))

    return ensure, time_plan, s


def _time_candidates(desc, j, time_plan, reps, kind="bf16x6"):
    A, B, C = desc
    _, mname, tile = specs(kind)[j]
    k = KINDS[kind]
    try:
        h = tc.tc_plan(_desc(A), _desc(B), _desc(C), k["dtype"], tc.MATH[k["math"]],
                       tc.MAPPING[mname], tile)
    except tc.TcError:
        return None
    try:
        return time_plan(h, reps)
    finally:
        tc.tc_plan_destroy(h)


def generate(n, seed, out, reps=5, checkpoint=500, ws_bytes=1 << 28, log=sys.stderr,
             kind="bf16x6"):
    """Time every candidate of a kind on its n descriptors; save features,
    times (ms; NaN if the candidate cannot compute it or its workspace exceeds
    ws_bytes), class    and the recipe's choice."""
    descs = descriptors(kind, n, seed)
    k = KINDS[kind]
    ensure, time_plan, s = _timer(ws_bytes, k["dtype"])
    ensure(max(max(_span(a), _span(b), _span(c)) for a, b, c in descs))
    F = np.zeros((n, tc.N_FEATURES), np.float32)
    T = np.full((n, len(specs(kind))), np.nan, np.float64)
    cls = np.zeros(n, np.int32)
    recipe = np.zeros(n, np.int32)
    start = 0
    if os.path.exists(out + ".partial.npz"):
        z = np.load(out + ".partial.npz")
        start = int(z["done"])
        F[:start], T[:start], cls[:start], recipe[:start] = z["F"][:start], z["T"][:start], \
            z["cls"][:start], z["recipe"][:start]
    t0 = time.time()
    for i in range(start, n):
        A, B, C = descs[i]
        h = tc.tc_plan(_desc(A), _desc(B), _desc(C), k["dtype"], tc.MATH[k["math"]],
                       tc.MAPPING["recipe"])
        info = tc.tc_plan_get_info(h)
        F[i] = tc.tc_plan_features(h)
        cls[i] = info.cls
        recipe[i] = info.mapping
        tc.tc_plan_destroy(h)
        for j in range(len(specs(kind))):
            t = _time_candidates(descs[i], j, time_plan, reps, kind)
            if t is not None:
                T[i, j] = t
        if (i + 1) % checkpoint == 0 or i + 1 == n:
            np.savez(out + ".partial.npz", F=F, T=T, cls=cls, recipe=recipe, done=i + 1)
            print(f"[selector] {i + 1}/{n} descriptors, {time.time() - t0:.0f} s", file=log,
                  flush=True)
    if tc.tc_device_status(s.cuda_stream) != tc.TC_OK:
        raise RuntimeError("device status not ok after timing")
    np.savez(out, F=F, T=T, cls=cls, recipe=recipe, candidates=np.array(cand_ids(kind), np.int32),
             seed=seed, kind=kind)
    if os.path.exists(out + ".partial.npz"):
        os.remove(out + ".partial.npz")
    return out


def fill(data, out, reps=5, ws_bytes=1 << 31, log=sys.stderr):
    """Time the candidates a dataset lacks (NaN) whose plans exist and whose
    workspace fits ws_bytes; write the completed dataset to out."""
    z = dict(np.load(data))
    kind = _kind_of(z)
    T = z["T"].copy()
    nc = len(specs(kind))
    if T.shape[1] < nc:   # candidates added since: untimed columns
        T = np.concatenate([T, np.full((len(T), nc - T.shape[1]), np.nan)], 1)
        z["candidates"] = np.array(cand_ids(kind), np.int32)
    descs = descriptors(kind, len(T), int(z["seed"]))
    ensure, time_plan, s = _timer(ws_bytes, KINDS[kind]["dtype"])
    todo = [(i, j) for i, j in zip(*np.where(~np.isfinite(T)))]
    rows = sorted({i for i, _ in todo})
    if rows:
        ensure(max(max(_span(a), _span(b), _span(c)) for a, b, c in (descs[i] for i in rows)))
    filled = 0
    for i, j in todo:
        t = _time_candidates(descs[i], j, time_plan, reps, kind)
        if t is not None:
            T[i, j] = t
            filled += 1
    if tc.tc_device_status(s.cuda_stream) != tc.TC_OK:
        raise RuntimeError("device status not ok after timing")
    print(f"[selector] filled {filled} of {len(todo)} missing timings", file=log, flush=True)
    z["T"] = T
    np.savez(out, **z)
    return out


def _kind_of(z):
    return str(z["kind"]) if "kind" in z else "bf16x6"


def split(n, holdout, seed=1):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    return perm[holdout:], perm[:holdout]


def _targets(T):
    """log2 of the runtime in microseconds; mask of candidates that ran."""
    mask = np.isfinite(T)
    Y = np.where(mask, np.log2(np.maximum(np.nan_to_num(T, nan=1.0), 1e-6) * 1e3), 0.0)
    return Y.astype(np.float32), mask.astype(np.float32)


def train(data, out, holdout=2000, epochs=400, batch=256, lr=2e-3, seed=0, log=sys.stderr):
    """Train the network on the GPU with libtc's kernels and write the
    selector file read by tc_selector_load."""
    import torch
    z = np.load(data)
    kind = _kind_of(z)
    F, T = z["F"].astype(np.float32), z["T"]
    tr, _ = split(len(F), holdout)
    Y, M = _targets(T)
    lo, hi = F[tr].min(axis=0), F[tr].max(axis=0)
    mean = F[tr].mean(axis=0)
    std = F[tr].std(axis=0)
    scale = np.where(std > 1e-6, 1.0 / np.maximum(std, 1e-6), 0.0).astype(np.float32)
    ym = float((Y[tr] * M[tr]).sum() / M[tr].sum())
    ys = float(np.sqrt(((Y[tr] - ym) ** 2 * M[tr]).sum() / M[tr].sum()))
    Xn = ((F - mean) * scale).astype(np.float32)
    Yn = ((Y - ym) / ys).astype(np.float32)
    dev = torch.device("cuda", 0)
    n_in, n_out = F.shape[1], T.shape[1]
    net = tc.tc_mlp_create(n_in, HIDDEN, n_out, batch)
    try:
        n_par = tc.tc_mlp_num_params(net)
        rng = np.random.default_rng(seed)
        theta = []
        for shape in ((HIDDEN, n_in), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (n_out, HIDDEN),
                      (n_out,)):
            if len(shape) == 2:   # He-uniform initialisation
                lim = np.sqrt(6.0 / shape[1])
                theta.append(rng.uniform(-lim, lim, shape).ravel())
            else:
                theta.append(np.zeros(shape))
        theta = np.concatenate(theta).astype(np.float32)
        assert theta.size == n_par
        tc.tc_mlp_set_params(net, theta.ctypes.data, n_par)
        dX = torch.from_numpy(Xn[tr]).to(dev)
        dY = torch.from_numpy(Yn[tr]).to(dev)
        dM = torch.from_numpy(M[tr]).to(dev)
        loss = torch.zeros(1, device=dev)
        grad = torch.zeros(n_par, device=dev)
        ntr = len(tr)
        step = 0
        hist = []
        for ep in range(epochs):
            perm = torch.from_numpy(np.random.default_rng(seed + ep).permutation(ntr)).to(dev)
            tot = 0.0
            nb = 0
            for b0 in range(0, ntr - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                xb, yb, mb = dX[idx].contiguous(), dY[idx].contiguous(), dM[idx].contiguous()
                tc.tc_mlp_loss_grad(net, xb.data_ptr(), yb.data_ptr(), mb.data_ptr(), batch,
                                    loss.data_ptr(), grad.data_ptr())
                step += 1
                cur = lr * 0.5 * (1 + np.cos(np.pi * ep / epochs))   # cosine schedule
                tc.tc_mlp_adam_step(net, grad.data_ptr(), float(cur), 0.9, 0.999, 1e-8, step)
                tot += float(loss.item()) if b0 == 0 else 0.0
                nb += 1
            hist.append(tot)
            if ep % 50 == 0 or ep == epochs - 1:
                print(f"[selector] epoch {ep} loss {tot:.4f}", file=log, flush=True)
        work = np.empty(n_par, np.float32)
        tc.tc_mlp_get_params(net, work.ctypes.data, n_par, working=True)
    finally:
        tc.tc_mlp_destroy(net)
    write_weights(out, n_in, HIDDEN, n_out, cand_ids(kind), lo, hi, mean, scale, ym, ys, work,
                  KINDS[kind]["dtype"], KINDS[kind]["math"])
    return out


def write_weights(path, n_in, n_hidden, n_out, cand, lo, hi, mean, scale, ym, ys, params,
                  dtype=tc.TC_F32, math=MATH):
    with open(path, "wb") as f:
        f.write(b"TCSEL01\0")
        f.write(struct.pack("<5i", n_in, n_hidden, n_out, dtype, tc.MATH[math]))
        f.write(np.asarray(cand, "<i4").tobytes())
        for a in (lo, hi, mean, scale):
            f.write(np.asarray(a, "<f4").tobytes())
        f.write(struct.pack("<2f", ym, ys))
        f.write(np.asarray(params, np.float32).astype("<f2").tobytes())


def feasible(cls, kind="bf16x6"):
    """Candidates able to compute a contraction of the given class: slicing and
    COPY+GEMM need a free index in each operand (Class 3); GER's limit on K
    shows as a missing timing."""
    ok = np.ones((len(cls), len(specs(kind))), bool)
    c3 = np.isin(cls, [31, 32])
    for j, (_, mname, _t) in enumerate(specs(kind)):
        if mname in ("slice_gemm", "copy_gemm"):
            ok[~c3, j] = False
    return ok


def planned_candidates(seed, n, holdout, mapping="recipe", kind="bf16x6"):
    """Candidate index of what tc_plan decides (mapping and tile) for each
    held-out descriptor, planned again on the host: mapping "recipe" is the
    paper's recipe, "auto" the loaded selector."""
    descs = descriptors(kind, n, seed)
    _, te = split(n, holdout)
    k = KINDS[kind]
    spec = {(tc.MAPPING[m], t): j for j, (_, m, t) in enumerate(specs(kind))}
    out = np.zeros(len(te), np.int64)
    for r, i in enumerate(te):
        A, B, C = descs[i]
        h = tc.tc_plan(_desc(A), _desc(B), _desc(C), k["dtype"], tc.MATH[k["math"]],
                       tc.MAPPING[mapping])
        try:
            info = tc.tc_plan_get_info(h)
        finally:
            tc.tc_plan_destroy(h)
        m, t = int(info.mapping), int(info.tile)
        out[r] = spec.get((m, t), spec.get((m, -1), 0))
    return out


def regret_stats(choice_t, best_t):
    r = choice_t / best_t - 1.0
    return {"mean": float(np.mean(r)), "median": float(np.median(r)),
            "p90": float(np.percentile(r, 90)), "max": float(np.max(r))}


def evaluate(data, weights, holdout=2000, use_gpu=True):
    """Regret of the network, of the recipe, and of each fixed candidate on the
    held-out descriptors (timings from the dataset)."""
    z = np.load(data)
    kind = _kind_of(z)
    F, T, cls, recipe = z["F"].astype(np.float32), z["T"], z["cls"], z["recipe"]
    _, te = split(len(F), holdout)
    F, T, cls, recipe = F[te], T[te], cls[te], recipe[te]
    ran = np.isfinite(T)
    keep = ran.any(axis=1)
    F, T, cls, recipe, ran = F[keep], T[keep], cls[keep], recipe[keep], ran[keep]
    ok = feasible(cls, kind) & ran
    best = np.where(ok, T, np.inf).min(axis=1)
    seed, n_all = int(z["seed"]), len(z["F"])
    tc.tc_selector_load(weights)
    try:
        pred, cand = tc.tc_selector_predict(F)
        # what tc_plan(AUTO) runs with this network loaded
        choice = planned_candidates(seed, n_all, holdout, "auto", kind)[keep]
    finally:
        tc.tc_selector_unload()
    gpu_pred = None
    if use_gpu:
        gpu_pred = gpu_forward(weights, F)
    t_choice = T[np.arange(len(T)), choice]
    rec_idx = planned_candidates(seed, n_all, holdout, "recipe", kind)[keep]
    t_recipe = np.where(ok[np.arange(len(T)), rec_idx], T[np.arange(len(T)), rec_idx], np.inf)
    res = {"kind": kind, "n": int(len(T)), "network": regret_stats(t_choice, best),
           "recipe": regret_stats(t_recipe, best),
           "total_time_ms": {"network": float(t_choice.sum()), "recipe": float(t_recipe.sum()),
                             "best": float(best.sum())}}
    for j, (c, _m, _t) in enumerate(specs(kind)):
        tj = np.where(ok[:, j], T[:, j], np.inf)
        fin = np.isfinite(tj)
        res["always_" + c] = {"coverage": float(fin.mean()),
                              "mean_regret_where_feasible": float(np.mean(tj[fin] / best[fin] - 1))}
    if gpu_pred is not None:
        res["gpu_host_max_abs_diff"] = float(np.max(np.abs(gpu_pred - pred)))
    return res


def gpu_forward(weights, F):
    """The trained network on the GPU (libtc's forward kernel) for rows of F;
    returns de-normalised log2 runtimes like tc_selector_predict."""
    import torch
    with open(weights, "rb") as f:
        raw = f.read()
    n_in, n_hidden, n_out, _, _ = struct.unpack("<5i", raw[8:28])
    off = 28 + 4 * n_out
    vec = []
    for _ in range(4):          # lo, hi, mean, scale
        vec.append(np.frombuffer(raw, "<f4", n_in, off))
        off += 4 * n_in
    mean, scale = vec[2], vec[3]
    ym, ys = struct.unpack("<2f", raw[off:off + 8])
    params = np.frombuffer(raw, "<f2", -1, off + 8).astype(np.float32)
    dev = torch.device("cuda", 0)
    X = torch.from_numpy(((F - mean) * scale).astype(np.float32)).to(dev)
    Y = torch.empty(len(F), n_out, device=dev)
    net = tc.tc_mlp_create(n_in, n_hidden, n_out, max(len(F), 1))
    try:
        tc.tc_mlp_set_params(net, np.ascontiguousarray(params).ctypes.data, params.size)
        tc.tc_mlp_forward(net, X.data_ptr(), Y.data_ptr(), len(F))
        torch.cuda.synchronize()
    finally:
        tc.tc_mlp_destroy(net)
    return Y.cpu().numpy() * ys + ym


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("generate")
    g.add_argument("--n", type=int, default=20000)
    g.add_argument("--seed", type=int, default=20130712)
    g.add_argument("--out", required=True)
    g.add_argument("--reps", type=int, default=5)
    g.add_argument("--kind", default="bf16x6", choices=sorted(KINDS))
    g.add_argument("--ws-gb", type=float, default=2.0)
    t = sub.add_parser("train")
    t.add_argument("--data", required=True)
    t.add_argument("--out", required=True)
    t.add_argument("--epochs", type=int, default=400)
    t.add_argument("--holdout", type=int, default=2000)
    fl = sub.add_parser("fill")
    fl.add_argument("--data", required=True)
    fl.add_argument("--out", required=True)
    fl.add_argument("--ws-gb", type=float, default=2.0)
    e = sub.add_parser("evaluate")
    e.add_argument("--data", required=True)
    e.add_argument("--weights", required=True)
    e.add_argument("--holdout", type=int, default=2000)
    a = ap.parse_args(argv)
    if a.cmd == "generate":
        generate(a.n, a.seed, a.out, a.reps, ws_bytes=int(a.ws_gb * (1 << 30)), kind=a.kind)
    elif a.cmd == "fill":
        fill(a.data, a.out, ws_bytes=int(a.ws_gb * (1 << 30)))
    elif a.cmd == "train":
        train(a.data, a.out, a.holdout, a.epochs)
    else:
        print(json.dumps(evaluate(a.data, a.weights, a.holdout)))


if __name__ == "__main__":
    main()
