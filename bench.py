#!/usr/bin/env python
"""Benchmark of the contraction path on one or more GB300 GPUs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass over the plain-method workload of the three classes, in
FP64 with the planner's automatic mapping:
  (i)   C[a,b,c,d] = sum_{i,j} A[a,i,j,b] B[i,j,c,d], extents 64  (Class 3.2, GEMM)
  (ii)  C[a,b,c,d] = sum_{i,j} A[i,a,j,b] B[j,c,i,d], extents 48  (Class 3.1, fused permute)
  (iii) C[a,b]     = sum_i     A[a,i,b]   B[i], a=b=1024, i=2048  (Class 2, GEMV)
Inputs are seeded uniform[-1,1) values (synthetic: the paper publishes no
data).  The L2 cache is flushed (256 MiB write) between timed steps, outside
the timed region.  Rank 0 prints one JSON line.

--impl reference times the CPU oracle (the plain FP64 loop nest) on the
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import tcsynth as ts  # noqa: E402

METRIC = ("contraction TFLOP/s & % roofline vs plain FP64 path at ≤1e-6 rel err; "
          "selector regret")
WORKLOAD = "plain FP64, three classes: (i) direct GEMM 64^6, (ii) fused permute 48^6, (iii) GEMV 1024x2048x1024"
N_SMS = 152
FP64_FLOP_PER_CLK_SM = 4     # nominal 1.25 TFLOP/s = 152 SMs x 4 flop/clk x 2.07 GHz
L2_FLUSH_BYTES = 256 << 20


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def replica_throughput(local_ms, units_per_rank, world, device="cpu"):
    """Replicas only: every rank runs the same workload.  Returns (slowest
    rank's ms, whole-job units per second / 1e12): the ranks' times are
    combined by an all-reduce MAX (no collective on the data path), and the
    units of all ranks count toward the value."""
    ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms / 1e3) / 1e12


def workloads(alloc=None, only=None, kind="class3_fp64", precision_v=128, gemv_b=1024):
    if kind == "precision":
        return [ts.precision_ccd(v=precision_v)]
    makers = {"direct_gemm_64": ts.direct_gemm_64, "fused_permute_48": ts.fused_permute_48,
              "gemv_1024": lambda: ts.gemv_1024_full(b=gemv_b, alloc=alloc)}
    names = list(makers) if not only else [n for n in only.split(",") if n]
    return [makers[n]() for n in names]


NPROD = {"bf16": 1, "bf16x3": 3, "bf16x6": 6}
FP8_PER_BF16 = 2.0   # nominal dense tensor rate of E4M3 over BF16 (4.5 / 2.25 PFLOP/s)


def sampled_error(p, got, nsamp=64):
    """Relative Frobenius error of sampled outputs against the FP64 oracle."""
    import oracle
    rng = np.random.default_rng(7)
    con = [l for l in p.A.labels if l in p.B.labels]
    ref, val = [], []
    for _ in range(nsamp):
        cidx = tuple(int(rng.integers(0, e)) for e in p.C.extents)
        fix = dict(zip(p.C.labels, cidx))
        parts = []
        for t in (p.A, p.B):
            off = sum(fix[l] * st for l, st in zip(t.labels, t.strides) if l in fix)
            keep = [k for k, l in enumerate(t.labels) if l in con]
            ext = [t.extents[k] for k in keep]
            stv = [t.strides[k] for k in keep]
            parts.append(([t.labels[k] for k in keep], ext, stv,
                          np.asarray(t.data[off:off + ts.span(ext, stv)], np.float64)))
        c = np.zeros(1)
        (la, ea, sa, a), (lb, eb, sb, b) = parts
        oracle.contract_raw(la, ea, sa, a, lb, eb, sb, b, [], [], [], c, 1.0, 0.0)
        ref.append(c[0])
        val.append(float(got[sum(i * st for i, st in zip(cidx, p.C.strides))]))
    return oracle.rel_fro(np.array(val), np.array(ref))


def read_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Sources each dominant kernel is built from: an ncu traffic figure recorded
# in profiles/ is used only while these files still hash to the value
# recorded with it.
KERNEL_SOURCES = {
    "gemm_simt": ["paper_1307_2100_gb300/csrc/k_simt.cu", "paper_1307_2100_gb300/csrc/groups.cuh",
                  "paper_1307_2100_gb300/csrc/tc_internal.h"],
}
TRAFFIC_FILES = {("gemm_simt", "direct_gemm_64"): "profiles/gemm_simt_fp64_direct_gemm_64.md"}


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
    the committed ncu summary of this kernel and workload, if its line
    'traffic_bytes_per_launch: B sources_sha256: H' still matches the sources."""
    f = TRAFFIC_FILES.get((kernel, workload))
    if f is None or kernel not in KERNEL_SOURCES:
        return None
    try:
        with open(os.path.join(ROOT, f)) as fh:
            for line in fh:
                if line.startswith("traffic_bytes_per_launch:"):
                    w = line.split()
                    if w[2] == "sources_sha256:" and w[3] == source_hash(kernel):
                        return float(w[1])
    except (OSError, IndexError, ValueError):
        pass
    return None


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r["sm"] for r in rows])),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample_problems(target_s: float, nthreads: int):
    """Bounded samples of the three contractions for the CPU oracle: the last
    free label of C is cut to s values, s chosen so each takes ~target_s."""
    import oracle
    full = [ts.direct_gemm_64(), ts.fused_permute_48(), None]
    out = []
    for j, p in enumerate(full):
        def cut(s, p=p, j=j):
            if j == 2:
                q = ts.gemv_1024_full(b=s)
                return q
            lastc = p.C.labels[-1]
            q = ts.Problem(p.name, p.A, p.B, p.C)
            for name in ("A", "B", "C"):
                t = getattr(p, name)
                if lastc in t.labels:
                    k = t.labels.index(lastc)
                    ext = list(t.extents)
                    ext[k] = s
                    n = ts.span(ext, t.strides)
                    setattr(q, name, ts.Tensor(t.labels, ext, t.strides, t.data[:n]))
            return q
        maxs = 1024 if j == 2 else p.C.extents[-1]
        q = cut(1)
        t0 = time.perf_counter()
        oracle.contract_problem(q, nthreads=nthreads)
        t1 = max(time.perf_counter() - t0, 1e-4)
        s = int(max(1, min(maxs, round(target_s / t1))))
        out.append(cut(s))
    return out


def time_oracle(problems, nthreads):
    import oracle
    t0 = time.perf_counter()
    for q in problems:
        oracle.contract_problem(q, nthreads=nthreads)
    return time.perf_counter() - t0


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def sample_desc(problems):
    return "; ".join(f"{q.name} with last output index cut to {q.C.extents[-1]}"
                     for q in problems)


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nth = cores()
    probs = oracle_sample_problems(1.5, nth)
    flops = sum(q.flops() for q in probs)
    for _ in range(args.warmup):
        time_oracle(probs, nth)
    times = [time_oracle(probs, nth) for _ in range(args.steps)]
    total = sum(times)
    value = flops * len(times) / total / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "bounded CPU sample per step"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": nth, "kind": "oracle",
                         "sample": sample_desc(probs)},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def launches_of(info) -> int:
    n = 2 if ((info.kernel == 4 and info.M * info.N * info.batch == 1) or info.kernel == 5) else 1
    return n + (1 if info.mapping == 4 else 0)


def run_ours(args):
    import torch
    rank, local_rank, world = env_rank()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_1307_2100_gb300 import build as _b
    _b.build()
    from paper_1307_2100_gb300 import Contraction, tc

    def pinned(n, dtype):
        t = torch.empty(n, dtype=torch.float64 if dtype == np.float64 else torch.float32,
                        pin_memory=True)
        return t.numpy()

    probs = workloads(alloc=pinned, only=args.only, kind=args.workload,
                      precision_v=args.precision_v, gemv_b=args.gemv_b)
    fp64 = args.workload == "class3_fp64"
    math = "fp64" if fp64 else args.math
    tdt = torch.float64 if fp64 else torch.float32
    plans, dA, dB, dC = [], [], [], []
    for p in probs:
        pl = Contraction((p.A.labels, p.A.extents, p.A.strides),
                         (p.B.labels, p.B.extents, p.B.strides),
                         (p.C.labels, p.C.extents, p.C.strides), "f64" if fp64 else "f32",
                         math, args.mapping, args.tile)
        plans.append(pl)
        dA.append(torch.from_numpy(np.ascontiguousarray(p.A.data)).to(dev))
        dB.append(torch.from_numpy(np.ascontiguousarray(p.B.data)).to(dev))
        dC.append(torch.empty(p.C.data.size, dtype=tdt, device=dev))
    def host_pinned(a):
        t = torch.from_numpy(a)
        return t if t.is_pinned() else t.pin_memory()

    hA = [host_pinned(p.A.data) for p in probs]
    hB = [host_pinned(p.B.data) for p in probs]
    hC = [torch.empty(c.numel(), dtype=c.dtype, pin_memory=True) for c in dC]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    ws = [pl.workspace(dev) for pl in plans]

    def contract(j):
        w = ws[j]
        tc.tc_contract(plans[j].handle, 1.0, dA[j].data_ptr(), dB[j].data_ptr(), 0.0,
                       dC[j].data_ptr(), w.data_ptr() if w is not None else 0,
                       w.numel() if w is not None else 0, sptr)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    nprob = len(probs)
    for _ in range(args.warmup):
        for j in range(nprob):
            contract(j)
    torch.cuda.synchronize()
    if tc.tc_device_status(sptr) != tc.TC_OK:
        raise RuntimeError("device status not ok after warm-up")

    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nprob)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                     # L2 flush, outside the events
        for j in range(nprob):
            ev[k][j][0].record(stream)
            contract(j)
            ev[k][j][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    per = np.array([[ev[k][j][0].elapsed_time(ev[k][j][1]) for j in range(nprob)]
                    for k in range(args.steps)])        # ms
    step_ms = per.sum(axis=1)
    flops_step = sum(p.flops() for p in probs)
    total_ms, value = replica_throughput(step_ms.sum(), flops_step * args.steps, world, dev)

    # ---- e2e: host buffers, copies inside the timed region.  Inputs go up on
    # one copy stream and results come down on another, so that the copies of
    # one contraction overlap the compute of the others; events order each
    # buffer's uses (a step's upload of A, B after the previous step's
    # contraction read them; a contraction's write of C after the previous
    # step's download of it).
    h2d = sum(p.A.data.nbytes + p.B.data.nbytes for p in probs)
    d2h = sum(c.numel() * c.element_size() for c in dC)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: [torch.cuda.Event() for _ in range(nprob)]
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    up.wait_event(e0)
    down.wait_event(e0)
    done, fetched = None, None
    for _ in range(args.steps if not args.no_e2e else 0):
        ready, done_k, fetched_k = ev(), ev(), ev()
        for j in range(nprob):
            if done is not None:
                up.wait_event(done[j])
            with torch.cuda.stream(up):
                dA[j].copy_(hA[j], non_blocking=True)
                dB[j].copy_(hB[j], non_blocking=True)
            ready[j].record(up)
        for j in range(nprob):
            stream.wait_event(ready[j])
            if fetched is not None:
                stream.wait_event(fetched[j])
            contract(j)
            done_k[j].record(stream)
            down.wait_event(done_k[j])
            with torch.cuda.stream(down):
                hC[j].copy_(dC[j], non_blocking=True)
            fetched_k[j].record(down)
        done, fetched = done_k, fetched_k
    stream.wait_stream(up)
    stream.wait_stream(down)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms, e2e_value = replica_throughput(max(e0.elapsed_time(e1), 1e-6),
                                           flops_step * args.steps, world, dev)
    status = tc.tc_device_status(sptr)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs", 6784.5)
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = N_SMS * FP64_FLOP_PER_CLK_SM * sm_mhz * 1e6 / 1e12  # TFLOP/s
    bf16_peak = peaks.get("bf16_tflops", 1884.0)
    parts = []
    for j, p in enumerate(probs):
        info = plans[j].info
        kms = float(per[:, j].mean())
        if info.kernel == 5:  # FP8 form: one E4M3 product per multiply-add
            cpeak, work, cbound = bf16_peak * FP8_PER_BF16, p.flops(), "tensor"
        elif fp64 or info.kernel != 2:
            cpeak, work, cbound = fp64_peak if fp64 else 77.7, p.flops(), "alu"
        else:  # tensor-core forms: NPROD BF16 products per logical multiply-add
            cpeak, work, cbound = bf16_peak, p.flops() * NPROD[math], "tensor"
        t_alu = work / (cpeak * 1e12)
        t_mem = p.min_bytes() / (hbm * 1e9)
        bound = cbound if t_alu >= t_mem else "hbm"
        achieved = work / (kms / 1e3) / 1e12 if bound != "hbm" else \
            p.min_bytes() / (kms / 1e3) / 1e9
        peak = cpeak if bound != "hbm" else hbm
        parts.append({"name": p.name, "class": int(info.cls),
                      "mapping": tc.MAPPING_NAME[info.mapping],
                      "kernel": tc.KERNEL_NAME[info.kernel], "ms": kms,
                      "tflops": p.flops() / (kms / 1e3) / 1e12,
                      "bound": bound, "achieved": achieved, "peak": peak,
                      "unit": "TFLOP/s" if bound != "hbm" else "GB/s",
                      "frac": achieved / peak,
                      "roofline_ms": 1e3 * max(t_alu, t_mem)})
    if not fp64:
        for j, p in enumerate(probs):
            parts[j]["rel_err_vs_fp64_oracle_sampled"] = sampled_error(
                p, dC[j].cpu().numpy().astype(np.float64))
    dom = max(parts, key=lambda d: d["ms"])
    traffic = recorded_traffic(dom["kernel"], dom["name"])
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp64 else "f32 storage, " + math,
        "data": "synthetic (seeded uniform[-1,1), shapes of the paper's Eq. xy and Class 2)",
        "config": {"workload": (WORKLOAD if not args.only and args.gemv_b == 1024 else
                                f"plain FP64: {args.only or 'three classes'}, GEMV b={args.gemv_b}")
                   if fp64 else
                   f"precision: CCD-like {args.precision_v}^4 x {args.precision_v}^2*32^2",
                   "mapping": "auto (recipe)" if args.mapping == "auto" else args.mapping,
                   "math": math,
                   "l2": "flushed between steps (256 MiB write, outside timing)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": dom["bound"], "kernel": dom["kernel"], "workload": dom["name"],
                     "achieved": dom["achieved"], "peak": dom["peak"], "unit": dom["unit"],
                     "frac": dom["frac"], "traffic": traffic,
                     "peak_source": (("derived: 152 SMs x 4 FP64 flop/clk x median SM clock "
                                      f"{sm_mhz:.0f} MHz") if dom["bound"] == "alu"
                                     else "measured bf16_tflops burst (MEASURED_PEAKS.json) x 2 "
                                     "(nominal FP8/BF16 dense ratio); achieved = FLOPs over the "
                                     "pack pass and the GEMM"
                                     if dom["bound"] == "tensor" and math == "fp8"
                                     else "measured bf16_tflops burst (MEASURED_PEAKS.json); "
                                     "achieved counts every BF16 product"
                                     if dom["bound"] == "tensor"
                                     else "measured hbm_gbs (MEASURED_PEAKS.json)")},
        "parts": parts,
        "e2e": None if args.no_e2e else {
            "value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms / args.steps,
            "copies": "pinned host buffers; uploads and downloads on their own streams, "
                      "overlapping the other contractions' compute"},
        "gpu_launches": int(args.steps * sum(launches_of(pl.info) for pl in plans)),
        "clocks": clk,
        "device_status": tc.tc_status_string(status),
        "wall_s": wall,
    }
    if world == 1 and not args.no_cpu_baseline and fp64:
        import oracle
        oracle.build()
        nth = cores()
        sprobs = oracle_sample_problems(3.0, nth)
        t = time_oracle(sprobs, nth)
        line["cpu_baseline"] = {"value": sum(q.flops() for q in sprobs) / t / 1e12,
                                "unit": "TFLOP/s", "cores": nth, "kind": "oracle",
                                "sample": sample_desc(sprobs), "seconds": t}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batching(args):
    """512 independent contractions (orders 2-5, extents log-uniform in
    [8, 192], 1-3 contracted indices, random storage orders, FP32) in one
    graph-captured tc_contract_batched, against 512 tc_contract calls."""
    import torch
    import oracle
    from paper_1307_2100_gb300 import build as _b
    _b.build()
    from paper_1307_2100_gb300 import Contraction, tc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    items = ts.batching_items(args.items)
    math = args.math
    plans, bufs = [], []
    for p in items:
        plans.append(Contraction((p.A.labels, p.A.extents, p.A.strides),
                                 (p.B.labels, p.B.extents, p.B.strides),
                                 (p.C.labels, p.C.extents, p.C.strides), "f32", math, "auto"))
        bufs.append((torch.from_numpy(p.A.data).to(dev), torch.from_numpy(p.B.data).to(dev),
                     torch.empty(max(p.C.data.size, 1), dtype=torch.float32, device=dev)))
    ptr = lambda k: torch.tensor([b[k].data_ptr() for b in bufs], dtype=torch.int64, device=dev)
    pa, pb, pc = ptr(0), ptr(1), ptr(2)
    al = torch.ones(len(items), dtype=torch.float64, device=dev)
    be = torch.zeros(len(items), dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(device=dev)
    handles = [pl.handle for pl in plans]
    tuned = None
    if args.no_autotune:
        batch = tc.tc_batch_plan(handles)
    else:  # routes per size bucket, chosen by timing (outside the timed region)
        from paper_1307_2100_gb300 import autotune
        routes, tuned = autotune.tune_routes(handles, (pa, pb, pc, al, be), s)
        batch = tc.tc_batch_plan_routes(handles, routes)
    info = tc.tc_batch_get_info(batch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ws = [pl.workspace(dev) for pl in plans]

    def batched():
        tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(), al.data_ptr(),
                               be.data_ptr(), s.cuda_stream)

    def separate():
        for j, pl in enumerate(plans):
            w = ws[j]
            tc.tc_contract(pl.handle, 1.0, bufs[j][0].data_ptr(), bufs[j][1].data_ptr(), 0.0,
                           bufs[j][2].data_ptr(), w.data_ptr() if w is not None else 0,
                           w.numel() if w is not None else 0, s.cuda_stream)

    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            batched()
            if not args.no_separate:
                separate()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batched()

    def timed(fn):
        ts_ = []
        for _ in range(args.steps):
            with torch.cuda.stream(s):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fn()
                e1.record(s)
            torch.cuda.synchronize()
            ts_.append(e0.elapsed_time(e1))
        return float(np.median(ts_)), ts_

    clocks = ClockSampler(0)
    clocks.start()
    t_graph, all_graph = timed(g.replay)
    t_sep = None if args.no_separate else timed(separate)[0]
    clk = clocks.stop()
    status = tc.tc_device_status(s.cuda_stream)
    # accuracy of every item against the FP64 oracle
    g.replay()
    torch.cuda.synchronize()
    errs = []
    for p, b in zip(items, bufs):
        got = b[2].cpu().numpy().astype(np.float64)[: p.C.data.size]
        errs.append(oracle.rel_fro(got, oracle.contract_problem(p, nthreads=cores())))
    tc.tc_batch_destroy(batch)
    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs", 6784.5)
    bf16_peak = peaks.get("bf16_tflops", 1884.0)
    flops = info.flops
    roof_ms = 1e3 * max(flops * NPROD[math] / (bf16_peak * 1e12), info.min_bytes / (hbm * 1e9))
    value = flops / (t_graph / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_graph, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 storage, " + math,
        "data": "synthetic (seeded uniform[-1,1); shapes of the batched workload)",
        "config": {"workload": f"batching: {len(items)} contractions, orders 2-5, extents "
                               "log-uniform [8,192], 1-3 contracted, random storage orders",
                   "l2": "flushed between steps (256 MiB write, outside timing)",
                   "launch": "one CUDA graph of tc_contract_batched",
                   "routes": "threshold rule" if args.no_autotune else
                   "autotuned per size bucket (paper_1307_2100_gb300/autotune.py)"},
        "roofline": {"bound": "hbm" if info.min_bytes / (hbm * 1e9) >
                     flops * NPROD[math] / (bf16_peak * 1e12) else "tensor",
                     "achieved_ms": t_graph, "roofline_ms": roof_ms, "frac": roof_ms / t_graph,
                     "traffic": None},
        "batched_vs_separate": None if t_sep is None else {
            "batched_ms": t_graph, "separate_ms": t_sep, "speedup": t_sep / t_graph},
        "routes": {"tensor_core_items": info.n_tc_items, "cuda_core_items": info.n_simt_items,
                   "tc_tiles": info.n_tiles, "simt_work": info.n_simt_work,
                   "simt_tiles": info.n_simt_tiles, "tc_split_tiles": info.n_tc_split},
        "autotune": None if tuned is None else {
            "buckets": tuned["buckets"], "default_ms": tuned["default_ms"],
            "tuned_ms": tuned["tuned_ms"],
            "flipped": [t["bucket"] for t in tuned["trials"] if t["kept"]]},
        "rel_err_vs_fp64_oracle": {"max": float(np.max(errs)), "median": float(np.median(errs))},
        "sum_flops": flops, "sum_bytes": info.min_bytes, "clocks": clk,
        "device_status": tc.tc_status_string(status),
        "gpu_launches": args.steps * (2 * int(info.n_tiles > 0) + int(info.n_tc_split > 0) +
                                      int(info.n_simt_work > 0) +
                                      int(info.n_simt_tiles > 0) +
                                      int(info.n_simt_work + info.n_simt_tiles > 0)),
    }
    print(json.dumps(line), flush=True)
    return 0


SKEWED = [(30, 100), (30, 300), (30, 600), (100, 4), (300, 4)]   # (free a=c=d, occupied i=j)


def run_skewed(args):
    """The skewed CCD / GR suite of Sec. 4.2: R[a,b,c,d] = sum_{i,j}
    X[i,a,j,b] Y[i,c,j,d] with a = c = d = free, b = 8, i = j = occ; short free
    and long contracted extents (CCD) and the GR case i = j = 4.  Each shape
    runs in FP64 on the recipe's mapping (and on GER where K <= 32), and with
    FP32 storage in BF16x6 on the selector's choice (the packaged GB300
    selector; outside its training range it falls back to the recipe), on
    packed operands, and on GER where K <= 32.  Sampled outputs against the
    FP64 oracle for every run."""
    import torch
    from paper_1307_2100_gb300 import build as _b
    _b.build()
    from paper_1307_2100_gb300 import Contraction, tc
    import os
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    sel = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1307_2100_gb300",
                       "data", "selector_gb300.bin")
    tc.tc_selector_load(sel)
    s = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(0)
    clocks.start()
    parts = []
    for free, occ in SKEWED:
        p64 = ts.ccd_skewed(free, occ)
        p32 = ts.ccd_skewed(free, occ, dtype=np.float32)
        K = occ * occ
        runs = [("fp64", "recipe", -1, p64), ("bf16x6", "auto", -1, p32),
                ("bf16x6", "fused_gemm", 3, p32)]
        if K <= 32:
            runs += [("fp64", "ger", -1, p64), ("fp32", "ger", -1, p32)]
        for math, mapping, tile, p in runs:
            dt = "f64" if p.A.data.dtype == np.float64 else "f32"
            plan = Contraction((p.A.labels, p.A.extents, p.A.strides),
                               (p.B.labels, p.B.extents, p.B.strides),
                               (p.C.labels, p.C.extents, p.C.strides), dt, math, mapping, tile)
            A = torch.from_numpy(p.A.data).to(dev)
            B = torch.from_numpy(p.B.data).to(dev)
            C = torch.zeros(p.C.data.size, dtype=A.dtype, device=dev)
            ws = plan.workspace(dev)
            call = lambda: tc.tc_contract(plan.handle, 1.0, A.data_ptr(), B.data_ptr(), 0.0,
                                          C.data_ptr(), ws.data_ptr() if ws is not None else 0,
                                          ws.numel() if ws is not None else 0, s.cuda_stream)
            times = []
            with torch.cuda.stream(s):
                for _ in range(args.warmup):
                    call()
                for _ in range(args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    call()
                    e1.record(s)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
            ms = float(np.median(times))
            info = plan.info
            err = sampled_error(p, C.cpu().numpy().astype(np.float64))
            parts.append({"shape": p.name, "free": free, "occ": occ, "M": int(info.M),
                          "N": int(info.N), "K": int(info.K), "math": math,
                          "mapping_asked": mapping, "mapping": tc.MAPPING_NAME[info.mapping],
                          "kernel": tc.KERNEL_NAME[info.kernel], "tile": int(info.tile), "ms": ms,
                          "tflops": p.flops() / (ms / 1e3) / 1e12,
                          "rel_err_vs_fp64_oracle_sampled": err})
            del A, B, C, ws, plan
            torch.cuda.empty_cache()
    clk = clocks.stop()
    tc.tc_selector_unload()
    status = tc.tc_device_status(s.cuda_stream)
    best64 = {}
    for q in parts:
        if q["math"] == "fp64":
            best64[q["shape"]] = min(best64.get(q["shape"], 1e30), q["ms"])
    total64 = sum(best64.values())
    best32 = {}
    for q in parts:
        if q["math"] != "fp64":
            best32[q["shape"]] = min(best32.get(q["shape"], 1e30), q["ms"])
    line = {
        "metric": "skewed CCD/GR suite: ms per shape (FP64 recipe vs reduced-precision choices)",
        "value": sum(best32.values()), "unit": "ms (sum over shapes, fastest FP32-storage run)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 and f32 storage", "data": "synthetic (seeded uniform[-1,1))",
        "config": {"workload": "skewed: X[i,a,j,b] Y[i,c,j,d], a=c=d=free, b=8, i=j=occ, "
                               "(free, occ) in " + str(SKEWED),
                   "l2": "flushed between steps (256 MiB write, outside timing)"},
        "fp64_best_ms_sum": total64, "parts": parts, "clocks": clk,
        "device_status": tc.tc_status_string(status)}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--workload", default="class3_fp64",
                    choices=["class3_fp64", "precision", "batching", "skewed"])
    ap.add_argument("--items", type=int, default=512, help="batching: number of contractions")
    ap.add_argument("--no-separate", action="store_true",
                    help="batching: skip the comparison with one tc_contract call per item")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batching: the threshold route rule instead of tuned routes")
    ap.add_argument("--math", default="bf16x6",
                    choices=["bf16", "bf16x3", "bf16x6", "fp8", "fp32"],
                    help="math of the precision workload")
    ap.add_argument("--tile", type=int, default=-1)
    ap.add_argument("--mapping", default="auto",
                    choices=["auto", "recipe", "slice_gemm", "fused_gemm", "copy_gemm", "gemv",
                             "dot", "ger"],
                    help="mapping of every contraction of the step (profiling a kernel)")
    ap.add_argument("--gemv-b", type=int, default=1024,
                    help="extent b of the GEMV workload (1024: the full 17.2 GB matrix)")
    ap.add_argument("--precision-v", type=int, default=128,
                    help="precision workload: virtual extent a=b=e=f (128 is the named "
                         "configuration; smaller values are profiling cases)")
    ap.add_argument("--only", default="", help="comma-separated subset of the workload "
                    "(direct_gemm_64, fused_permute_48, gemv_1024), for profiling")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "skewed":
        return run_skewed(args)
    if args.workload == "batching":
        if args.math == "bf16x6" and "--math" not in (argv or sys.argv):
            args.math = "bf16x3"
        return run_batching(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
