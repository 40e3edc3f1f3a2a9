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


NPROD = {"bf16": 1, "bf16x3": 3, "bf16x6": 6, "fp16": 1}
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
def oracle_sample_problems(target_s: float, nthreads: int, fn=None):
    """Bounded samples of the three contractions for a CPU baseline (the
    oracle, or `fn`): the last free label of C is cut to s values, s chosen so
    each takes ~target_s."""
    import oracle
    if fn is None:
        fn = lambda q, nthreads: oracle.contract_problem(q, nthreads=nthreads)
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
        fn(q, nthreads)  # warm (library loads, thread pools)
        t0 = time.perf_counter()
        fn(q, nthreads)
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


# ------------------------------------------------------------ peak probes
PEAK_KINDS = ("dfma", "dmma", "ffma", "bf16", "bf16_n256", "fp8")


def measure_peaks(tc, stream, target_ms=25.0, reps=3):
    """Peak rates (TFLOP/s) of each arithmetic on this GPU, measured in this
    process by the library's probe kernels (tc_peak_probe): a calibration
    launch sizes each probe to about target_ms, then the best of `reps`
    event-timed launches."""
    import torch
    out = {}
    for name in PEAK_KINDS:
        kind = tc.PEAK[name]
        iters = 64
        for _ in range(4):  # calibrate the length
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tc.tc_peak_probe(kind, iters, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if ms >= 0.5 * target_ms:
                break
            iters = int(iters * min(64.0, max(2.0, target_ms / max(ms, 1e-3))))
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = tc.tc_peak_probe(kind, iters, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
        out[name] = best
    return out


# ------------------------------------------------- the paper's method on the CPU
def recipe_cpu(p, nthreads=None):
    """The paper's method on the host: the class recipe's slicing vectors
    (Sec. 3.2), each slice one host-BLAS call through torch's CPU matmul in
    FP64.  Sliced free indices become batch dimensions of one matmul (the loop
    over those slices runs inside torch), sliced contracted indices are a loop
    that accumulates into C (R2's beta = 1).  Non-unit-stride slices are
    copied by matmul before the BLAS call, as COPY+GEMM does.  Returns C's
    buffer (float64, C's layout)."""
    import itertools
    import torch
    from oracle import classify as ocl
    if nthreads:
        torch.set_num_threads(int(nthreads))
    A, B, C = p.A, p.B, p.C
    cl = ocl.classify(A, B, C)
    ext = {}
    for t in (A, B, C):
        for l, e in zip(t.labels, t.extents):
            ext[l] = int(e)
    con = [l for l in A.labels if l in B.labels]
    sl_a = {l for l, f in zip(A.labels, cl.slice_a) if f}
    sl_b = {l for l, f in zip(B.labels, cl.slice_b) if f}
    k_loop = [l for l in con if l in sl_a or l in sl_b]       # accumulated slices
    k_keep = [l for l in con if l not in k_loop]
    fa_bat = [l for l in A.labels if l not in con and l in sl_a]
    fb_bat = [l for l in B.labels if l not in con and l in sl_b]
    fa_mat = [l for l in A.labels if l not in con and l not in sl_a]
    fb_mat = [l for l in B.labels if l not in con and l not in sl_b]
    cbuf = np.zeros(max(C.data.size, 1), dtype=np.float64)
    if any(ext[l] == 0 for l in C.labels):
        return cbuf[: C.data.size]
    tA = torch.from_numpy(np.asarray(A.data, np.float64))
    tB = torch.from_numpy(np.asarray(B.data, np.float64))
    tC = torch.from_numpy(cbuf)

    def view(t, labels, strides, order, off):  # None: a broadcast dimension of size 1
        st = dict(zip(labels, strides))
        return torch.as_strided(t, [1 if l is None else ext[l] for l in order],
                                [0 if l is None else st[l] for l in order], off)

    def flat(x, groups):  # merge consecutive dims of each group into one
        shape, i = [], 0
        for g in groups:
            n = 1
            for _ in range(g):
                n *= x.shape[i]
                i += 1
            shape.append(n)
        return x.reshape(shape)

    c_order = fa_bat + fb_bat + fa_mat + fb_mat
    cv = view(tC, C.labels, C.strides, c_order, 0)
    for kv in itertools.product(*[range(ext[l]) for l in k_loop]):
        fix = dict(zip(k_loop, kv))
        oa = sum(fix[l] * s for l, s in zip(A.labels, A.strides) if l in fix)
        ob = sum(fix[l] * s for l, s in zip(B.labels, B.strides) if l in fix)
        av = view(tA, A.labels, A.strides, fa_bat + [None] * len(fb_bat) + fa_mat + k_keep, oa)
        bv = view(tB, B.labels, B.strides, [None] * len(fa_bat) + fb_bat + k_keep + fb_mat, ob)
        nb = len(fa_bat) + len(fb_bat)
        am = flat(av, [1] * nb + [len(fa_mat), len(k_keep)])
        bm = flat(bv, [1] * nb + [len(k_keep), len(fb_mat)])
        r = torch.matmul(am, bm)                     # one BLAS call per batch slice
        cv += r.reshape(cv.shape)
    out = cbuf[: C.data.size]
    if p.alpha != 1.0:
        out *= p.alpha
    return out


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


# ------------------------------------------------- parts of the default line
def _event_times(fn, stream, flush, n):
    """Event-timed runs of fn on `stream`, the L2 flushed before each (outside
    the events); returns the list of ms."""
    import torch
    out = []
    for _ in range(n):
        with torch.cuda.stream(stream):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def precision_part(peaks, steps, warmup, v=128):
    """The precision workload (the CCD-shaped C[a,b,i,j] = sum_{e,f}
    A[a,b,e,f] B[e,f,i,j] of Sec. 4.2, a=b=e=f=v, i=j=32) on the plain FP64
    path and in every reduced-precision form, on the same FP32-representable
    inputs: time (median, L2 flushed), effective TFLOP/s, roofline fraction and
    the sampled relative error against the FP64 oracle."""
    import torch
    from paper_1307_2100_gb300 import Contraction, tc
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = ts.precision_ccd(v=v)
    std = peaks_std()
    A32 = torch.from_numpy(p.A.data).to(dev)
    B32 = torch.from_numpy(p.B.data).to(dev)
    out = []
    for form in ("fp64", "bf16x6", "bf16x3", "bf16", "fp8"):
        f64 = form == "fp64"
        A, B = (A32.double(), B32.double()) if f64 else (A32, B32)
        C = torch.empty(p.C.data.size, dtype=A.dtype, device=dev)
        plan = Contraction((p.A.labels, p.A.extents, p.A.strides),
                           (p.B.labels, p.B.extents, p.B.strides),
                           (p.C.labels, p.C.extents, p.C.strides), "f64" if f64 else "f32",
                           form, "auto")
        ws = plan.workspace(dev)
        call = lambda: tc.tc_contract(plan.handle, 1.0, A.data_ptr(), B.data_ptr(), 0.0,
                                      C.data_ptr(), ws.data_ptr() if ws is not None else 0,
                                      ws.numel() if ws is not None else 0, stream.cuda_stream)
        nw, ns = (1, 2) if f64 else (warmup, steps)
        with torch.cuda.stream(stream):
            for _ in range(nw):
                call()
        ms = float(np.median(_event_times(call, stream, flush, ns)))
        info = plan.info
        flops = p.flops()
        bytes_ = p.min_bytes() * (2 if f64 else 1)
        if f64:
            cpeak, work, bound_c, src = peaks["fp64"], flops, "alu", peaks["fp64_source"]
        elif form == "fp8":
            cpeak, work, bound_c, src = peaks["fp8"], flops, "tensor", peaks["fp8_source"]
        else:
            cpeak, work, bound_c = std["bf16"], flops * NPROD[form], "tensor"
            src = f"bf16_tflops burst {std['bf16']} (MEASURED_PEAKS.json) x {NPROD[form]} products"
        t_c, t_m = work / (cpeak * 1e12), bytes_ / (std["hbm"] * 1e9)
        err = sampled_error(p, C.cpu().numpy().astype(np.float64))
        out.append({"form": form, "kernel": tc.KERNEL_NAME[info.kernel], "tile": int(info.tile),
                    "ms": ms, "tflops_effective": flops / (ms / 1e3) / 1e12,
                    "bound": bound_c if t_c >= t_m else "hbm",
                    "roofline_ms": 1e3 * max(t_c, t_m), "frac": 1e3 * max(t_c, t_m) / ms,
                    "peak_source": src if t_c >= t_m else f"hbm_gbs {std['hbm']} GB/s",
                    "rel_err_vs_fp64_oracle_sampled": err, "samples": 64,
                    "gpu_launches": launches_of(info)})
        del C, ws, plan, A, B
        torch.cuda.empty_cache()
    base = out[0]["ms"]
    for q in out:
        q["speedup_vs_plain_fp64"] = base / q["ms"]
    fp32c = [q for q in out[1:] if q["rel_err_vs_fp64_oracle_sampled"] <= 1e-6]
    best = min(fp32c, key=lambda q: q["ms"]) if fp32c else None
    return {"workload": f"precision: C[a,b,i,j] = sum_ef A[a,b,e,f] B[e,f,i,j], a=b=e=f={v}, "
                        "i=j=32; A = N(0,1)/(1+|a-e|), B = N(0,1); FP32 values (FP64 storage "
                        "for the plain path)",
            "l2": "flushed before each timed run", "forms": out,
            "fastest_fp32_class": None if best is None else {
                "form": best["form"], "ms": best["ms"],
                "speedup_vs_plain_fp64": best["speedup_vs_plain_fp64"],
                "rel_err": best["rel_err_vs_fp64_oracle_sampled"], "bound": 1e-6}}


def config1_part(peaks, steps):
    """Config 1, C[a,b,c] = sum_i A[a,i,c] B[i,b] with every extent 48 (case
    (iii) of Eq. tenscases), FP64: 1.8 MB of operands, launch-latency bound.
    Timed by CUDA-graph replay of one tc_contract: back to back with the
    operands in L2, and one replay at a time with the L2 flushed; also as a
    plain launch.  The oracle on the host: one thread and every core."""
    import torch
    import oracle
    from paper_1307_2100_gb300 import Contraction, tc
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    p = ts.slice_gemm_48()
    plan = Contraction((p.A.labels, p.A.extents, p.A.strides),
                       (p.B.labels, p.B.extents, p.B.strides),
                       (p.C.labels, p.C.extents, p.C.strides), "f64", "fp64", "auto")
    A = torch.from_numpy(p.A.data).to(dev)
    B = torch.from_numpy(p.B.data).to(dev)
    C = torch.empty(p.C.data.size, dtype=torch.float64, device=dev)
    ws = plan.workspace(dev)
    call = lambda: tc.tc_contract(plan.handle, 1.0, A.data_ptr(), B.data_ptr(), 0.0,
                                  C.data_ptr(), ws.data_ptr() if ws is not None else 0,
                                  ws.numel() if ws is not None else 0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        for _ in range(5):
            call()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        call()
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize()
    nrep = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(nrep):
            g.replay()
        e1.record(stream)
    e1.synchronize()
    warm_ms = e0.elapsed_time(e1) / nrep
    cold_ms = float(np.median(_event_times(g.replay, stream, flush, max(steps, 10))))
    plain_ms = float(np.median(_event_times(call, stream, flush, max(steps, 10))))
    torch.cuda.synchronize()
    ref = oracle.contract_problem(p)
    err = oracle.rel_fro(C.cpu().numpy(), ref)
    info = plan.info
    flops = p.flops()
    t_c = flops / (peaks["fp64"] * 1e12)
    t_m = p.min_bytes() / (peaks_std()["hbm"] * 1e9)
    t1 = time.perf_counter()
    oracle.contract_problem(p, nthreads=1)
    cpu1 = time.perf_counter() - t1
    nth = cores()
    t1 = time.perf_counter()
    oracle.contract_problem(p, nthreads=nth)
    cpun = time.perf_counter() - t1
    del g
    return {"workload": "config 1: C[a,b,c] = sum_i A[a,i,c] B[i,b], all extents 48, FP64, "
                        "uniform[-1,1)",
            "class": int(info.cls), "mapping": tc.MAPPING_NAME[info.mapping],
            "kernel": tc.KERNEL_NAME[info.kernel],
            "graph_replay_l2_warm_us": 1e3 * warm_ms, "graph_replay_l2_flushed_us": 1e3 * cold_ms,
            "plain_launch_l2_flushed_us": 1e3 * plain_ms,
            "tflops_graph_l2_warm": flops / (warm_ms / 1e3) / 1e12,
            "tflops_graph_l2_flushed": flops / (cold_ms / 1e3) / 1e12,
            "roofline": {"bound": "alu" if t_c >= t_m else "hbm",
                         "roofline_us": 1e6 * max(t_c, t_m),
                         "frac_graph_l2_flushed": 1e3 * max(t_c, t_m) / cold_ms,
                         "peak_source": peaks["fp64_source"]},
            "rel_err_vs_fp64_oracle": err,
            "cpu_oracle": {"one_thread_s": cpu1, "all_cores_s": cpun, "cores": nth,
                           "one_thread_tflops": flops / cpu1 / 1e12,
                           "all_cores_tflops": flops / cpun / 1e12, "kind": "oracle",
                           "sample": "the whole config"}}


SELECTORS = [  # (kind, weights, timing table, held-out descriptors re-timed)
    ("bf16x6", "selector_gb300.bin", "selector_timings_gb300.npz", 160),
    ("fp64", "selector_gb300_fp64.bin", "selector_timings_gb300_fp64.npz", 80),
]


def selector_part(budget_s=90.0, reps=3):
    """The learned selectors re-timed on this GPU: for each kind (FP32 storage
    with BF16x6; FP64), held-out descriptors of the selector workload (orders
    2-6, extents log-uniform [4, 256], random label placement and strides; the
    network never saw them), each timed under every candidate mapping and tile
    (exhaustive timing, median of `reps` runs), and the regret t(choice) /
    t(best) - 1 of the network's choice (tc_plan with TC_MAP_AUTO, packaged
    weights) and of the paper's recipe.  Stops at `budget_s` seconds."""
    import torch
    from paper_1307_2100_gb300 import selector as sel
    from paper_1307_2100_gb300 import tc
    data = os.path.join(ROOT, "paper_1307_2100_gb300", "data")
    out = {"timing": f"median of {reps} event-timed runs per candidate, live on this GPU"}
    t0 = time.perf_counter()
    for kind, wfile, tfile, n_desc in SELECTORS:
        if not os.path.exists(os.path.join(data, wfile)):
            out[kind] = {"error": "no packaged weights"}
            continue
        z = np.load(os.path.join(data, tfile))
        seed, n_all = int(z["seed"]), len(z["F"])
        descs = sel.descriptors(kind, n_all, seed)
        _, te = sel.split(n_all, 2000)
        k = sel.KINDS[kind]
        ensure, time_plan, s = sel._timer(1 << 31, k["dtype"])
        ensure(max(max(sel._span(t) for t in descs[i]) for i in te[:n_desc]))
        spec = {(tc.MAPPING[m], t): j for j, (_, m, t) in enumerate(sel.specs(kind))}

        def planned(A, B, C, mapping):
            h = tc.tc_plan(sel._desc(A), sel._desc(B), sel._desc(C), k["dtype"],
                           tc.MATH[k["math"]], tc.MAPPING[mapping])
            try:
                info = tc.tc_plan_get_info(h)
            finally:
                tc.tc_plan_destroy(h)
            m, t = int(info.mapping), int(info.tile)
            return spec.get((m, t), spec.get((m, -1), 0))

        tc.tc_selector_load(os.path.join(data, wfile))
        rn, rr, rows = [], [], 0
        tk = time.perf_counter()
        try:
            for i in te[:n_desc]:
                if time.perf_counter() - t0 > budget_s:
                    break
                A, B, C = descs[i]
                T = [sel._time_candidates(descs[i], j, time_plan, reps, kind)
                     for j in range(len(sel.specs(kind)))]
                ok = [t for t in T if t is not None]
                if not ok:
                    continue
                best = min(ok)
                cn, cr = planned(A, B, C, "auto"), planned(A, B, C, "recipe")
                if T[cn] is None or T[cr] is None:
                    continue
                rn.append(T[cn] / best - 1.0)
                rr.append(T[cr] / best - 1.0)
                rows += 1
        finally:
            tc.tc_selector_unload()
        torch.cuda.synchronize()
        stat = lambda r: {"mean": float(np.mean(r)), "median": float(np.median(r)),
                          "p90": float(np.percentile(r, 90))} if r else None
        out[kind] = {"workload": "held-out selector descriptors (orders 2-6, extents "
                                 "log-uniform [4,256], random placement and strides), "
                                 f"{'FP64' if kind == 'fp64' else 'FP32 storage, BF16x6'}",
                     "descriptors_timed": rows, "candidates": len(sel.specs(kind)),
                     "regret_network": stat(rn), "regret_recipe": stat(rr),
                     "seconds": time.perf_counter() - tk}
    return out


def peaks_std():
    """Measured copy bandwidth and cuBLAS BF16 rate (MEASURED_PEAKS.json)."""
    pk = read_peaks()
    return {"hbm": pk.get("hbm_gbs", 6784.5), "bf16": pk.get("bf16_tflops", 1884.0),
            "sm_max_mhz": pk.get("sm_max_mhz", 2070.0)}


def roofline_peaks(measured, clk):
    """Peaks the roofline fractions use.  FP64: the larger of the in-run DFMA
    probe and the nominal rate at the maximum SM clock (152 SMs x 4 FP64
    flop/clk); FP8: the in-run block-scaled probe."""
    std = peaks_std()
    smax = (clk or {}).get("sm_max_mhz") or std["sm_max_mhz"]
    nominal = N_SMS * FP64_FLOP_PER_CLK_SM * smax * 1e6 / 1e12
    fp64 = max(measured.get("dfma", 0.0), nominal)
    return {"fp64": fp64, "fp8": measured.get("fp8") or std["bf16"] * FP8_PER_BF16,
            "fp64_source": (f"max(in-run DFMA probe {measured.get('dfma', 0.0):.4f}, "
                            f"152 SMs x 4 flop/clk x max SM clock {smax:.0f} MHz = "
                            f"{nominal:.4f}) TFLOP/s"),
            "fp8_source": (f"in-run tcgen05 kind::mxf8f6f4 probe {measured['fp8']:.1f} TFLOP/s"
                           if measured.get("fp8") else "2 x bf16_tflops (nominal ratio)")}


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

    measured = {} if args.no_peaks else measure_peaks(tc, stream)
    rp = roofline_peaks(measured, clk)
    hbm = peaks_std()["hbm"]
    fp64_peak = rp["fp64"]  # TFLOP/s
    bf16_peak = peaks_std()["bf16"]
    parts = []
    for j, p in enumerate(probs):
        info = plans[j].info
        kms = float(per[:, j].mean())
        if info.kernel == 5:  # FP8 form: one E4M3 product per multiply-add
            cpeak, work, cbound = rp["fp8"], p.flops(), "tensor"
        elif fp64 or info.kernel != 2:
            cpeak, work, cbound = (fp64_peak if fp64 else measured.get("ffma", 77.7),
                                   p.flops(), "alu")
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
                     "peak_source": (rp["fp64_source"] if dom["bound"] == "alu" and fp64
                                     else rp["fp8_source"] + "; achieved = FLOPs over the "
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
        rprobs = oracle_sample_problems(3.0, nth, fn=recipe_cpu)
        t0 = time.perf_counter()
        for q in rprobs:
            recipe_cpu(q, nth)
        t = time.perf_counter() - t0
        line["cpu_baseline_recipe"] = {
            "value": sum(q.flops() for q in rprobs) / t / 1e12, "unit": "TFLOP/s", "cores": nth,
            "kind": "the paper's method: class recipe slicing (Sec. 3.2) over host BLAS "
                    "(torch CPU FP64 matmul, sliced free indices as batch dimensions)",
            "sample": sample_desc(rprobs), "seconds": t}
    if world == 1 and fp64 and not args.headline_only:
        line["peaks_measured"] = dict(measured, unit="TFLOP/s", how=(
            "tc_peak_probe kernels in this process: DFMA/FFMA chains, DMMA m8n8k4, tcgen05 "
            "kind::f16 128x128x16 and 128x256x16, kind::mxf8f6f4 128x128x32 from shared "
            "memory; best of 3 event-timed launches of ~25 ms"))
        legs = [("precision", lambda: precision_part(rp, args.steps, args.warmup)),
                ("config1", lambda: config1_part(rp, args.steps))]
        items = ts.batching_items(512)
        refs = {}

        def batch_leg(m):
            r, refs["r"] = batch_measure(items, m, args.steps, args.warmup, refs=refs.get("r"),
                                         clock=False)
            return r
        legs += [("batching_bf16x6", lambda: batch_leg("bf16x6")),
                 ("batching_bf16x3", lambda: batch_leg("bf16x3")),
                 ("selector", lambda: selector_part())]
        extra = ClockSampler(local_rank)
        extra.start()
        for key, fn in legs:
            t0 = time.perf_counter()
            try:
                line[key] = fn()
            except Exception as e:  # a failing leg is reported, the line still prints
                line[key] = {"error": repr(e)}
            line[key]["leg_seconds"] = time.perf_counter() - t0
        line["clocks_parts"] = extra.stop()
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_measure(items, math, steps, warmup, autotune=True, separate=True, refs=None,
                  clock=True):
    """The batched workload in one form: a batch of `items` planned with
    autotuned routes (or the threshold rule), one CUDA graph of
    tc_contract_batched timed by events (L2 flushed before each replay),
    against one tc_contract call per item, every item checked against the
    FP64 oracle (`refs`: the oracle's outputs, computed here if None).
    Returns (result dict, refs)."""
    import torch
    import oracle
    from paper_1307_2100_gb300 import Contraction, tc
    dev = torch.device("cuda", 0)
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
    if not autotune:
        batch = tc.tc_batch_plan(handles)
    else:  # routes per size bucket, chosen by timing (outside the timed region)
        from paper_1307_2100_gb300 import autotune as at
        routes, tuned = at.tune_routes(handles, (pa, pb, pc, al, be), s)
        batch = tc.tc_batch_plan_routes(handles, routes)
    info = tc.tc_batch_get_info(batch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ws = [pl.workspace(dev) for pl in plans]

    def batched():
        tc.tc_contract_batched(batch, pa.data_ptr(), pb.data_ptr(), pc.data_ptr(), al.data_ptr(),
                               be.data_ptr(), s.cuda_stream)

    def separate_calls():
        for j, pl in enumerate(plans):
            w = ws[j]
            tc.tc_contract(pl.handle, 1.0, bufs[j][0].data_ptr(), bufs[j][1].data_ptr(), 0.0,
                           bufs[j][2].data_ptr(), w.data_ptr() if w is not None else 0,
                           w.numel() if w is not None else 0, s.cuda_stream)

    with torch.cuda.stream(s):
        for _ in range(warmup):
            batched()
        if separate:
            separate_calls()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batched()

    def timed(fn, n, label):
        ts_ = []
        for _ in range(n):
            with torch.cuda.stream(s):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.nvtx.range_push(label)   # marks the timed launches for profilers
                e0.record(s)
                fn()
                e1.record(s)
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            ts_.append(e0.elapsed_time(e1))
        return float(np.median(ts_))

    clocks = ClockSampler(0) if clock else None
    if clocks:
        clocks.start()
    for _ in range(warmup):
        g.replay()
    t_graph = timed(g.replay, steps, "batched")
    t_sep = timed(separate_calls, max(1, min(steps, 2)), "separate") if separate else None
    clk = clocks.stop() if clocks else None
    status = tc.tc_device_status(s.cuda_stream)
    g.replay()
    torch.cuda.synchronize()
    if refs is None:
        refs = [oracle.contract_problem(p, nthreads=cores()) for p in items]
    errs = []
    for p, b, ref in zip(items, bufs, refs):
        got = b[2].cpu().numpy().astype(np.float64)[: p.C.data.size]
        errs.append(oracle.rel_fro(got, ref))
    del g
    tc.tc_batch_destroy(batch)
    peaks = read_peaks()
    hbm = peaks.get("hbm_gbs", 6784.5)
    bf16_peak = peaks.get("bf16_tflops", 1884.0)
    flops = info.flops
    t_tc = flops * NPROD[math] / (bf16_peak * 1e12)
    t_mem = info.min_bytes / (hbm * 1e9)
    roof_ms = 1e3 * max(t_tc, t_mem)
    res = {
        "math": math, "items": len(items), "ms": t_graph,
        "tflops_effective": flops / (t_graph / 1e3) / 1e12,
        "roofline": {"bound": "hbm" if t_mem > t_tc else "tensor", "roofline_ms": roof_ms,
                     "frac": roof_ms / t_graph,
                     "peaks": f"bf16 {bf16_peak} TFLOP/s x {NPROD[math]} products, "
                              f"HBM {hbm} GB/s (MEASURED_PEAKS.json)"},
        "separate_calls_ms": t_sep, "speedup_vs_separate": None if t_sep is None else t_sep / t_graph,
        "routes": {"tensor_core_items": info.n_tc_items, "cuda_core_items": info.n_simt_items,
                   "tc_tiles": info.n_tiles, "simt_work": info.n_simt_work,
                   "simt_tiles": info.n_simt_tiles, "tc_split_tiles": info.n_tc_split},
        "autotune": None if tuned is None else {
            "buckets": tuned["buckets"], "default_ms": tuned["default_ms"],
            "tuned_ms": tuned["tuned_ms"],
            "flipped": [t["bucket"] for t in tuned["trials"] if t["kept"]]},
        "rel_err_vs_fp64_oracle": {"max": float(np.max(errs)), "median": float(np.median(errs)),
                                   "items_checked": len(errs)},
        "sum_flops": flops, "sum_bytes": info.min_bytes, "clocks": clk,
        "device_status": tc.tc_status_string(status),
        "gpu_launches_per_step": (2 * int(info.n_tiles > 0) + int(info.n_tc_split > 0) +
                                  int(info.n_simt_work > 0) + int(info.n_simt_tiles > 0) +
                                  int(info.n_simt_work + info.n_simt_tiles > 0)),
        "launch": "one CUDA graph of tc_contract_batched; L2 flushed before each replay",
    }
    del plans, bufs, ws
    torch.cuda.empty_cache()
    return res, refs


def run_batching(args):
    """512 independent contractions (orders 2-5, extents log-uniform in
    [8, 192], 1-3 contracted indices, random storage orders, FP32) in one
    graph-captured tc_contract_batched, against 512 tc_contract calls."""
    import torch
    from paper_1307_2100_gb300 import build as _b
    _b.build()
    torch.cuda.set_device(0)
    items = ts.batching_items(args.items)
    r, _ = batch_measure(items, args.math, args.steps, args.warmup, not args.no_autotune,
                         not args.no_separate)
    line = {
        "metric": METRIC, "value": r["tflops_effective"], "unit": "TFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 storage, " + args.math,
        "data": "synthetic (seeded uniform[-1,1); shapes of the batched workload)",
        "config": {"workload": f"batching: {len(items)} contractions, orders 2-5, extents "
                               "log-uniform [8,192], 1-3 contracted, random storage orders",
                   "l2": "flushed between steps (256 MiB write, outside timing)",
                   "launch": "one CUDA graph of tc_contract_batched",
                   "routes": "threshold rule" if args.no_autotune else
                   "autotuned per size bucket (paper_1307_2100_gb300/autotune.py)"},
        "roofline": r["roofline"], "batch": r, "clocks": r["clocks"],
        "gpu_launches": args.steps * r["gpu_launches_per_step"],
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
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload: only the FP64 three-class step, without the "
                    "precision, config-1, batching and selector parts")
    ap.add_argument("--no-peaks", action="store_true", help="skip the in-run peak probes")
    ap.add_argument("--workload", default="class3_fp64",
                    choices=["class3_fp64", "precision", "batching", "skewed"])
    ap.add_argument("--items", type=int, default=512, help="batching: number of contractions")
    ap.add_argument("--no-separate", action="store_true",
                    help="batching: skip the comparison with one tc_contract call per item")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batching: the threshold route rule instead of tuned routes")
    ap.add_argument("--math", default="bf16x6",
                    choices=["bf16", "bf16x3", "bf16x6", "fp8", "fp16", "fp32"],
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
