"""Benchmark: split-precision fp64 tensor contraction on one B300.

Workload (one "step"): the particle-particle ladder contraction
    C[a,b,i,j] += sum_{c,d} V[a,b,c,d] T[c,d,i,j]      (v = 128, o = 32)
in fp64 storage, computed by the split-precision path (6 bf16 integer
slices per operand on the tensor cores, exact fp32 accumulation, fp64
recombination and beta update): exponent pass + pack + product + fix-up,
inputs resident in HBM.  The labels fuse to a 16384 x 1024 x 16384
GEMM-shaped contraction (5.50e11 algorithmic flops).  V alone (2.1 GB)
exceeds L2, so every step streams its inputs from HBM.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(test infrastructure, the reference arm here) on a bounded sample instead.
`--workload <name>` (or `all`) prints the secondary workloads instead, one
line each with its roofline, the oracle's time on a slice of it and the
error of sampled entries against the oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contraction TFLOP/s, % tensor-pipe peak; split-precision vs FP64 speedup"
# DRAM bytes (read + write) of one product-kernel launch of this benchmark
# (v=128, 1.154e13 executed flops) from an ncu capture of its dram byte
# counters; None whenever the product kernel has changed since the capture.
PRODUCT_TRAFFIC = {"bytes": 14593853696.0 + 1262723840.0, "exec_flops": 1.1544872091648e13}
V_EXT, O_EXT, SLICES = 128, 32, 6
WORKLOAD = f"ccsd_ladder_v128_o32_f64_split{SLICES}"


def set_size(v: int, o: int):
    """Smaller ladders for profiling captures (the default is the benchmark size)."""
    global V_EXT, O_EXT, WORKLOAD
    V_EXT, O_EXT = v, o
    if (v, o) != (128, 32):
        WORKLOAD = f"ccsd_ladder_v{v}_o{o}_f64_split{SLICES}"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("bf16_tflops", 1800.0), d.get("bf16_tflops_sustained", 1400.0), "measured"
    except OSError:
        return 1800.0, 1400.0, "fallback"


class Clocks:
    """Samples nvidia-smi every 25 ms around the timed region; the summary keeps
    the samples whose own timestamps fall between mark_start() and mark_end()
    (all samples if none do, and says so)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.rows, self.proc, self.gpu = [], None, gpu_index
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.06)  # let the sampler emit the samples taken up to now

    @staticmethod
    def _when(stamp):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(stamp, fmt).timestamp()
            except ValueError:
                pass
        return None

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        rows = [r for r in self.rows if len(r) >= 10]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = rows
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if (w := self._when(r[0])) is not None and self.t0 <= w <= self.t1]
        window = "timed region" if inside else "around the timed region"
        rows = inside or rows
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if num(r[3]) is not None]
        load = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        reasons = sorted({self.NAMES[i] for r in rows for i in range(4)
                          if r[6 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "window": window}


def dist_setup():
    import torch
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier_max(x: float, world: int) -> float:
    """Max of x over the ranks (after a barrier); x itself on one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(local_ms: float, flops_per_rank: float, world: int):
    """Whole-job (ms, TFLOP/s): every replica does the same work, the slowest
    rank's time counts."""
    ms = barrier_max(local_ms, world)
    return ms, world * flops_per_rank / (ms * 1e-3) / 1e12


def make_inputs():
    from paper_2604_07311_b300 import inputs as W
    return W.ladder(v=V_EXT, o=O_EXT)


def cpu_sample(p, cols: int):
    """Times the oracle on C[:, :, 0, 0:cols] of the same workload (all host cores)."""
    import oracle
    V = p.A.view()
    T = p.B.view()[:, :, :1, :cols]
    C = np.array(p.C.view()[:, :, :1, :cols], copy=True)
    t0 = time.perf_counter()
    oracle.contract(p.alpha, V, p.A.labels, T, p.B.labels, p.beta, C, p.C.labels)
    dt = time.perf_counter() - t0
    flops = 2.0 * V_EXT ** 4 * cols
    return flops, dt, oracle.default_threads()


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on a bounded sample."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    p = make_inputs()
    # size each step's sample so that the whole run stays near two minutes
    _, t1, _ = cpu_sample(p, 1)
    budget_s = 120.0
    cols = max(1, min(args.ref_cols, int(budget_s / max(t1, 1e-3) / (args.steps + args.warmup))))
    for _ in range(args.warmup):
        cpu_sample(p, cols)
    times, flops, cores = [], 0.0, 1
    for _ in range(args.steps):
        flops, dt, cores = cpu_sample(p, cols)
        times.append(dt)
    total = sum(times)
    value = flops * args.steps / total / 1e12
    sample = f"C[:, :, 0, 0:{cols}] of the v={V_EXT},o={O_EXT} ladder ({flops:.3g} flop per step)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "v": V_EXT, "o": O_EXT},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300._lib import KERNELS

    rank, world, local = dist_setup()
    p = make_inputs()
    flops = float(p.flops)
    dev = torch.device("cuda")

    def dev_operand(op):
        buf = torch.from_numpy(op.buf).to(dev)
        return torch.as_strided(buf, op.extents, op.strides)

    V, T, C0 = dev_operand(p.A), dev_operand(p.B), dev_operand(p.C)
    C = C0.clone()
    la, lb, lc = p.A.labels, p.B.labels, p.C.labels
    stream = torch.cuda.current_stream()

    def step(Cout, **kw):
        return fm.contract(p.alpha, V, la, T, lb, p.beta, Cout, lc, dtype="f64_emu", slices=SLICES,
                           return_info=True, **kw)

    _, info = step(C)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step(C)
    torch.cuda.synchronize()

    # ---- timed region: K steps on resident inputs
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk.mark_start()
        start.record(stream)
        for _ in range(args.steps):
            step(C)
        end.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
        if world > 1:
            torch.distributed.barrier()
    ms, value = replica_throughput(start.elapsed_time(end) / args.steps, flops, world)
    launches = info["launches"] * args.steps

    # ---- the product kernel alone (events recorded by the library around it)
    kev = []
    for _ in range(max(3, min(args.steps, 5))):
        b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        step(C, events=(b, e))
        kev.append((b, e))
    torch.cuda.synchronize()
    kms = statistics.mean(b.elapsed_time(e) for b, e in kev)
    pairs = SLICES * (SLICES + 1) // 2
    exec_flops = pairs * flops
    burst, sustained, src = peaks()
    achieved = exec_flops / (kms * 1e-3) / 1e12

    # ---- the same product on CTA pairs (cta_group::2), for comparison: step
    # and product times, and whether the result is bit-identical
    Cp, Cq = C0.clone(), C0.clone()
    step(Cp)
    _, pinfo = step(Cq, ctas_per_mma=2)
    torch.cuda.synchronize()
    pev = []
    for _ in range(max(3, min(args.steps, 5))):
        b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        step(C, events=(b, e), ctas_per_mma=2)
        s1.record(stream)
        pev.append((b, e, s0, s1))
    torch.cuda.synchronize()
    pair_cmp = {"ctas_per_mma": pinfo["ctas_per_mma"],
                "product_ms": statistics.mean(b.elapsed_time(e) for b, e, _, _ in pev),
                "step_ms": statistics.mean(s0.elapsed_time(s1) for _, _, s0, s1 in pev),
                "bit_identical": bool(torch.equal(Cp, Cq))}
    del Cp, Cq

    # ---- native fp64 on the GPU (the speedup denominator) and agreement
    Ce = C0.clone()
    step(Ce)
    torch.cuda.synchronize()
    # the error against the oracle: 4096 entries of the full result against
    # the oracle's compensated (Dot2) sums, outside the timed region
    err_oracle, err_note = sampled_error(p.alpha, p.A.view(), la, p.B.view(), lb, p.beta, p.C.view(), lc,
                                         host64(Ce), n=4096, seed=21, dot2=True)
    Cn = C0.clone()
    fm.contract(p.alpha, V, la, T, lb, p.beta, Cn, lc, dtype="f64")  # warm-up
    Cn.copy_(C0)
    b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.record(stream)
    fm.contract(p.alpha, V, la, T, lb, p.beta, Cn, lc, dtype="f64")
    e.record(stream)
    torch.cuda.synchronize()
    native_ms = b.elapsed_time(e)
    rel = float((Ce - Cn).norm() / Cn.norm())
    rel_ab = float((Ce - Cn).norm() / (Cn - p.beta * C0).norm())
    del Ce, Cn

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(p.A.buf).pin_memory()
        hT = torch.from_numpy(p.B.buf).pin_memory()
        hC = torch.from_numpy(p.C.buf).pin_memory()
        st = lambda h, op: np.lib.stride_tricks.as_strided(h.numpy(), op.extents,
                                                          tuple(8 * s for s in op.strides))
        Vn, Tn, Cn_h = st(hV, p.A), st(hT, p.B), st(hC, p.C)
        fm.contract_host(p.alpha, Vn, la, Tn, lb, p.beta, Cn_h, lc, dtype="f64_emu", slices=SLICES)
        e2e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fm.contract_host(p.alpha, Vn, la, Tn, lb, p.beta, Cn_h, lc, dtype="f64_emu",
                             slices=SLICES)
        e2e_s = barrier_max((time.perf_counter() - t0) / e2e_steps, world)
        e2e = {"value": world * flops / e2e_s / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * (p.A.span + p.B.span + p.C.span),
               "d2h_bytes_per_step": 8 * p.C.span, "host_memory": "pinned"}

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (bf16 slices, exact fp32 accumulate, fp64 recombine)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "v": V_EXT, "o": O_EXT, "m": info["m"], "n": info["n"],
                   "k": info["k"], "slices": SLICES, "beta": p.beta, "l2": "inputs larger than L2",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "speedup_vs_native_f64": native_ms / ms,
        "cta_pairs": pair_cmp,
        "native_f64": {"ms": native_ms, "tflops": flops / (native_ms * 1e-3) / 1e12},
        "rel_err_vs_oracle": err_oracle, "error_sample": err_note,
        "rel_err_vs_native_f64": rel, "rel_err_vs_native_f64_ab_term": rel_ab,
        "roofline": {"bound": "tensor", "kernel": "k_pair_gemm<bf16, fp64-split>",
                     "achieved": achieved, "peak": burst, "unit": "TFLOP/s",
                     "frac": achieved / burst,
                     "traffic": (PRODUCT_TRAFFIC["bytes"] * exec_flops / PRODUCT_TRAFFIC["exec_flops"]
                                 if PRODUCT_TRAFFIC else None),
                     "traffic_note": "ncu dram bytes of one launch of this workload (read + write)",
                     "peak_kind": (f"bf16 burst ({src}): the timed region is ~0.1 s and the SM "
                                   f"clock stays near its maximum, unlike the power-capped "
                                   f"seconds-long loop behind the sustained figure"),
                     "frac_of_sustained": achieved / sustained,
                     "kernel_ms": kms, "exec_flops_per_launch": exec_flops},
        "e2e": e2e,
        "gpu_launches": launches,
        "kernel_path": KERNELS.get(info["kernel"], "?"),
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        cflops, cdt, cores = cpu_sample(p, args.ref_cols)
        line["cpu_baseline"] = {"value": cflops / cdt / 1e12, "unit": "TFLOP/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"C[:, :, 0, 0:{args.ref_cols}] ({cflops:.3g} flop)"}
    status = fm.device_status()
    if status != 0:
        line["device_status"] = status
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _cuda_ms(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(steps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / steps


def _product_ms(fn, n=5):
    """Mean CUDA-event time of the main product kernel (events recorded by the library around it)."""
    import torch
    evs = []
    for _ in range(n):
        b, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn(events=(b, e))
        evs.append((b, e))
    torch.cuda.synchronize()
    return statistics.mean(b.elapsed_time(e) for b, e in evs)


# Nominal dense rates relative to bf16 (2.25 PFLOP/s): tf32 1.1 PFLOP/s.  The
# fp64 CUDA-core rate has no measured figure here: 1.25 TFLOP/s nominal.
TF32_OVER_BF16 = 1.1 / 2.25
FP64_NOMINAL_TFLOPS = 1.25


def roofline(kind, exec_flops, kernel_ms, kernel, note=None):
    """roofline object of one kernel: executed flops per launch / its CUDA-event time
    against the dtype's peak (bf16 measured burst; tf32 from it by the nominal ratio;
    fp64 CUDA cores nominal)."""
    burst, _, src = peaks()
    if kind == "bf16":
        peak, bound, pk = burst, "tensor", f"bf16 burst ({src})"
    elif kind == "tf32":
        peak, bound, pk = burst * TF32_OVER_BF16, "tensor", f"tf32 = bf16 burst ({src}) x nominal 1.1/2.25"
    else:
        peak, bound, pk = FP64_NOMINAL_TFLOPS, "alu", "fp64 CUDA cores, nominal 1.25 TFLOP/s"
    achieved = exec_flops / (kernel_ms * 1e-3) / 1e12
    r = {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
         "frac": achieved / peak, "traffic": None, "peak_kind": pk, "kernel_ms": kernel_ms,
         "exec_flops_per_launch": exec_flops}
    if note:
        r["note"] = note
    return r


def host64(t):
    """A device tensor's values (exactly, promoted to fp64) as a numpy array with the same strides."""
    import torch
    base = t.detach()
    flat = torch.as_strided(base, (base.untyped_storage().nbytes() // base.element_size(),), (1,), 0)
    buf = flat.to(torch.float64).cpu().numpy()
    return np.lib.stride_tricks.as_strided(buf[base.storage_offset():], tuple(base.shape),
                                           tuple(8 * x for x in base.stride()))


def sampled_error(alpha, A, la, B, lb, beta, C0, lc, got, n=512, seed=11, dot2=True):
    """Relative Frobenius error of n sampled result entries against the oracle
    (compensated Dot2 sums, or plain fp64 sums) on the inputs as the device held them."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.integers(0, e, n) for e in C0.shape], axis=1)
    want = oracle.entries(alpha, A, la, B, lb, beta, C0, lc, idx, dot2=dot2)
    g = np.asarray(got)[tuple(idx.T)]
    den = np.linalg.norm(want)
    return float(np.linalg.norm(g - want) / den) if den > 0 else float(np.linalg.norm(g)), \
        f"{n} sampled entries vs the oracle's {'Dot2' if dot2 else 'fp64'} sums"


def cpu_slice(alpha, A, la, B, lb, beta, C0, lc, budget_s=3.0):
    """cpu_baseline: the oracle (all host cores) on C restricted along its largest
    mode to a slice sized for about budget_s seconds."""
    import oracle
    lab = lc[int(np.argmax(C0.shape))]

    def cut(x, labels, s):
        if lab not in labels:
            return x
        i = list(labels).index(lab)
        return x[(slice(None),) * i + (slice(0, s),)]

    def run(s):
        Cs = np.array(cut(C0, lc, s), copy=True)
        As, Bs = cut(A, la, s), cut(B, lb, s)
        ext = {}
        for x, ls in ((As, la), (Bs, lb), (Cs, lc)):
            ext.update(zip(ls, x.shape))
        t0 = time.perf_counter()
        oracle.contract(alpha, As, la, Bs, lb, beta, Cs, lc)
        return time.perf_counter() - t0, 2.0 * float(np.prod(list(ext.values())))
    full = C0.shape[list(lc).index(lab)]
    dt, fl = run(1)
    s = max(1, min(full, int(budget_s / max(dt, 1e-4))))
    if s > 1:
        dt, fl = run(s)
    import oracle as _o
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": _o.default_threads(), "kind": "oracle",
            "sample": f"C restricted to {s} of {full} along label {lab} ({fl:.3g} flop)"}


def emit(workload, flops, ms, roof, cpu, err, err_note, **extra):
    line = {"workload": workload, "metric": "contraction TFLOP/s", "value": flops / (ms * 1e-3) / 1e12,
            "unit": "TFLOP/s", "ms_per_step": ms, "flops_per_step": flops, "roofline": roof,
            "cpu_baseline": cpu, "rel_err_vs_oracle": err, "error_sample": err_note, **extra}
    print(json.dumps(line), flush=True)


def _put(op, dt):
    import torch
    buf = torch.from_numpy(op.buf).to(device="cuda", dtype=dt)
    return torch.as_strided(buf, op.extents, op.strides)


def wl_four_index(args):
    """C1: C[a,b,i,j] = sum_{c,k} A[a,c,i,k] B[c,k,b,j], extents 16, fp64."""
    import torch
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300 import inputs as W
    p = W.four_index(ext=16)
    A, B = _put(p.A, torch.float64), _put(p.B, torch.float64)
    for dt, kind, kname, pairs in (("f64", "fp64", "k_simt<double>", 1),
                                   ("f64_emu", "bf16", "k_pair_gemm<bf16, fp64-split>", 21)):
        C = _put(p.C, torch.float64)
        f = lambda **kw: fm.contract(p.alpha, A, p.A.labels, B, p.B.labels, p.beta, C, p.C.labels, dtype=dt, **kw)
        ms = _cuda_ms(f, args.steps, args.warmup)
        kms = _product_ms(f)
        C.copy_(_put(p.C, torch.float64))
        f()
        torch.cuda.synchronize()
        err, note = sampled_error(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(),
                                  p.C.labels, host64(C), n=4096)
        emit("four_index_ext16_" + dt, p.flops, ms, roofline(kind, pairs * p.flops, kms, kname),
             cpu_slice(p.alpha, p.A.view(), p.A.labels, p.B.view(), p.B.labels, p.beta, p.C.view(), p.C.labels, 1.0),
             err, note, dtype=dt, note="launch-latency-sized problem (3.4e7 flop)")


def wl_transpose_free(args):
    """C3: C[b,j,a,i] = sum_{c,k} A[a,c,i,k] B[b,k,j,c], v=96, o=48, A's first mode padded by 7."""
    import torch
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300 import inputs as W
    p = W.transpose_free(v=96, o=48, pad=7)
    cpu = None
    for dt, kernel, path, kind, pairs, kname in (
            ("bf16", 0, "direct (default)", "bf16", 1, "k_box<bf16>"),
            ("bf16", 2, "packed", "bf16", 1, "k_pair_gemm<bf16>"),
            ("f32", 0, "packed tf32x3 (default)", "tf32", 3, "k_pair_gemm<tf32x3>"),
            ("f32", 1, "cuda_cores", "fp32", 1, "k_simt<float>")):
        tin = torch.bfloat16 if dt == "bf16" else torch.float32
        A, B, C = _put(p.A, tin), _put(p.B, tin), _put(p.C, torch.float32)
        f = lambda **kw: fm.contract(1.0, A, p.A.labels, B, p.B.labels, 0.0, C, p.C.labels, dtype=dt,
                                     kernel=kernel, **kw)
        ms = _cuda_ms(f, args.steps, args.warmup)
        kms = _product_ms(f)
        _, info = fm.contract(1.0, A, p.A.labels, B, p.B.labels, 0.0, C, p.C.labels, dtype=dt, kernel=kernel,
                              return_info=True)
        torch.cuda.synchronize()
        Ah, Bh = host64(A), host64(B)
        err, note = sampled_error(1.0, Ah, p.A.labels, Bh, p.B.labels, 0.0, np.zeros(p.C.extents), p.C.labels,
                                  host64(C), n=512, dot2=False)
        if cpu is None:
            cpu = cpu_slice(1.0, Ah, p.A.labels, Bh, p.B.labels, 0.0, np.zeros(p.C.extents), p.C.labels, 3.0)
        roof = (roofline(kind, pairs * p.flops, kms, kname) if kind != "fp32" else
                {"bound": "alu", "kernel": kname, "achieved": p.flops / (kms * 1e-3) / 1e12, "peak": None,
                 "unit": "TFLOP/s", "frac": None, "traffic": None, "kernel_ms": kms,
                 "note": "fp32 CUDA cores: reference point, no fp32 peak stated"})
        emit("transpose_free_v96_o48_pad7", p.flops, ms, roof, cpu, err, note, dtype=dt, path=path,
             launches=info["launches"], kernel_path=info["kernel_name"])


def wl_block_sparse(args):
    """C4: 2000 independent four-index blocks, each extent from {8,...,96} (and a
    small-block variant, extents 8..32), emulated fp64, grouped launch + graph vs
    one call per block; sampled entries of at least 50 blocks against Dot2."""
    import torch
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300 import inputs as W
    import oracle
    for nblocks, choices in ((2000, [8, 16, 24, 32]), (2000, None)):
        ext = W.block_sparse_extents(nblocks=nblocks, choices=choices)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        pooled = choices is None
        pool = torch.rand(1 << 28, device="cuda", dtype=torch.float64, generator=gen) if pooled else None
        offs = np.random.default_rng(W.SEED_BASE + 40).integers(0, (1 << 28) - 96 ** 4, size=(nblocks, 2))
        As, Bs, Cs, la, lb, lc, flops = [], [], [], [], [], [], 0
        for bi, (a, b, c, i, j, k) in enumerate(map(int, e) for e in ext):
            if pooled:
                As.append(torch.as_strided(pool, (a, c, i, k), W.colmajor_strides((a, c, i, k)), int(offs[bi, 0])))
                Bs.append(torch.as_strided(pool, (c, k, b, j), W.colmajor_strides((c, k, b, j)), int(offs[bi, 1])))
            else:
                As.append(torch.rand((k, i, c, a), device="cuda", dtype=torch.float64, generator=gen).permute(3, 2, 1, 0))
                Bs.append(torch.rand((j, b, k, c), device="cuda", dtype=torch.float64, generator=gen).permute(3, 2, 1, 0))
            Cs.append(torch.zeros((j, i, b, a), device="cuda", dtype=torch.float64).permute(3, 2, 1, 0))
            la.append(W.L("acik")); lb.append(W.L("ckbj")); lc.append(W.L("abij"))
            flops += 2 * a * b * c * i * j * k
        res = {}
        for name, graph in (("grouped_graph", True), ("grouped_nograph", False)):
            f = lambda: fm.contract_batched(1.0, As, la, Bs, lb, 0.0, Cs, lc, dtype="f64_emu", use_graph=graph)
            ms = _cuda_ms(f, max(1, min(args.steps, 3)), 1)
            res[name] = {"ms": ms, "tflops": flops / ms / 1e9}

        def loop():
            for x in zip(As, la, Bs, lb, Cs, lc):
                fm.contract(1.0, x[0], x[1], x[2], x[3], 0.0, x[4], x[5], dtype="f64_emu")
        if args.no_per_block:  # profiling captures: the grouped calls' launches only
            ms_loop = None
        else:
            ms_loop = _cuda_ms(loop, max(1, min(args.steps, 3)), 1)
            res["one_call_per_block"] = {"ms": ms_loop, "tflops": flops / ms_loop / 1e9}
        # accuracy: the grouped result of 64 blocks (the largest one included), 32 entries each
        for c in Cs:
            c.zero_()
        fm.contract_batched(1.0, As, la, Bs, lb, 0.0, Cs, lc, dtype="f64_emu", use_graph=True)
        torch.cuda.synchronize()
        sizes = np.array([float(np.prod(e)) for e in ext])
        pick = sorted(set([int(np.argmax(sizes))] + list(np.random.default_rng(12).choice(nblocks, 63, replace=False))))
        pool_h = pool.cpu().numpy() if pooled else None
        num = den = 0.0
        t_or, fl_or = 0.0, 0.0
        rng = np.random.default_rng(13)
        for bi in pick:
            if pooled:
                Ah = np.lib.stride_tricks.as_strided(pool_h[int(offs[bi, 0]):], As[bi].shape,
                                                     tuple(8 * x for x in As[bi].stride()))
                Bh = np.lib.stride_tricks.as_strided(pool_h[int(offs[bi, 1]):], Bs[bi].shape,
                                                     tuple(8 * x for x in Bs[bi].stride()))
            else:
                Ah, Bh = host64(As[bi]), host64(Bs[bi])
            got = host64(Cs[bi])
            idx = np.stack([rng.integers(0, e, 32) for e in got.shape], axis=1)
            z = np.zeros(got.shape)
            want = oracle.entries(1.0, Ah, la[bi], Bh, lb[bi], 0.0, z, lc[bi], idx, dot2=True)
            g = got[tuple(idx.T)]
            num += float(np.sum((g - want) ** 2))
            den += float(np.sum(want ** 2))
        err = (num / den) ** 0.5
        # cpu baseline: the oracle on a whole block of median size
        mid = int(np.argsort(sizes)[len(sizes) // 2])
        if pooled:
            Ah = np.lib.stride_tricks.as_strided(pool_h[int(offs[mid, 0]):], As[mid].shape,
                                                 tuple(8 * x for x in As[mid].stride()))
            Bh = np.lib.stride_tricks.as_strided(pool_h[int(offs[mid, 1]):], Bs[mid].shape,
                                                 tuple(8 * x for x in Bs[mid].stride()))
        else:
            Ah, Bh = host64(As[mid]), host64(Bs[mid])
        cpu = cpu_slice(1.0, Ah, la[mid], Bh, lb[mid], 0.0, np.zeros(tuple(Cs[mid].shape)), lc[mid], 3.0)
        best = res["grouped_graph"]["ms"]
        emit(f"block_sparse_{nblocks}_ext_{'8-32' if choices else '8-96_pooled_inputs'}_f64_split{SLICES}",
             flops, best, roofline("bf16", 21 * flops, best, "grouped k_pair_gemm<bf16, fp64-split> (+pack)",
                                   note="whole grouped call timed (product and packs), so a lower bound"),
             cpu, err, f"32 entries in each of {len(pick)} blocks (the largest included) vs Dot2",
             dtype="f64_emu", **res, speedup_grouped_vs_per_block=ms_loop / best if ms_loop else None)
        del As, Bs, Cs, pool, pool_h
        torch.cuda.empty_cache()


def wl_autograd(args):
    """C5: L = ||contract(A,B) - T||^2, C[i,j,l] = sum_{k,m} A[i,k,m,l] B[k,m,j], fp32,
    forward and both adjoints; gradients against the oracle's on sampled entries."""
    import torch
    import oracle
    from paper_2604_07311_b300 import inputs as W
    from paper_2604_07311_b300.autograd import contract_autograd
    d = W.autograd_problem()
    A = torch.from_numpy(d["A"].astype(np.float32)).cuda().requires_grad_()
    B = torch.from_numpy(d["B"].astype(np.float32)).cuda().requires_grad_()
    T = torch.from_numpy(d["T"].astype(np.float32)).cuda()

    def fb():
        A.grad = B.grad = None
        ((contract_autograd(A, d["la"], B, d["lb"], d["lc"]) - T) ** 2).sum().backward()
    ms = _cuda_ms(fb, args.steps, args.warmup)
    fb()
    torch.cuda.synchronize()
    gA_eager, gB_eager = A.grad.clone(), B.grad.clone()
    # the same training step captured once into a CUDA graph (every library
    # call is stream-ordered, workspace included) and replayed
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            fb()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    A.grad = B.grad = None
    with torch.cuda.graph(graph):
        ((contract_autograd(A, d["la"], B, d["lb"], d["lc"]) - T) ** 2).sum().backward()
    ms_graph = _cuda_ms(graph.replay, args.steps, args.warmup)
    graph.replay()
    torch.cuda.synchronize()
    graph_matches_eager = bool(torch.equal(A.grad, gA_eager) and torch.equal(B.grad, gB_eager))
    Ah = A.detach().double().cpu().numpy()
    Bh = B.detach().double().cpu().numpy()
    Th = T.double().cpu().numpy()
    Ch = np.zeros(Th.shape)
    t0 = time.perf_counter()
    oracle.contract(1.0, Ah, d["la"], Bh, d["lb"], 0.0, Ch, d["lc"])
    cdt = time.perf_counter() - t0
    dC = 2.0 * (Ch - Th)
    gA, gB = A.grad.double().cpu().numpy(), B.grad.double().cpu().numpy()
    # dA[i,k,m,l] = sum_j dC[i,j,l] B[k,m,j];  dB[k,m,j] = sum_{i,l} A[i,k,m,l] dC[i,j,l]
    eA, _ = sampled_error(1.0, dC, d["lc"], Bh, d["lb"], 0.0, np.zeros(gA.shape), d["la"], gA, n=512, dot2=False)
    eB, _ = sampled_error(1.0, Ah, d["la"], dC, d["lc"], 0.0, np.zeros(gB.shape), d["lb"], gB, n=256, dot2=False)
    fl = 3 * 2 * 64 * 64 * 64 * 48 * 48
    import oracle as _o
    cpu = {"value": (fl / 3) / cdt / 1e12, "unit": "TFLOP/s", "cores": _o.default_threads(), "kind": "oracle",
           "sample": "the forward contraction (1.21e9 flop) in full"}
    emit("autograd_i64_k48_fwd_bwd_fp32", fl, ms,
         roofline("tf32", 3 * fl, ms, "forward + two adjoint contractions (tf32x3), whole step",
                  note="the whole training step is timed (host and loss ops included), so a lower bound"),
         cpu, max(eA, eB), "512 entries of dA and 256 of dB vs the oracle's gradient (fp64 sums)",
         dtype="f32", rel_err_dA=eA, rel_err_dB=eB, graph_step_ms=ms_graph,
         graph_step_tflops=fl / (ms_graph * 1e-3) / 1e12, graph_grads_equal_eager=graph_matches_eager)


def wl_network(args):
    """f1: the two-step network X = T.Y (kept on the device), R += V.X, emulated
    fp64, against two separate calls; sampled R entries against the oracle
    applied step by step."""
    import torch
    import oracle
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300 import inputs as W
    v, o = 96, 32
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    V = torch.randn(v, v, v, v, device="cuda", dtype=torch.float64, generator=gen) / 128
    T = torch.randn(v, v, o, o, device="cuda", dtype=torch.float64, generator=gen) * 1e-2
    Y = torch.randn(o, o, o, o, device="cuda", dtype=torch.float64, generator=gen)
    R = torch.zeros(v, v, o, o, device="cuda", dtype=torch.float64)
    X = torch.empty(v, v, o, o, device="cuda", dtype=torch.float64)
    lv, lt, ly, lx, lr = W.L("abcd"), W.L("cdkl"), W.L("klij"), W.L("cdij"), W.L("abij")
    # the library lays an intermediate out first mode fastest: listing X's
    # labels as (j, i, d, c) gives it the layout of the row-major tensor
    # X[c,d,i,j] of the separate calls (d fastest in V too, so the
    # contracted pair (c, d) fuses into one mode in both operands)
    net = [(V, lv), (T, lt), (Y, ly), ((o, o, v, v), W.L("jidc")), (R, lr)]
    steps = [(1, 2, 3, 1.0, 0.0), (0, 3, 4, 1.0, 1.0)]
    flops = 2 * v * v * o * o * o * o + 2 * v * v * v * v * o * o
    ms = _cuda_ms(lambda: fm.contract_network(net, steps, dtype="f64_emu"), args.steps, args.warmup)

    def separate():
        fm.contract(1.0, T, lt, Y, ly, 0.0, X, lx, dtype="f64_emu")
        fm.contract(1.0, V, lv, X, lx, 1.0, R, lr, dtype="f64_emu")
    ms_sep = _cuda_ms(separate, args.steps, args.warmup)
    R.zero_()
    fm.contract_network(net, steps, dtype="f64_emu")
    torch.cuda.synchronize()
    Vh, Th, Yh, Rh = host64(V), host64(T), host64(Y), host64(R)
    rng = np.random.default_rng(14)
    num = den = 0.0
    t_cpu, fl_cpu = 0.0, 0.0
    for _ in range(6):  # (i, j) pairs: X[:, :, i, j] by the oracle, then sampled R[a, b, i, j]
        i, j = (int(x) for x in rng.integers(0, o, 2))
        Xs = np.zeros((v, v, 1, 1))
        t0 = time.perf_counter()
        oracle.contract(1.0, Th, lt, Yh[:, :, i:i + 1, j:j + 1], ly, 0.0, Xs, lx)
        t_cpu += time.perf_counter() - t0
        fl_cpu += 2.0 * v * v * o * o
        ab = np.stack([rng.integers(0, v, 64), rng.integers(0, v, 64), np.zeros(64, int), np.zeros(64, int)], 1)
        want = oracle.entries(1.0, Vh, lv, Xs, lx, 0.0, np.zeros((v, v, 1, 1)), lr, ab, dot2=True)
        g = Rh[ab[:, 0], ab[:, 1], i, j]
        num += float(np.sum((g - want) ** 2))
        den += float(np.sum(want ** 2))
    import oracle as _o
    cpu = {"value": fl_cpu / t_cpu / 1e12, "unit": "TFLOP/s", "cores": _o.default_threads(), "kind": "oracle",
           "sample": f"the first step's X[:, :, i, j] for 6 (i, j) pairs ({fl_cpu:.3g} flop)"}
    emit("network_ladder_v96_o32_two_steps_f64_split6", flops, ms,
         roofline("bf16", 21 * flops, ms, "two k_pair_gemm<bf16, fp64-split> steps (+packs)",
                  note="whole network call timed, so a lower bound"),
         cpu, (num / den) ** 0.5, "64 entries of R in each of 6 (i, j) columns vs Dot2 on the oracle's X",
         dtype="f64_emu", separate_calls_ms=ms_sep, speedup_vs_separate=ms_sep / ms)


def wl_ladder_sym(args):
    """f2: the ladder with V read as its packed lower triangle, against the dense call."""
    import torch
    import paper_2604_07311_b300 as fm
    from paper_2604_07311_b300 import inputs as W
    v, o = V_EXT, O_EXT
    n = v * v
    gen = torch.Generator(device="cuda")
    gen.manual_seed(6)
    Vd = torch.randn(n, n, device="cuda", dtype=torch.float64, generator=gen) / 128
    Vd = torch.tril(Vd) + torch.tril(Vd, -1).T
    iu = torch.triu_indices(n, n, device="cuda")
    Vp = Vd[iu[0], iu[1]].contiguous()  # row q of the upper triangle = column q of the lower
    del iu
    Vd = Vd.reshape(v, v, v, v)  # row-major flattening of a symmetric matrix is column-major
    T = torch.randn(o, o, v, v, device="cuda", dtype=torch.float64, generator=gen).permute(3, 2, 1, 0) * 1e-2
    C0 = torch.rand(o, o, v, v, device="cuda", dtype=torch.float64, generator=gen).permute(3, 2, 1, 0)
    Cs, Cd = C0.clone(), C0.clone()
    lv, lt, lc = W.L("dcba"), W.L("cdij"), W.L("abij")  # Vd's torch order is (d, c, b, a)
    ext = (v, v, v, v)
    flops = 2 * v ** 4 * o * o
    f_sym = lambda **kw: fm.contract_sym(1.0, Vp, ext, W.L("abcd"), T, lt, 1.0, Cs, lc, **kw)
    f_den = lambda: fm.contract(1.0, Vd, lv, T, lt, 1.0, Cd, lc, dtype="f64_emu")
    ms_sym = _cuda_ms(f_sym, args.steps, args.warmup)
    kms = _product_ms(f_sym)
    ms_den = _cuda_ms(f_den, args.steps, args.warmup)
    Cs.copy_(C0)
    Cd.copy_(C0)
    f_sym()
    f_den()
    torch.cuda.synchronize()
    diff = float((Cs - Cd).abs().max())
    Vh, Th, C0h = host64(Vd), host64(T), host64(C0)
    err, note = sampled_error(1.0, Vh, lv, Th, lt, 1.0, C0h, lc, host64(Cs), n=1024)
    cpu = cpu_slice(1.0, Vh, lv, Th[:, :, :1, :], lt, 1.0, C0h[:, :, :1, :], lc, 3.0)
    emit(f"ladder_v{v}_o{o}_f64_split6_packed_symmetric_V", flops, ms_sym,
         roofline("bf16", 21 * flops, kms, "k_pair_gemm<bf16, fp64-split>"), cpu, err, note,
         dtype="f64_emu", dense_V_ms=ms_den, V_bytes_packed=Vp.numel() * 8, V_bytes_dense=Vd.numel() * 8,
         max_abs_diff_sym_vs_dense=diff)


def wl_gemmt(args):
    """f3: C := C - A T A^T (T skew-symmetric tridiagonal), lower triangle of C;
    flops counted as n (n + 1) k."""
    import torch
    import oracle
    import paper_2604_07311_b300 as fm
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    for n, k in ((16384, 256), (8192, 8192)):
        flops = n * (n + 1) * k
        for dt, tdt, kind, pairs, kname in (("f64_emu", torch.float64, "bf16", 21, "k_pair_gemm<bf16, fp64-split>"),
                                            ("f32", torch.float32, "tf32", 3, "k_pair_gemm<tf32x3>"),
                                            ("f64", torch.float64, "fp64", 1, "k_simt<double>")):
            A = torch.randn(k, n, device="cuda", dtype=tdt, generator=gen).t()  # column-major
            sub = torch.randn(k - 1, device="cuda", dtype=tdt, generator=gen)
            C = torch.randn(n, n, device="cuda", dtype=tdt, generator=gen).t()
            C0 = C.clone()
            f = lambda **kw: fm.gemmt_tridiag(-1.0, A, sub, None, None, 1.0, C, dtype=dt, **kw)
            steps = args.steps if dt != "f64" else max(1, min(args.steps, 3))
            ms = _cuda_ms(f, steps, min(args.warmup, 3) if dt == "f64" else args.warmup)
            kms = _product_ms(f, 3)
            C.copy_(C0)
            f()
            torch.cuda.synchronize()
            # oracle: B = T A^T formed on the host (the band, as the oracle's own
            # gemmt does), then sampled entries i >= j of C0 - A B
            Ah, sh, C0h = host64(A), host64(sub), host64(C0)
            Bt = np.zeros((k, n))
            Bt[1:] += sh[:, None] * Ah.T[:-1]
            Bt[:-1] -= sh[:, None] * Ah.T[1:]
            rng = np.random.default_rng(15)
            i = rng.integers(0, n, 512)
            j = (rng.random(512) * (i + 1)).astype(np.int64)
            idx = np.stack([i, j], 1)
            want = oracle.entries(-1.0, Ah, [1, 3], Bt, [3, 2], 1.0, C0h, [1, 2], idx, dot2=dt == "f64_emu")
            got = host64(C)[i, j]
            err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
            cpu = cpu_slice(-1.0, Ah, [1, 3], Bt, [3, 2], 1.0, C0h, [1, 2], 2.0)
            emit(f"gemmt_skew_tridiag_n{n}_k{k}", flops, ms, roofline(kind, pairs * flops, kms, kname), cpu, err,
                 "512 sampled entries i >= j vs the oracle (B = T A^T on the host, then its sums)", dtype=dt)
            del A, C, C0
            torch.cuda.empty_cache()


def wl_mttkrp(args):
    """f4: CP-ALS's M = X_(n) (Khatri-Rao of the other factors), X 512^3, R = 64, every mode."""
    import torch
    import oracle
    import paper_2604_07311_b300 as fm
    gen = torch.Generator(device="cuda")
    gen.manual_seed(8)
    I, R = 512, 64
    flops = 2 * I ** 3 * R
    for dt, tdt, kind, pairs, kname in (("f64_emu", torch.float64, "bf16", 21, "k_pair_gemm<bf16, fp64-split>"),
                                        ("f32", torch.float32, "tf32", 3, "k_pair_gemm<tf32x3>"),
                                        ("f64", torch.float64, "fp64", 1, "k_simt<double>")):
        X = torch.randn(I, I, I, device="cuda", dtype=tdt, generator=gen).permute(2, 1, 0)  # column-major
        U = [torch.randn(R, I, device="cuda", dtype=tdt, generator=gen).t() for _ in range(3)]
        Xh = host64(X)
        Uh = [host64(u) for u in U]
        for mode in range(3):
            M = torch.zeros(R, I, device="cuda", dtype=tdt).t()
            f = lambda **kw: fm.mttkrp(1.0, X, mode, U, 0.0, M, dtype=dt, **kw)
            steps = args.steps if dt != "f64" else max(1, min(args.steps, 3))
            ms = _cuda_ms(f, steps, min(args.warmup, 2) if dt == "f64" else args.warmup)
            kms = _product_ms(f, 3)
            f()
            torch.cuda.synchronize()
            Kt = oracle.khatri_rao(Uh, mode, 3)  # Kt[i_a, i_b, r] over the other modes a < b
            others = [m for m in range(3) if m != mode]
            lx = [1, 2, 3]
            lk = [others[0] + 1, others[1] + 1, 9]
            err, note = sampled_error(1.0, Xh, lx, Kt, lk, 0.0, np.zeros((I, R)), [mode + 1, 9], host64(M), n=256,
                                      dot2=dt == "f64_emu")
            cpu = cpu_slice(1.0, Xh, lx, Kt, lk, 0.0, np.zeros((I, R)), [mode + 1, 9], 2.0)
            emit(f"mttkrp_3way_{I}_R{R}_mode{mode}", flops, ms, roofline(kind, pairs * flops, kms, kname), cpu, err,
                 note, dtype=dt)
        del X, U, Xh, Uh
        torch.cuda.empty_cache()


def run_other(args):
    """Secondary workloads (one JSON line each): not the headline metric."""
    import torch
    torch.cuda.set_device(0)
    fns = {"four_index": wl_four_index, "transpose_free": wl_transpose_free, "block_sparse": wl_block_sparse,
           "autograd": wl_autograd, "network": wl_network, "ladder_sym": wl_ladder_sym, "gemmt": wl_gemmt,
           "mttkrp": wl_mttkrp}
    names = list(fns) if args.workload == "all" else [args.workload]
    for n in names:
        fns[n](args)
        torch.cuda.empty_cache()
    import paper_2604_07311_b300 as fm
    print(json.dumps({"device_status": fm.device_status()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="ladder",
                    choices=["ladder", "four_index", "transpose_free", "block_sparse", "autograd", "network",
                             "ladder_sym", "gemmt", "mttkrp", "all"],
                    help="ladder is the benchmark line; the others print secondary measurements")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="famlies", choices=["famlies", "reference"])
    ap.add_argument("--ref-cols", type=int, default=32,
                    help="output columns (i,j pairs) in the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-block", action="store_true",
                    help="block_sparse: skip the one-call-per-block comparison (profiling captures only)")
    ap.add_argument("--v", type=int, default=128, help="virtual extent (profiling captures only)")
    ap.add_argument("--o", type=int, default=32, help="occupied extent (profiling captures only)")
    args = ap.parse_args()
    set_size(args.v, args.o)
    if args.workload != "ladder":
        run_other(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
