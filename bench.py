#!/usr/bin/env python
"""Benchmark: 3D FCGLE on a 256^3 grid, Krogstad's exponential RK4 (phi_1..phi_3),
tau = 1e-3, complex64 storage with split-BF16 tensor-core mode products.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One "step" is one Krogstad time step of the whole hot path (4 forward + 4
backward 3D Tucker operators = 24 mode products, the nonlinearity, the
spectral stage combinations) over the 256^3 tensor.  The timed region is one
fcgle_integrate call of K steps (CUDA events on the handle's stream, inputs
resident in HBM, every tensor 134 MB > L2).  Prints one JSON line on rank 0.

Multi-GPU: one independent replica per GPU (the single-instance path has no
data-parallel split without an all-to-all exchange), weak scaling.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_GRID = 256
BOXES = [(-10.0, 10.0)] * 3
ALPHAS = [1.2, 1.5, 1.8]
PARS = dict(nu=1.0, eta=0.5, gamma=1.0, kappa=1.0, zeta=0.5)
TAU = 1e-3
KROGSTAD_BYTES_PER_ELEM = 16 * 16 + 32 + 3 * 24 + 32 + 40 + 40 + 24   # 496 B per complex element
SLAB_SAVED_BYTES_PER_ELEM = 8 * 16   # slab-fused modes 1 + 2: one 16-byte pass less per Tucker operator


def tucker_form_of(report, n):
    """'slab-fused' or 'rotating': the autotuner's choice for an n^3 split-BF16
    handle (its extents are n rounded up to a multiple of 8)."""
    p = (n + 7) // 8 * 8
    m = re.search(r"tucker p=\(%d,%d,%d\):.*-> (\S+)" % (p, p, p), report)
    return m.group(1) if m else "rotating"

# 2D 1023 x 1024 workload (linearly-implicit Euler and ETD2RK, 500 steps): the
# mode products contract p = 1024, so they are bound by the tensor pipe, not HBM
C2_NS = [1023, 1024]
C2_BOXES = [(-20.0, 20.0)] * 2
C2_ALPHAS = [1.3, 1.7]
C2_PARS = dict(nu=1.0, eta=1.0, gamma=0.5, kappa=1.0, zeta=-1.0)
C2_STEPS = 500


def etd2rk_bytes_per_elem(d):
    """Algorithmic bytes per complex element of one split-BF16 ETD2RK step in d
    dimensions: 4 Tucker operators of d - 1 plain mode products (16 B each) and
    the epilogues of their last products (EpiFhat without F^: X, U^ read, S, U^
    written, 32 B; EpiStageD 24; EpiEtd2 32; EpiUpdateG 24)."""
    return 4 * 16 * (d - 1) + 32 + 24 + 32 + 24
METRIC = "DoF*steps/s"
UNIT = "DoF*steps/s"


SCHEME_NAMES = {"krogstad": "Krogstad exponential RK4 (phi_1..phi_3)", "etd2rk": "ETD2RK", "lie": "linearly-implicit Euler",
                "lbdf2": "linearised BDF2", "strang": "Strang splitting", "lawson_euler": "Lawson-Euler",
                "lawson_rk2": "Lawson-RK2"}


def workload_config(n, precision="bf16x3", scheme="krogstad", tau=TAU, exp_form="tucker"):
    return {
        "exp_form": exp_form,
        "workload": f"3D FCGLE {n}^3 on (-10,10)^3, alpha=(1.2,1.5,1.8), nu=1, eta=0.5, gamma=1, kappa=1, "
                    f"zeta=0.5; {SCHEME_NAMES[scheme]}, tau={tau:g}; u0 = Gaussian bump x "
                    f"smoothed random phase (seed 1)",
        "grid": [n, n, n],
        "scheme": scheme,
        "tau": tau,
        "precision": precision,
        "storage": "complex64" if precision == "bf16x3" else "complex128",
        "l2": "inputs larger than L2 (each 256^3 tensor is 134 MB complex64)",
        "parallelism": "replicas (one independent instance per GPU)",
    }


# --------------------------------------------------------------- CPU oracle
def cpu_sample(n, max_steps, budget_s):
    """The FP64 oracle (as it stands) on the same workload: setup, then whole
    Krogstad steps until max_steps or the time budget is used."""
    import numpy as np
    from oracle import schemes, tensor
    from paper_2510_21394_gb300 import inputs
    ns = [n, n, n]
    t0 = time.perf_counter()
    P = tensor.Problem(ns, BOXES, ALPHAS, *PARS.values())
    S = tensor.Spectral(P)
    for l in (1, 2):
        S.F("phi", l, TAU / 2)
    for l in (1, 2, 3):
        S.F("phi", l, TAU)
    setup = time.perf_counter() - t0
    u = inputs.gaussian_random_phase(ns, BOXES, seed=1)
    g = schemes.Nonlinearity(P)
    done, t_run = 0, 0.0
    while done < max_steps:
        t1 = time.perf_counter()
        u = schemes.krogstad_step(S, g, TAU, done * TAU, u)
        t_run += time.perf_counter() - t1
        done += 1
        if t_run > budget_s:
            break
    assert np.all(np.isfinite(u))
    return {"value": n ** 3 * done / t_run, "seconds": t_run, "steps": done, "setup_s": setup,
            "cores": os.cpu_count()}


def cpu_sample_batched(ninst, max_steps, budget_s):
    """The FP64 oracle on the batched workload: instances taken in a fixed
    order alternating 2D and 3D (setup excluded), ETD2RK steps each, until
    ninst instances are done or the time budget is used."""
    from oracle import schemes, tensor
    from paper_2510_21394_gb300 import inputs
    specs = inputs.batched_instances()
    two = [sp for sp in specs if len(sp["ns"]) == 2]
    three = [sp for sp in specs if len(sp["ns"]) == 3]
    order = [x for pair in zip(two, three) for x in pair]
    dofsteps, t_run, done, setup = 0, 0.0, 0, 0.0
    for sp in order[:ninst]:
        t0 = time.perf_counter()
        P = tensor.Problem(sp["ns"], sp["boxes"], sp["alphas"], sp["nu"], sp["eta"], sp["gamma"], sp["kappa"],
                           sp["zeta"])
        S = tensor.Spectral(P)
        S.F("phi", 1, TAU)
        S.F("phi", 2, TAU)
        setup += time.perf_counter() - t0
        g = schemes.Nonlinearity(P)
        u = inputs.gaussian_pulse(sp["ns"], sp["boxes"])
        t1 = time.perf_counter()
        u = schemes.integrate(S, g, "etd2rk", TAU, max_steps, u)
        t_run += time.perf_counter() - t1
        dofsteps += int(np.prod(sp["ns"])) * max_steps
        done += 1
        if t_run > budget_s:
            break
    return {"value": dofsteps / t_run, "seconds": t_run, "instances": done, "steps": max_steps, "setup_s": setup,
            "cores": os.cpu_count()}


def cpu_sample_2d(scheme, max_steps, budget_s):
    """The FP64 oracle (as it stands) on the 2D 1023 x 1024 workload: setup,
    then whole steps of `scheme` until max_steps or the time budget is used."""
    from oracle import schemes, tensor
    from paper_2510_21394_gb300 import inputs
    t0 = time.perf_counter()
    P = tensor.Problem(C2_NS, C2_BOXES, C2_ALPHAS, *C2_PARS.values())
    S = tensor.Spectral(P)
    if scheme == "lie":
        S.F("inv", 0, TAU)
    else:
        S.F("phi", 1, TAU)
        S.F("phi", 2, TAU)
    setup = time.perf_counter() - t0
    u = inputs.sech_pulse_noise(C2_NS, C2_BOXES, seed=0)
    g = schemes.Nonlinearity(P)
    done, t_run = 0, 0.0
    while done < max_steps:
        t1 = time.perf_counter()
        u = schemes.integrate(S, g, scheme, TAU, 1, u, t0=done * TAU)
        t_run += time.perf_counter() - t1
        done += 1
        if t_run > budget_s:
            break
    assert np.all(np.isfinite(u))
    return {"value": int(np.prod(C2_NS)) * done / t_run, "seconds": t_run, "steps": done, "setup_s": setup,
            "cores": os.cpu_count()}


def run_cpu_sample_subprocess(n, max_steps, budget_s, timeout_s, batched=False):
    if batched:
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample-batched", str(n), str(max_steps),
               str(budget_s)]
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
        for line in r.stdout.splitlines()[::-1]:
            if line.startswith("{"):
                return json.loads(line)
        raise RuntimeError(f"cpu sample failed: {r.stderr[-2000:]}")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(n), str(max_steps), str(budget_s)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError(f"cpu sample failed: {r.stderr[-2000:]}")


def run_cpu_sample_2d_subprocess(scheme, max_steps, budget_s, timeout_s):
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample-2d", scheme, str(max_steps), str(budget_s)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError(f"cpu sample failed: {r.stderr[-2000:]}")


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(gpu_index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None
        self.t_start = self.t_end = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        import statistics
        reasons = sorted({self.NAMES[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------ helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def measured_bf16_peak():
    """Dense bf16 tensor peak in TFLOP/s (burst, sustained) and its provenance."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    return 1900.0, 1700.0, "fallback"


def l2_flush_buffer(torch):
    """A 256 MB device buffer; writing it evicts every line of the 129 MB L2."""
    return torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")


def tf32_peak_tflops(torch, n=8192, reps=5):
    """TF32 tensor-core matrix-multiply rate, measured here: torch.matmul on
    n x n float32 operands with TF32 allowed (cuBLAS), best of reps, CUDA events."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(n, n, dtype=torch.float32, device="cuda")
        b = torch.randn(n, n, dtype=torch.float32, device="cuda")
        c = a @ b
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def dgemm_peak_tflops(torch, n=4096, reps=5):
    """FP64 matrix-multiply rate of this GPU, measured here: torch.matmul on
    n x n float64 operands (cuBLAS DGEMM), best of reps, CUDA events."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


PLAIN_SOURCES = ("b3_plain.cuh", "b3_kernel.cuh")
SLAB_SOURCES = ("b3_slab.cuh", "b3_kernel.cuh")


def kernel_source_sha(files=PLAIN_SOURCES):
    """sha256[:16] of a kernel's sources (the files in order; the plain mode
    product: b3_plain.cuh, then b3_kernel.cuh)."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2510_21394_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(n, profile="mp_b3_plain_256cube.md", files=PLAIN_SOURCES):
    """DRAM bytes per launch of a kernel from its committed ncu summary, if the
    summary was taken on the current kernel source."""
    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    sha = kernel_source_sha(files)
    text = open(prof).read()
    m_sha = re.search(r"kernel source sha256\[:16\]:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic bytes per launch \(scaled to %d\^3\):\s*([0-9.eE+]+)" % n, text)
    if not m_sha or not m_tr or m_sha.group(1) != sha:
        return None
    return float(m_tr.group(1))


def gpu_index_for(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ------------------------------------------------------------ multi-rank
def max_over_ranks(x, world):
    """Largest value of x over all ranks (x itself at world size 1); works on
    NCCL (CUDA tensor) and gloo (CPU tensor) process groups."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, steps, seconds, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / seconds


# -------------------------------------------------------------- main arms
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    budget = float(os.environ.get("FCGLE_REF_BUDGET_S", "60"))
    res = run_cpu_sample_subprocess(N_GRID, max(1, args.steps), budget, timeout_s=1800)
    line = {
        "impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(N_GRID, "fp64-oracle"),
        "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                         "sample": f"{res['steps']} whole Krogstad step(s) of the {N_GRID}^3 workload "
                                   f"(of the {args.steps} requested; time budget {budget:.0f} s), numpy FP64 "
                                   f"tensor-form oracle, setup ({res['setup_s']:.1f} s) excluded"},
        "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if rank == 0:
        import __graft_entry__ as g
        g.build()
    if world > 1:
        dist.barrier()
    from paper_2510_21394_gb300 import fcgle, inputs

    n = args.n
    ns = [n, n, n]
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    solver = fcgle.Solver(ns, BOXES, ALPHAS, **PARS, precision="bf16x3")
    if args.exp_form != "tucker":
        solver.set_exp_form(args.exp_form)
    setup_s = time.perf_counter() - t0
    u0_np = inputs.gaussian_random_phase(ns, BOXES, seed=1)
    u0 = torch.from_numpy(u0_np).to(torch.complex64).cuda()
    out = torch.empty_like(u0)

    # warm-up (also fills the cached phi tensors)
    solver.integrate(args.scheme, args.tau, args.warmup, u0, out=out)
    solver.sync()
    torch.cuda.synchronize()

    clock = ClockSampler(gpu_index_for(local_rank)) if rank == 0 else None
    time.sleep(0.3 if clock else 0.0)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = solver.launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.integrate(args.scheme, args.tau, args.steps, u0, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = solver.launches() - l0
    solver.sync()
    ms = max_over_ranks(ms, world)
    clocks = clock.stop() if clock else None
    dof = n ** 3
    value = aggregate_rate(dof, args.steps, ms / 1e3, world)

    # ---- dominant kernel: the split-BF16 mode product, timed alone on the same stream
    P = fcgle.fcgle_internal_elems(solver.h)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float32).to(torch.bfloat16)
    X = torch.cat([X, torch.zeros_like(X)])      # split input: hi planes, lo planes
    Y = torch.empty_like(X)
    for d_ in range(3):
        fcgle.fcgle_mode_product(solver.h, d_, 3, X, Y)
    torch.cuda.synchronize()
    reps = 5
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        for d_ in range(3):
            fcgle.fcgle_mode_product(solver.h, d_, 3, X, Y)
    k1.record(stream)
    torch.cuda.synchronize()
    solver.sync()
    mp_ms = k0.elapsed_time(k1) / (3 * reps)
    mp_bytes = 2 * (2 * P * 4)       # read X, write Y (hi + lo bf16 = 4 B per real)
    peak, peak_kind = measured_peaks()
    achieved = mp_bytes / (mp_ms / 1e3) / 1e9
    plain_roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                  "frac": round(achieved / peak, 4), "traffic": ncu_traffic(n),
                  "kernel": "mp_b3_plain_kernel (one 256^3 mode product, split in/out)",
                  "peak_kind": f"{peak_kind} hbm_gbs (burst)", "launch_ms": round(mp_ms, 4), "algorithmic_bytes": mp_bytes}
    # ---- the slab-fused mode-1 + mode-2 product and the natural-order mode-3 product
    form = tucker_form_of(fcgle.fcgle_autotune_report(), n)
    slab_eligible = (n + 7) // 8 * 8 <= 256      # the slab kernel needs p_2 <= 256
    timed = {}
    for name, d_, fl in ((("slab12", 0, 1 | 2 | 8), ("mn3", 2, 1 | 2 | 16)) if slab_eligible else ()):
        fcgle.fcgle_mode_product(solver.h, d_, fl, X, Y)
        torch.cuda.synchronize()
        k0.record(stream)
        for _ in range(reps):
            fcgle.fcgle_mode_product(solver.h, d_, fl, X, Y)
        k1.record(stream)
        torch.cuda.synchronize()
        solver.sync()
        timed[name] = k0.elapsed_time(k1) / reps
    # FLOPs of the slab kernel: two mode products, 3 split passes, 2 p flops per real element
    sl_flops = 2 * 3 * 2 * ((n + 7) // 8 * 8) * 2 * P
    bf_peak, _, bf_kind = measured_bf16_peak()
    slab_roof = mn_roof = None
    if slab_eligible:
        sl_tf = sl_flops / (timed["slab12"] / 1e3) / 1e12
        slab_roof = {"bound": "tensor", "achieved": round(sl_tf, 1), "peak": bf_peak, "unit": "TFLOP/s",
                     "frac": round(sl_tf / bf_peak, 4),
                     "traffic": ncu_traffic(n, "mp_b3_slab12_256cube.md", SLAB_SOURCES),
                     "kernel": f"mp_b3_slab12_kernel (modes 1 + 2 of a {n}^3 Tucker operator, split in/out)",
                     "peak_kind": f"{bf_kind} bf16_tflops (burst)", "launch_ms": round(timed["slab12"], 4),
                     "algorithmic_flops": sl_flops, "algorithmic_bytes": mp_bytes,
                     "hbm_frac": round(mp_bytes / (timed["slab12"] / 1e3) / 1e9 / peak, 4)}
        mn_gbs = mp_bytes / (timed["mn3"] / 1e3) / 1e9
        mn_roof = {"bound": "hbm", "achieved": round(mn_gbs, 1), "peak": peak, "unit": "GB/s",
                   "frac": round(mn_gbs / peak, 4),
                   "kernel": "mp_b3_kernel<EpiStoreSplitGen, natural order> (mode 3 on the slab kernel's output)",
                   "launch_ms": round(timed["mn3"], 4), "algorithmic_bytes": mp_bytes}
    roofline = slab_roof if (form == "slab-fused" and slab_roof) else plain_roof
    del X, Y
    # ---- the precise end-transform product (split-TF32 on the tensor cores, FP32 in and out:
    # the split pass 24 B + the product 24 B per complex element), per launch pair
    Xf = torch.randn(2 * P, device="cuda", dtype=torch.float32)
    Yf = torch.empty_like(Xf)
    fcgle.fcgle_mode_product(solver.h, 0, 1 | 4, Xf, Yf)
    torch.cuda.synchronize()
    k0 = torch.cuda.Event(enable_timing=True)
    k1 = torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(reps):
        fcgle.fcgle_mode_product(solver.h, 0, 1 | 4, Xf, Yf)
    k1.record(stream)
    torch.cuda.synchronize()
    solver.sync()
    pt_ms = k0.elapsed_time(k1) / reps
    pt_bytes = 48 * P
    precise = {"kernels": "tf32_split_kernel + mp_b3_plain_kernel<kOpTF32F> (one 256^3 product, FP32 in/out)",
               "ms": round(pt_ms, 4), "achieved_gbs": round(pt_bytes / (pt_ms / 1e3) / 1e9, 1),
               "frac_of_hbm": round(pt_bytes / (pt_ms / 1e3) / 1e9 / peak, 4), "algorithmic_bytes": pt_bytes,
               "tflops": round(3 * 2 * n * 2 * P / (pt_ms / 1e3) / 1e12, 1)}
    del Xf, Yf
    # the whole step against HBM: algorithmic bytes per element of one Krogstad step
    # (16 plain products x 16 B; EpiFhat 32, 3 x EpiStageD 24, EpiKrog2 32, EpiKrog3 40,
    # EpiKrogFinal 40, EpiUpdateG 24) over the padded tensor
    step_roof = None
    if args.scheme == "krogstad":
        step_bytes = (KROGSTAD_BYTES_PER_ELEM - (SLAB_SAVED_BYTES_PER_ELEM if form == "slab-fused" else 0)) * P
        step_gbs = step_bytes / (ms / args.steps / 1e3) / 1e9
        step_roof = {"algorithmic_bytes": step_bytes, "achieved": round(step_gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_gbs / peak, 4), "floor_ms": round(step_bytes / (peak * 1e9) * 1e3, 4)}

    # ---- end to end through the C ABI with host buffers
    hin = torch.from_numpy(u0_np.astype(np.complex64)).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    solver.integrate_host(args.scheme, args.tau, args.steps, hin, hout)
    e2e_s = max_over_ranks(time.perf_counter() - t1, world)
    e2e = {"value": aggregate_rate(dof, args.steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": hin.numel() * 8 / args.steps, "d2h_bytes_per_step": hout.numel() * 8 / args.steps,
           "note": "fcgle_integrate_host: one H2D of u0 (pinned) and one D2H of u(T) per call of K steps, "
                   "synchronised, wall clock"}

    extra = {}
    if not args.no_fp64 and rank == 0:
        # ---- the plain FP64 GPU form on the same workload, and the accuracy of BF16x3 against it
        acc_steps = min(args.steps, args.accuracy_steps)
        s64 = fcgle.Solver(ns, BOXES, ALPHAS, **PARS, precision="fp64")
        v64 = torch.from_numpy(u0_np).cuda()
        o64 = torch.empty_like(v64)
        s64.integrate(args.scheme, args.tau, 1, v64, out=o64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64.integrate(args.scheme, args.tau, 2, v64, out=o64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / 2
        s64.integrate(args.scheme, args.tau, acc_steps, v64, out=o64)
        solver.integrate(args.scheme, args.tau, acc_steps, u0, out=out)
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm(out.to(torch.complex128) - o64) / torch.linalg.vector_norm(o64))
        s64.sync()
        s64.close()
        extra["fp64_gpu"] = {"value": dof / (ms64 / 1e3), "unit": UNIT, "ms_per_step": round(ms64, 2),
                             "speedup_of_bf16x3": round((dof * args.steps / (ms / 1e3) / world) / (dof / (ms64 / 1e3)), 1)}
        extra["accuracy"] = {"steps": acc_steps, "rel_err_vs_fp64_gpu": err,
                             "note": "FP64 GPU path is parity-tested against the FP64 oracle at <= 1e-12"}
    solver.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.scheme == "krogstad":
        try:
            res = run_cpu_sample_subprocess(n, 1, 0.0, timeout_s=900)
            cpu = {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                   "sample": f"{res['steps']} whole Krogstad step of the {n}^3 workload ({res['seconds']:.1f} s), "
                             f"numpy FP64 tensor-form oracle on the host cores, setup ({res['setup_s']:.1f} s) excluded"}
        except Exception as e:  # report, do not fail the GPU measurement
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}

    if rank == 0:
        extra["autotune"] = fcgle.fcgle_autotune_report().strip().splitlines()
        extra["precise_transform"] = precise
        extra["tucker_form"] = form
        extra["kernels"] = {"plain": plain_roof, "slab12": slab_roof, "mn3": mn_roof}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic", "config": workload_config(n, "bf16x3", args.scheme, args.tau, args.exp_form),
                "roofline": roofline, "step_roofline": step_roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "setup_s": round(setup_s, 3)}
        line.update(extra)
        print(json.dumps(line))
    return 0


def run_config2(args, rank, world, local_rank):
    """2D 1023 x 1024 on (-20,20)^2, alpha = (1.3, 1.7), sech pulse + noise (seed 0),
    linearly-implicit Euler and ETD2RK, tau = 1e-3, 500 steps, split-BF16.  Here
    every mode product contracts p = 1024 (arithmetic intensity 256 FLOP/B at
    complex64, x 3 for the split passes), so the roofline is the tensor pipe."""
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        import __graft_entry__ as g
        g.build()
    if world > 1:
        dist.barrier()
    from paper_2510_21394_gb300 import fcgle, inputs
    steps = args.steps if args.steps is not None else C2_STEPS
    stream = torch.cuda.current_stream()
    dof = int(np.prod(C2_NS))
    u0_np = inputs.sech_pulse_noise(C2_NS, C2_BOXES, seed=0)
    u0 = torch.from_numpy(u0_np).to(torch.complex64).cuda()
    out = torch.empty_like(u0)
    solver = fcgle.Solver(C2_NS, C2_BOXES, C2_ALPHAS, **C2_PARS, precision="bf16x3")
    flush = l2_flush_buffer(torch)
    per = {}
    clocks = None
    for scheme in ("lie", "etd2rk"):
        solver.integrate(scheme, TAU, args.warmup, u0, out=out)
        solver.sync()
        clock = ClockSampler(gpu_index_for(local_rank)) if (rank == 0 and scheme == "etd2rk") else None
        time.sleep(0.3 if clock else 0.0)
        flush.fill_(1.0)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = solver.launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.integrate(scheme, TAU, steps, u0, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        solver.sync()
        if clock:
            clocks = clock.stop()
        per[scheme] = {"value": aggregate_rate(dof, steps, ms / 1e3, world), "unit": UNIT,
                       "ms_per_step": ms / steps, "gpu_launches": solver.launches() - l0}

    # ---- dominant kernel: one split-BF16 mode product contracting p = 1024, per launch,
    # L2 flushed before each launch, CUDA events on the launching stream
    P = fcgle.fcgle_internal_elems(solver.h)
    X = torch.randn(2 * P, device="cuda", dtype=torch.float32).to(torch.bfloat16)
    X = torch.cat([X, torch.zeros_like(X)])
    Y = torch.empty_like(X)
    for d_ in range(2):
        fcgle.fcgle_mode_product(solver.h, d_, 3, X, Y)
    torch.cuda.synchronize()
    times = []
    for rep in range(10):
        for d_ in range(2):
            flush.fill_(float(rep))
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
            fcgle.fcgle_mode_product(solver.h, d_, 3, X, Y)
            k1.record(stream)
            torch.cuda.synchronize()
            times.append(k0.elapsed_time(k1))
    solver.sync()
    mp_ms = sum(times) / len(times)
    p = 1024                                   # both directions pad to 1024
    mp_flop = 3 * 2 * p * (2 * P)              # 3 split passes x 2 p flop per real output element
    peak, peak_sus, peak_kind = measured_bf16_peak()
    achieved = mp_flop / (mp_ms / 1e3) / 1e12
    roofline = {"bound": "tensor", "achieved": round(achieved, 1), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "mp_b3_plain_kernel (one 1024 x 1024 mode product, p = 1024, split in/out)",
                "peak_kind": f"{peak_kind} bf16_tflops (burst)", "launch_ms": round(mp_ms, 5),
                "algorithmic_flop": mp_flop,
                "flop_note": "3 bf16 passes (hi.hi + hi.lo + lo.hi) x 2 p FLOP per real output element"}
    del X, Y
    # whole ETD2RK step against the tensor peak (sustained): 4 Tucker operators x 2 mode products
    step_flop = 4 * 2 * mp_flop
    step_tf = step_flop / (per["etd2rk"]["ms_per_step"] / 1e3) / 1e12
    step_roof = {"algorithmic_flop": step_flop, "achieved": round(step_tf, 1), "peak": peak_sus,
                 "unit": "TFLOP/s", "frac": round(step_tf / peak_sus, 4),
                 "peak_kind": f"{peak_kind} bf16_tflops_sustained"}

    # ---- end to end through the C ABI with host buffers (ETD2RK)
    hin = torch.from_numpy(u0_np.astype(np.complex64)).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    solver.integrate_host("etd2rk", TAU, steps, hin, hout)
    e2e_s = max_over_ranks(time.perf_counter() - t1, world)
    e2e = {"value": aggregate_rate(dof, steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": hin.numel() * 8 / steps, "d2h_bytes_per_step": hout.numel() * 8 / steps,
           "note": "fcgle_integrate_host: one H2D of u0 (pinned) and one D2H of u(T) per call of K steps, "
                   "synchronised, wall clock"}

    extra = {}
    if not args.no_fp64 and rank == 0:
        # ---- the plain FP64 GPU form: rate, its mode product against the measured DGEMM rate,
        # and the split-BF16 error at T against it
        dpeak = dgemm_peak_tflops(torch)
        s64 = fcgle.Solver(C2_NS, C2_BOXES, C2_ALPHAS, **C2_PARS, precision="fp64")
        v64 = torch.from_numpy(u0_np).cuda()
        o64 = torch.empty_like(v64)
        f64 = {}
        acc_steps = min(steps, args.accuracy_steps if args.accuracy_steps is not None else steps)
        for scheme in ("lie", "etd2rk"):
            s64.integrate(scheme, TAU, 1, v64, out=o64)
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            s64.integrate(scheme, TAU, 5, v64, out=o64)
            f1.record(stream)
            torch.cuda.synchronize()
            ms64 = f0.elapsed_time(f1) / 5
            s64.integrate(scheme, TAU, acc_steps, v64, out=o64)
            solver.integrate(scheme, TAU, acc_steps, u0, out=out)
            torch.cuda.synchronize()
            d = out.to(torch.complex128) - o64
            f64[scheme] = {"value": dof / (ms64 / 1e3), "ms_per_step": round(ms64, 3),
                           "speedup_of_bf16x3": round(per[scheme]["value"] / world / (dof / (ms64 / 1e3)), 1),
                           "rel_err_at_T": float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(o64)),
                           "max_rel_err_at_T": float(d.abs().max() / o64.abs().max()),
                           "T_steps": acc_steps}
        P64 = fcgle.fcgle_internal_elems(s64.h)
        X64 = torch.randn(2 * P64, device="cuda", dtype=torch.float64)
        Y64 = torch.empty_like(X64)
        fcgle.fcgle_mode_product(s64.h, 0, 1, X64, Y64)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(3):
            fcgle.fcgle_mode_product(s64.h, 0, 1, X64, Y64)
        g1.record(stream)
        torch.cuda.synchronize()
        ms_mp64 = g0.elapsed_time(g1) / 3
        p64 = 1024
        tf64 = 2 * p64 * (2 * P64) / (ms_mp64 / 1e3) / 1e12
        s64.sync()
        s64.close()
        del X64, Y64
        extra["tf32_peak_tflops"] = {"value": round(tf32_peak_tflops(torch), 1),
                                     "how": "measured here: cuBLAS TF32 (torch.matmul float32, TF32 allowed, 8192^3, "
                                            "best of 5); context for the split-TF32 end transforms"}
        extra["fp64_gpu"] = f64
        extra["fp64_roofline"] = {"bound": "fp64", "achieved": round(tf64, 3), "peak": round(dpeak, 3),
                                  "unit": "TFLOP/s", "frac": round(tf64 / dpeak, 4),
                                  "kernel": "mp_simt_kernel<double> (one 1024 x 1024 mode product)",
                                  "peak_kind": "measured here: cuBLAS DGEMM (torch.matmul float64, 4096^3, best of 5)"}
    solver.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            res = run_cpu_sample_2d_subprocess("etd2rk", steps, 20.0, timeout_s=900)
            cpu = {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                   "sample": f"{res['steps']} ETD2RK steps of the 1023 x 1024 workload ({res['seconds']:.1f} s), "
                             f"numpy FP64 tensor-form oracle on the host cores, setup ({res['setup_s']:.1f} s) "
                             f"excluded"}
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    if rank == 0:
        extra["autotune"] = fcgle.fcgle_autotune_report().strip().splitlines()
        line = {"metric": METRIC, "value": per["etd2rk"]["value"], "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": per["etd2rk"]["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
                "config": {"workload": "2D FCGLE 1023x1024 on (-20,20)^2, alpha=(1.3,1.7), nu=1, eta=1, gamma=0.5, "
                                       "kappa=1, zeta=-1, no source; u0 = sech(|x|) exp(0.5 i x_1) + U(-1e-3,1e-3) "
                                       "noise (seed 0); ETD2RK (value) and linearly-implicit Euler, tau=1e-3",
                           "grid": C2_NS, "scheme": "etd2rk", "tau": TAU, "precision": "bf16x3",
                           "storage": "complex64",
                           "l2": "the workload's own working set (about 70 MB) fits in L2; L2 flushed before the "
                                 "timed call and before each timed kernel launch",
                           "parallelism": "replicas (one independent instance per GPU)"},
                "schemes": per, "roofline": roofline, "step_roofline": step_roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": per["etd2rk"]["gpu_launches"], "clocks": clocks}
        line.update(extra)
        print(json.dumps(line))
    return 0


def batched_config(specs, use_graph):
    n2 = [sp["ns"][0] for sp in specs if len(sp["ns"]) == 2]
    n3 = [sp["ns"][0] for sp in specs if len(sp["ns"]) == 3]
    return {
        "workload": f"batched: {len(n2)} 2D grids n^2, n ~ U[128,768], and {len(n3)} 3D grids n^3, n ~ U[48,160] "
                    f"on (-10,10)^d; seeded alpha_mu in [1.1,1.9], nu in [0.5,2], eta, zeta in [-1,1], "
                    f"gamma in [0,1], kappa in [0.5,2]; Gaussian pulse u0; ETD2RK, tau=1e-3",
        "instances": len(specs), "dof_total": int(sum(int(np.prod(sp["ns"])) for sp in specs)),
        "n2_range": [min(n2), max(n2)] if n2 else None, "n3_range": [min(n3), max(n3)] if n3 else None,
        "scheme": "etd2rk", "tau": TAU, "precision": "bf16x3", "storage": "complex64",
        "launch": "grouped: one persistent launch per phase of a step over all instances, captured in a CUDA graph"
                  if use_graph else "direct launches",
        "l2": "working set of the batch (GBs) far above L2",
        "parallelism": "instances sharded over the GPUs (greedy balance by mode-product work), no collective",
    }


def run_batched(args, rank, world, local_rank):
    """The batched workload: many uneven instances advanced together, one
    CUDA-graph launch per step."""
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        import __graft_entry__ as g
        g.build()
    if world > 1:
        dist.barrier()
    from paper_2510_21394_gb300 import fcgle, inputs, sharding
    all_specs = inputs.batched_instances()
    # the instances are independent: each rank advances its share, balanced by
    # mode-product work, with no exchange on the data path (strong scaling)
    owner, _ = sharding.assign_instances([sp["ns"] for sp in all_specs], world)
    specs = [all_specs[i] for i in sharding.instances_of(owner, rank)]
    dof_all = sum(int(np.prod(sp["ns"])) for sp in all_specs)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    b = fcgle.Batch(specs, precision="bf16x3", stream=stream)
    setup_s = time.perf_counter() - t0
    u0n = [inputs.gaussian_pulse(sp["ns"], sp["boxes"]) for sp in specs]
    u0 = [torch.from_numpy(x).to(torch.complex64).cuda() for x in u0n]
    outs = [torch.empty_like(u) for u in u0]
    dof = sum(int(np.prod(sp["ns"])) for sp in specs)
    res = {}
    for mode in ("direct", "graph", "grouped"):
        use_graph, grouped = mode != "direct", mode == "grouped"
        b.integrate("etd2rk", TAU, args.warmup, u0, out=outs, use_graph=use_graph, grouped=grouped)
        torch.cuda.synchronize()
        clock = ClockSampler(gpu_index_for(local_rank)) if (rank == 0 and grouped) else None
        time.sleep(0.3 if clock else 0.0)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0, g0 = b.launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.integrate("etd2rk", TAU, args.steps, u0, out=outs, use_graph=use_graph, grouped=grouped)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        l1, g1 = b.launches()
        ms = max_over_ranks(ms, world)
        res[mode] = dict(ms=ms, launches=l1 - l0, graphs=g1 - g0, clocks=clock.stop() if clock else None)
    for i in range(len(specs)):
        fcgle.fcgle_sync(b.instance(i))
    # end to end: H2D of every u0 from pinned memory, the K graph steps, D2H of every u(T)
    hin = [torch.from_numpy(x.astype(np.complex64)).pin_memory() for x in u0n]
    hout = [torch.empty_like(x).pin_memory() for x in hin]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    dev = [x.to("cuda", non_blocking=True) for x in hin]
    b.integrate("etd2rk", TAU, args.steps, dev, out=outs, grouped=True)
    for o, h in zip(outs, hout):
        h.copy_(o, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t1, world)
    nbytes = sum(x.numel() * 8 for x in hin)
    b.close()
    r = res["grouped"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            c = run_cpu_sample_subprocess(96, 5, 20.0, timeout_s=900, batched=True)
            cpu = {"value": c["value"], "unit": UNIT, "cores": c["cores"], "kind": "oracle",
                   "sample": f"{c['instances']} instances (alternating 2D / 3D in draw order) x {c['steps']} ETD2RK "
                             f"steps ({c['seconds']:.1f} s), numpy FP64 tensor-form oracle, setup excluded"}
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
    if rank == 0:
        # the whole grouped step against HBM, over the instances' grid points
        peak, peak_kind = measured_peaks()
        step_bytes = sum(etd2rk_bytes_per_elem(len(sp["ns"])) * int(np.prod(sp["ns"])) for sp in all_specs)
        step_gbs = step_bytes / (r["ms"] / args.steps / 1e3) / 1e9
        step_roof = {"algorithmic_bytes": step_bytes, "achieved": round(step_gbs, 1), "peak": peak * world,
                     "unit": "GB/s", "frac": round(step_gbs / (peak * world), 4),
                     "floor_ms": round(step_bytes / (peak * world * 1e9) * 1e3, 4),
                     "peak_kind": f"{peak_kind} hbm_gbs (burst) x {world} GPU(s)"}
        tune = [ln for ln in fcgle.fcgle_autotune_report().strip().splitlines() if ln.startswith("batch phase")]
        line = {"metric": METRIC, "value": dof_all * args.steps / (r["ms"] / 1e3), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "bf16x3",
                "data": "synthetic", "config": batched_config(all_specs, True), "step_roofline": step_roof,
                "rank0_instances": len(specs),
                "e2e": {"value": dof_all * args.steps / e2e_s, "unit": UNIT,
                        "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
                        "note": "all u0 copied in from pinned memory and all u(T) copied out per call of K steps"},
                "gpu_launches": r["launches"], "graph_launches": r["graphs"], "clocks": r["clocks"],
                "cpu_baseline": cpu,
                "direct_launch": {"value": dof_all * args.steps / (res["direct"]["ms"] / 1e3),
                                  "ms_per_step": res["direct"]["ms"] / args.steps, "kernels": res["direct"]["launches"]},
                "graph_of_per_instance_launches": {
                    "value": dof_all * args.steps / (res["graph"]["ms"] / 1e3),
                    "ms_per_step": res["graph"]["ms"] / args.steps},
                "setup_s": round(setup_s, 2), "autotune_phases": tune}
        print(json.dumps(line))
    return 0


def run_adjoint(args, rank, world, local_rank):
    """Gradient of J = 1/2 ||u(T) - u_target||^2 w.r.t. u0 and (nu, eta, gamma, kappa, zeta):
    3D 128^3, alpha = 1.5, Lawson-RK2, tau = 2e-3, 250 steps, checkpoints every 25,
    u_target from a forward run with the parameters scaled by 1.05."""
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if rank == 0:
        import __graft_entry__ as g
        g.build()
    if world > 1:
        dist.barrier()
    from paper_2510_21394_gb300 import fcgle, inputs
    ns, boxes, al = [128] * 3, [(-10.0, 10.0)] * 3, [1.5] * 3
    pars = [1.0, 0.5, 1.0, 1.0, 0.5]
    tau, m, ck = 2e-3, 250, 25
    u0n = inputs.gaussian_random_phase(ns, boxes, seed=3)
    out = {}
    stream = torch.cuda.current_stream()
    s64 = fcgle.Solver(ns, boxes, al, *pars, precision="fp64")
    v64 = torch.from_numpy(u0n).cuda()
    s64.set_coefficients(*[1.05 * x for x in pars])
    target = s64.integrate("lawson_rk2", tau, m, v64)
    s64.set_coefficients(*pars)
    for prec in ("bf16x3", "fp64"):
        s = s64 if prec == "fp64" else fcgle.Solver(ns, boxes, al, *pars, precision=prec)
        dt = torch.complex128 if prec == "fp64" else torch.complex64
        v, tg = v64.to(dt), target.to(dt)
        s.adjoint("lawson_rk2", tau, 5, v, tg, ckpt_every=5)   # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss, gu, gp = s.adjoint("lawson_rk2", tau, m, v, tg, ckpt_every=ck)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
        out[prec] = dict(seconds=sec, loss=loss, gu=gu.to(torch.complex128), gp=gp)
        if prec != "fp64":
            s.close()
    dof = 128 ** 3
    g64 = out["fp64"]["gu"]
    o = out["bf16x3"]
    acc = {"loss_rel": abs(o["loss"] - out["fp64"]["loss"]) / out["fp64"]["loss"],
           "grad_u0_rel": float(torch.linalg.vector_norm(o["gu"] - g64) / torch.linalg.vector_norm(g64)),
           "params_max_rel": float(max(abs(a - b) / abs(b) for a, b in zip(o["gp"], out["fp64"]["gp"])))}
    s64.close()
    if rank == 0:
        line = {"metric": METRIC, "value": aggregate_rate(dof, m, o["seconds"], world), "unit": UNIT,
                "n_gpus": world, "steps": m, "warmup": 1, "ms_per_step": 1e3 * o["seconds"] / m,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3",
                "data": "synthetic",
                "config": {"workload": "adjoint: 3D 128^3 on (-10,10)^3, alpha=1.5, nu=1, eta=0.5, gamma=1, kappa=1, "
                                       "zeta=0.5, Lawson-RK2, tau=2e-3, 250 steps, checkpoints every 25; target from "
                                       "parameters x 1.05; gradient w.r.t. u0 and (nu, eta, gamma, kappa, zeta)",
                           "note": "value = grid points x steps of the forward map per second of one gradient "
                                   "(forward sweep, recompute and backward sweep)",
                           "parallelism": "replicas (one independent gradient per GPU)"},
                "fp64_gpu": {"value": aggregate_rate(dof, m, out["fp64"]["seconds"], world),
                             "seconds": out["fp64"]["seconds"]},
                "seconds": o["seconds"], "accuracy_vs_fp64_gpu": acc}
        print(json.dumps(line))
    return 0


def run_mp_only(args):
    """Raw mode products on internal-layout buffers, for kernel profiling."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2510_21394_gb300 import fcgle
    n = args.n
    if args.workload == "config2":
        s = fcgle.Solver(C2_NS, C2_BOXES, C2_ALPHAS, **C2_PARS, precision=args.precision)
        dims = 2
    else:
        ns = [n, n, args.n3 or n]
        s = fcgle.Solver(ns, BOXES, ALPHAS, **PARS, precision=args.precision)
        dims = 3
    P = fcgle.fcgle_internal_elems(s.h)
    if args.precision == "bf16x3":
        X = torch.randn(4 * P, device="cuda", dtype=torch.float32).to(torch.bfloat16)
        flags = 3                                   # forward, split input and output
    else:
        X = torch.randn(2 * P, device="cuda", dtype=torch.float64)
        flags = 1
    Y = torch.empty_like(X)
    # 3D split-BF16: also the slab-fused modes 1 + 2 and the natural-order mode 3
    extra = [(0, flags | 8), (2, flags | 16)] if dims == 3 and args.precision == "bf16x3" else []
    for _ in range(args.mp_only):
        for d_ in range(dims):
            fcgle.fcgle_mode_product(s.h, d_, flags, X, Y)
        for d_, fl in extra:
            fcgle.fcgle_mode_product(s.h, d_, fl, X, Y)
    torch.cuda.synchronize()
    s.sync()
    s.close()
    print(json.dumps({"mp_only": args.mp_only, "workload": args.workload, "n": n, "precision": args.precision,
                      "ok": True}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 200 for the cube workload, 500 for config2)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--accuracy-steps", type=int, default=None,
                    help="steps of the split-BF16 vs FP64 comparison (default: 20 for the cube, all for config2)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", nargs=3, default=None)
    ap.add_argument("--cpu-sample-batched", nargs=3, default=None)
    ap.add_argument("--cpu-sample-2d", nargs=3, default=None)
    ap.add_argument("--mp-only", type=int, default=0, metavar="REPS",
                    help="only run REPS x 3 raw mode products (all directions) of the n^3 workload (profiling)")
    ap.add_argument("--n3", type=int, default=None,
                    help="--mp-only, cube workload: third extent (default n), for profiling a smaller case")
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp64"])
    ap.add_argument("--scheme", default="krogstad", choices=sorted(SCHEME_NAMES),
                    help="cube workload: time-stepping scheme (default krogstad, the benchmark)")
    ap.add_argument("--tau", type=float, default=TAU)
    ap.add_argument("--exp-form", default="tucker", choices=["tucker", "kron"],
                    help="cube workload, split-BF16: how e^{tau K} is applied by Lawson-Euler, Lawson-RK2 and "
                         "Strang (Tucker form, or the Kronecker-product form with complex E_mu)")
    ap.add_argument("--workload", default="cube", choices=["cube", "batched", "adjoint", "config2"],
                    help="cube: one 3D n^3 instance (default Krogstad); batched: 96 uneven ETD2RK instances; "
                         "adjoint: gradient of a final-time misfit, 128^3 Lawson-RK2; config2: 2D 1023x1024 LIE "
                         "and ETD2RK (tensor-pipe bound)")
    args = ap.parse_args()
    if args.workload != "config2":
        if args.steps is None:
            args.steps = 200
        if args.accuracy_steps is None:
            args.accuracy_steps = 20
    if args.mp_only:
        return run_mp_only(args)
    if args.cpu_sample_batched:
        k, steps, budget = int(args.cpu_sample_batched[0]), int(args.cpu_sample_batched[1]), \
            float(args.cpu_sample_batched[2])
        print(json.dumps(cpu_sample_batched(k, steps, budget)))
        return 0
    if args.cpu_sample_2d:
        print(json.dumps(cpu_sample_2d(args.cpu_sample_2d[0], int(args.cpu_sample_2d[1]),
                                       float(args.cpu_sample_2d[2]))))
        return 0
    if args.cpu_sample:
        n, steps, budget = int(args.cpu_sample[0]), int(args.cpu_sample[1]), float(args.cpu_sample[2])
        print(json.dumps(cpu_sample(n, steps, budget)))
        return 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "batched":
            return run_batched(args, rank, world, local_rank)
        if args.workload == "adjoint":
            return run_adjoint(args, rank, world, local_rank)
        if args.workload == "config2":
            return run_config2(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
