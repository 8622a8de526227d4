"""Benchmark: QBX layer-potential targets/s on one GB300 (and N replicas under torchrun).

Default workload (the metric's mixed-vs-FP64 configuration): 200 random
non-overlapping ellipses in [0, 100]^2, k = 20, 65 536 panels x 16
Gauss-Legendre nodes (2^20 sources, 2^21 centres), double layer with a random
complex density, p = 16, p_fmm = 30, 9e5 uniform + 1e5 near-surface targets.
One step is one qbx_layer_potential_eval over all targets with the plan
prebuilt and the density resident on the device. Inputs are larger than L2,
and L2 is flushed (a 256 MiB write) before every timed step anyway.

The headline is the mixed-precision path (FP32 M2M/M2L/L2L and P2QBXL
accumulation, FP64 special functions and final sums) at its stated error
against the FP64 path, which is timed on the same plan and inputs and
reported beside it, with the speedup over the fastest FP64 plan of equal
accuracy. The same line carries the starfish (k = 10) and 256-curve batch
workloads as extra keys, and the FP64 oracle timed on all host cores and on
one core.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--mode fmm|direct] [--impl ours|reference] [--config 2|3|4|5]

--impl reference times the FP64 CPU oracle (the plain, slow definition) on the
host cores over a bounded sample of the same workload.
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

METRIC = "QBX-FMM layer-potential targets/sec at stated rel err, mixed vs FP64 on 1 GB300"
UNIT = "targets/s"
CONFIG_NUM = 5
WORKLOADS = {2: "%s: starfish r=1+0.3cos5t, k=10, 512 panels x 16 GL (8192 sources, 16384 "
                "centres), D+ikS with random Fourier density |n|<=20, p=12, p_fmm=20, 316x316 "
                "grid targets on [-2,2]^2",
             3: "%s: starfish r=1+0.3cos5t, k=50, 8192 panels x 16 GL (131072 sources, 262144 "
                "centres), D+ikS with random Fourier density |n|<=20, p=16, p_fmm=30, 316x316 "
                "grid targets on [-2,2]^2",
             4: "%s: 256 random curves r=1+sum_{m<=5} a_m cos(m t+phi_m), k~U(1,40), panels "
                "U{16..1024} x 16 GL raised to ceil(kL/5), D+ik_cS, p=12, p_fmm=20, every node "
                "an exterior on-surface target; one graph-captured batch, plans autotuned",
             5: "%s: 200 ellipses in [0,100]^2, k=20, 65536 panels x 16 GL (2^20 sources), "
                "double layer, p=16, p_fmm=30, 9e5 uniform + 1e5 near-surface targets"}
# FP64 FMA peak of a GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz (max SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 FMA peak: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
PROFILES = os.path.join(ROOT, "profiles")
# bf16 dense tensor rate measured on the GB300s (burst; the M2L stage is
# timed on its own), the denominator of the tensor-core M2L
BF16_FALLBACK_TFLOPS = 1900.0


def bf16_peak():
    """(TFLOP/s, basis) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured (MEASURED_PEAKS.json, burst)"
    except (OSError, KeyError, ValueError):
        return BF16_FALLBACK_TFLOPS, "fallback"


def tc_slices(pb):
    """bf16 slices of the FP64 tensor-core M2L at box order pb (0: CUDA cores)."""
    kp = (2 * (2 * pb + 1) + 63) // 64 * 64
    return 6 if kp <= 128 else 7 if kp <= 576 else 8 if kp <= 2048 else 0


def m2l_tensor_roofline(lp, m2l_ms):
    """Roofline of the FP64 M2L stage on the tensor cores: per level, the
    algorithmic 8 Q^2 flops of each V entry need S (S + 1) / 2 bf16 slice
    products (S slices per operand), so its time at peak is flops x products /
    bf16 peak; levels too wide for the split run at the FP64 FMA peak."""
    t = lp.export_tree()
    pbl = lp.box_orders().astype(np.int64)
    lev = t["level"].astype(np.int64)
    nv = np.diff(t["off"][1]).astype(np.int64)
    peak, basis = bf16_peak()
    t_roof, alg, rows = 0.0, 0.0, []
    for l in range(len(pbl)):
        n = int(nv[lev == l].sum())
        if n == 0:
            continue
        Q = 2 * int(pbl[l]) + 1
        fl = 8.0 * Q * Q * n
        S = tc_slices(int(pbl[l]))
        prod = S * (S + 1) // 2
        t_roof += fl * prod / (peak * 1e12) if S else fl / (FP64_PEAK_TFLOPS * 1e12)
        alg += fl
        rows.append({"level": l, "Q": Q, "v_entries": n, "slices": S, "products": prod})
    return {"bound": "tensor", "kernel": "m2l (fp64 leg)", "ms_per_launch": m2l_ms,
            "algorithmic_fp64_tflops": alg / (m2l_ms * 1e-3) / 1e12,
            "peak": peak, "peak_basis": basis + "; divided per level by the slice products",
            "roofline_ms": 1e3 * t_roof, "frac": 1e3 * t_roof / m2l_ms, "levels": rows}


def function_text(src, name):
    """Source text of the first definition of function `name` in src: from
    the line that declares it to its matching closing brace."""
    i = 0
    while True:
        i = src.find(name + "(", i)
        if i < 0:
            return None
        j = src.find("{", i)
        k = src.find(";", i)
        if j >= 0 and (k < 0 or j < k):   # a definition, not a call or declaration
            break
        i += len(name)
    depth, e = 0, j
    while e < len(src):
        depth += {"{": 1, "}": -1}.get(src[e], 0)
        e += 1
        if depth == 0:
            break
    return src[src.rfind("\n", 0, i) + 1:e]


def kernel_sha256(spec):
    """sha256 over the definitions named by spec, "file:fn+fn;file:fn" (files
    relative to the repository root), so that an ncu summary stays valid for
    edits elsewhere in those files and goes stale when the kernel changes."""
    import hashlib
    h = hashlib.sha256()
    for part in spec.split(";"):
        path, fns = part.split(":")
        text = open(os.path.join(ROOT, path)).read()
        for fn in fns.split("+"):
            body = function_text(text, fn)
            if body is None:
                return None
            h.update(body.encode())
    return h.hexdigest()


def known_pipe(stage, workload, precision):
    """FP64-pipe utilisation of a stage's kernel (fraction of the FP64
    instruction rate) from a committed ncu summary ("bench-pipe:" lines, keyed
    like the traffic lines); None when absent or stale."""
    import glob
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(path):
            if not line.startswith("bench-pipe:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if (kv.get("stage"), kv.get("workload"), kv.get("precision")) != (stage, workload,
                                                                              precision):
                continue
            try:
                sha = kernel_sha256(kv.get("functions", ""))
            except (OSError, ValueError):
                return None
            if sha is None or sha != kv.get("functions_sha256"):
                return None
            return float(kv["fp64_pipe"]), os.path.relpath(path, ROOT)
    return None


def known_traffic(stage, workload, precision):
    """DRAM bytes per launch of a stage's kernels, from a committed ncu summary
    under profiles/ ("bench-traffic:" lines: stage, workload, precision, bytes,
    and the sha256 of the kernel's source functions when it was captured). None
    when no summary covers the stage or its kernel has changed since."""
    import glob
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        for line in open(path):
            if not line.startswith("bench-traffic:"):
                continue
            kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
            if (kv.get("stage"), kv.get("workload"), kv.get("precision")) != (stage, workload,
                                                                              precision):
                continue
            try:
                sha = kernel_sha256(kv.get("functions", ""))
            except (OSError, ValueError):
                return None
            if sha is None or sha != kv.get("functions_sha256"):
                return None
            return float(kv["bytes_per_launch"]), os.path.relpath(path, ROOT)
    return None


# ---------------------------------------------------------------- helpers
def max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over all ranks (the slowest rank sets the job time)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, ws: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return ws * units_per_rank * steps / (max_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# FP64 flops of the base Hankel values H0, H1 of one pair: four polynomials
# of the library's tables by Horner's rule, degree 10 on the FP64 path and 8 on
# the mixed one (the logarithm below x = 2 is not charged), and of one step of
# the upward Hankel recurrence (a real-scaled complex step, 6 flops).
HANKEL01_FLOPS = {False: 4 * 10 * 2, True: 4 * 8 * 2}
REC_STEP_FLOPS = 6


def flop_model(lp, stats, p, has_S, has_D, assoc, fmm, mixed=False, active_frac=1.0):
    """Algorithmic flops per kernel class as (FP64, FP32) pairs: complex
    multiply-add = 8 flops; special-function values as stated above. P = 2p+1
    QBX terms; a box on tree level l carries Q_l = 2 pb_l + 1 terms (per-level
    orders), and every translation is charged with the orders of its boxes. In
    mixed precision M2M, M2L, L2L and the P2QBXL accumulation are FP32.
    active_frac scales the centre stages to the centres whose coefficients are
    formed (those some target uses)."""
    P = 2 * p + 1
    lay = (1 if has_S else 0) + (1 if has_D else 0)
    acc = (18 * P if has_S else 0) + (10 * P if has_D else 0)
    pairs = stats["p2qbxl_pairs"] * active_frac
    base = pairs * (HANKEL01_FLOPS[mixed] + REC_STEP_FLOPS * p)
    f = {}
    f["p2qbxl"] = (base, pairs * acc) if mixed else (base + pairs * acc, 0.0)
    # P2P evaluates only the Hankel functions its layers read (H0 for S, H1 for D)
    f["p2p"] = (stats["p2p_pairs"] * (HANKEL01_FLOPS[False] * lay / 2 + 8 * lay), 0.0)
    f["qbxl2p"] = (stats["n_qbx_targets"] * 16 * P, 0.0)
    if not fmm:
        return f
    t = lp.export_tree()
    pbl = lp.box_orders().astype(np.int64)
    lev = t["level"].astype(np.int64)
    nb = lev.size
    Qb = 2 * pbl[lev] + 1
    child = t["child"]
    rng = t["range"].astype(np.int64)
    nsrc = rng[:, 0, 1] - rng[:, 0, 0]
    nctr = rng[:, 1, 1] - rng[:, 1, 0]
    # direct (non-QBX) targets per box, from the sorted target order
    direct = (assoc[t["perm_tgt"][:lp.n_targets]] < 0).astype(np.int64)
    cdir = np.concatenate([[0], np.cumsum(direct)])
    ndir = cdir[rng[:, 2, 1]] - cdir[rng[:, 2, 0]]
    leaf = np.all(child < 0, axis=1)
    info = t["info"]
    base = np.concatenate([[0], np.cumsum(info[2:6])]).astype(np.int64)
    def entries(i):  # (box, entry) pairs of list i in U, V, W, X order
        cnt = np.diff(t["off"][i]).astype(np.int64)
        own = np.repeat(np.arange(nb), cnt)
        return own, t["idx"][base[i]:base[i] + cnt.sum()].astype(np.int64)
    vb, _ = entries(1)
    tr = lambda v: (0.0, float(v)) if mixed else (float(v), 0.0)  # FP32 translations in mixed
    f["m2l"] = tr(8 * np.sum(Qb[vb] ** 2))
    parent = np.full(nb, -1, np.int64)
    for q in range(4):
        has = child[:, q] >= 0
        parent[child[has, q]] = np.nonzero(has)[0]
    mm = (lev >= 3) & (parent >= 0)
    f["m2m"] = f["l2l"] = tr(8 * np.sum(Qb[mm] * Qb[parent[mm]]))
    # P2M: one FP64 Miller row per source (about pb + 8 orders, 6 flops each);
    # the sums over the sources, 8 flops per layer and coefficient, are FP64 on
    # the FP64 path and FP32 (with 8 more for the compensation) in mixed precision
    srcQ = np.sum((nsrc * Qb)[leaf & (lev >= 2)])
    f["p2m"] = ((3.0 * srcQ, 16.0 * lay * srcQ) if mixed else (16.0 * lay * srcQ, 0.0))
    xb, xc = entries(3)
    f["p2l"] = (16.0 * lay * np.sum(Qb[xb] * nsrc[xc]), 0.0)
    wb, wc = entries(2)
    wq = np.bincount(wb, weights=Qb[wc], minlength=nb)
    # M2QBXL runs for the (centre, W box) pairs whose box is far enough from the
    # centre's disk (stats m2qbxl_pairs; the others are P2QBXL pairs), charged at
    # the mean box order over the W lists of the centres' leaves
    w_all = float(np.sum((nctr * (wq > 0) * np.diff(t["off"][2]))[leaf]))
    w_q = float(np.sum((nctr * wq)[leaf]))
    mq = stats["m2qbxl_pairs"] * active_frac * (w_q / w_all if w_all else 0.0)
    lq = np.sum((nctr * Qb)[leaf]) * active_frac
    # M2P: per (direct target, W box) pair the Hankel recurrence (6 FP64 flops
    # per order, about Q/2 orders) and a complex product-sum per coefficient,
    # FP64 on the FP64 path, FP32 with compensation (16 flops) in mixed
    nw = np.bincount(wb, minlength=nb).astype(np.int64)
    w_pairs = float(np.sum((ndir * nw)[leaf]))
    w_coef = float(np.sum((ndir * wq)[leaf]))
    if mixed:
        # M2QBXL / L2QBXL: products on split FP32 factors (about 16 flops per
        # term with the scaling and compensation), recurrences in FP64
        f["m2qbxl"] = (3.0 * mq, 16.0 * P * mq)
        f["m2p"] = (HANKEL01_FLOPS[True] * w_pairs + 3.0 * w_coef, 16.0 * w_coef)
        f["l2qbxl"] = (0.0, 16.0 * P * lq)
    else:
        f["m2qbxl"] = (8.0 * P * mq, 0.0)
        f["m2p"] = (16.0 * w_coef, 0.0)
        f["l2qbxl"] = (8.0 * P * lq, 0.0)
    # L2P: per order Miller's step (6 flops) and Clenshaw's two complex steps
    # (16 flops), for the two coefficients of orders +-m: 11 per coefficient
    f["l2p"] = (11.0 * np.sum((ndir * Qb)[leaf]), 0.0)
    return f


# ---------------------------------------------------------------- our arm
def timed_steps(step, steps, warmup, stream, flush, ws, dev, lp):
    """Device time of `steps` calls of step() (after `warmup` untimed ones), L2
    flushed before each, CUDA events on the launching stream; max over ranks."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    launches = 0
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        launches += lp.stats()["launches"]
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
    return total_ms, launches


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_ours(args, w, ws, rank, local):
    import torch
    from paper_1602_05301_gb300 import qbx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = w["geom"]
    fmm = args.mode == "fmm"
    mode = qbx.QBX_FMM if fmm else qbx.QBX_DIRECT
    prec = qbx.QBX_MIXED if args.precision == "mixed" else qbx.QBX_FP64
    lp = qbx.LayerPotential(g.as_dict(), w["p"], sides=w["sides"])
    t0 = time.perf_counter()
    assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"], mode=mode,
                     p_fmm=w["p_fmm"], p_add=-1, n_max=args.n_max, eps_assoc=w["eps_assoc"])
    tree_s = time.perf_counter() - t0
    n_t = lp.n_targets
    sS = torch.from_numpy(np.ascontiguousarray(w["sigma_S"])).to(dev) if w["sigma_S"] is not None else None
    sD = torch.from_numpy(np.ascontiguousarray(w["sigma_D"])).to(dev) if w["sigma_D"] is not None else None
    out = torch.empty(n_t, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def stepper(handle, pr, o):
        return lambda: handle.eval(sigma_S=sS, sigma_D=sD, cS=w["cS"], cD=w["cD"], out=o,
                                   precision=pr, stream=sp)

    with ClockSampler(local) as clk:
        total_ms, launches = timed_steps(stepper(lp, prec, out), args.steps, args.warmup, stream,
                                         flush, ws, dev, lp)
    value = job_throughput(n_t, ws, args.steps, total_ms)
    stats = lp.stats()
    if args.only_headline:   # profiling runs: the timed evaluations and nothing else
        lp.close()
        return dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                    warmup=args.warmup, ms_per_step=total_ms / args.steps,
                    higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f64" if prec == qbx.QBX_FP64 else "f32+f64", data="synthetic",
                    config={"workload": WORKLOADS[args.config] % w["name"],
                            "precision": args.precision}, gpu_launches=launches,
                    clocks=clk.summary())
    u_main = out.cpu().numpy()

    # the other precision on the same plan and inputs: speed and the stated error
    other = qbx.QBX_FP64 if prec == qbx.QBX_MIXED else qbx.QBX_MIXED
    out2 = torch.empty_like(out)
    ms2, _ = timed_steps(stepper(lp, other, out2), args.steps, args.warmup, stream, flush, ws,
                         dev, lp)
    u_other = out2.cpu().numpy()
    # per-stage times of the other precision too (the FP64 leg's tensor-core M2L)
    lp.set_timing(True)
    per_other = {}
    for _ in range(3):
        flush.zero_()
        stepper(lp, other, out2)()
        for kname, ms in lp.stage_times().items():
            per_other.setdefault(kname, []).append(ms)
    lp.set_timing(False)
    per_other = {k: statistics.median(v) for k, v in per_other.items() if max(v) > 0}
    u64, u32 = (u_other, u_main) if prec == qbx.QBX_MIXED else (u_main, u_other)
    err_mixed = rel_l2(u32, u64)
    comparison = {"fp64" if other == qbx.QBX_FP64 else "mixed": {
        "value": job_throughput(n_t, ws, args.steps, ms2), "ms_per_step": ms2 / args.steps,
        "per_kernel_ms": per_other}}

    # speedup at equal accuracy: both precisions over box orders p_fmm + p_add
    # from 8 up to the workload's own; at each tolerance, the fastest plan of each
    # precision whose error against the workload's full-order FP64 result is
    # within it
    eq = None
    if fmm and not args.no_equal_accuracy:
        eq_rows = []
        ks = max(3, args.steps // 4)
        for pf, pa in [(q, 0) for q in (8, 12, 16, 20, 24, 28, 32)] + [(w["p_fmm"], -1)]:
            lq = qbx.LayerPotential(g.as_dict(), w["p"], sides=w["sides"])
            lq.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"], mode=mode,
                     p_fmm=pf, p_add=pa, n_max=args.n_max, eps_assoc=w["eps_assoc"])
            for pr, name in ((qbx.QBX_FP64, "fp64"), (qbx.QBX_MIXED, "mixed")):
                oq = torch.empty_like(out)
                msq, _ = timed_steps(stepper(lq, pr, oq), ks, 2, stream, flush, ws, dev, lq)
                eq_rows.append({"precision": name, "p_fmm": pf, "p_add": pa,
                                "p_box_finest": int(lq.stats()["p_box"]),
                                "rel_err_vs_fp64": rel_l2(oq.cpu().numpy(), u64),
                                "value": job_throughput(n_t, ws, ks, msq)})
            lq.close()
        at = {}
        for tol in (1e-6, 1e-8, 1e-10):
            best = {}
            for name in ("fp64", "mixed"):
                ok = [r for r in eq_rows if r["precision"] == name and r["rel_err_vs_fp64"] <= tol]
                best[name] = max(ok, key=lambda r: r["value"]) if ok else None
            at["%g" % tol] = {
                "fp64": best["fp64"], "mixed": best["mixed"],
                "speedup_mixed_over_fp64": (best["mixed"]["value"] / best["fp64"]["value"])
                if best["fp64"] and best["mixed"] else None}
        eq = {"mixed_rel_err_vs_fp64_at_workload_orders": err_mixed, "at_tolerance": at,
              "sweep": eq_rows}

    # per-kernel device times (events around each kernel class on the eval stream)
    lp.set_timing(True)
    per = {}
    for _ in range(3):
        flush.zero_()
        stepper(lp, prec, out)()
        for kname, ms in lp.stage_times().items():
            per.setdefault(kname, []).append(ms)
    lp.set_timing(False)
    per = {k: statistics.median(v) for k, v in per.items() if max(v) > 0}
    n_used = len(np.unique(assoc[assoc >= 0]))
    active = n_used / max(1, stats["n_centres"]) if fmm else 1.0
    flops = flop_model(lp, stats, w["p"], sS is not None, sD is not None, assoc, fmm,
                       mixed=prec == qbx.QBX_MIXED, active_frac=active)
    dom = max(per, key=per.get) if per else None
    roof = None
    if dom:
        f64, f32 = flops.get(dom, (0.0, 0.0))
        t = per[dom] / 1e3
        # roofline time = FP64 work at the FP64 peak + FP32 work at the FP32 peak;
        # achieved is expressed as the FP64-equivalent rate
        roof_ms = 1e3 * (f64 / (FP64_PEAK_TFLOPS * 1e12) + f32 / (FP32_PEAK_TFLOPS * 1e12))
        fp32_only = f64 == 0.0 and f32 > 0.0
        peak = FP32_PEAK_TFLOPS if fp32_only else FP64_PEAK_TFLOPS
        achieved = (f32 if fp32_only else f64 + f32 * FP64_PEAK_TFLOPS / FP32_PEAK_TFLOPS) / t / 1e12
        fma64, fma32 = qbx.qbx_measure_fma_rates()
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": roof_ms / per[dom],
                "traffic": None, "traffic_source": None,
                "flops64_per_launch": f64, "flops32_per_launch": f32,
                "roofline_ms": roof_ms, "ms_per_launch": per[dom],
                "peak_basis": ("FP32" if fp32_only else "FP64") +
                              " FMA rate derived from unit counts and the 2.070 GHz max clock "
                              "(152 SMs x 2 FP64 / 128 FP32 FMA per clock x 2 flop): 1.259 / "
                              "80.5 TFLOP/s (measured FMA rates in measured_fma_tflops). "
                              "achieved is FP64-equivalent (FP32 flops scaled by the peak "
                              "ratio) unless the kernel is FP32 only",
                "measured_fma_tflops": {"fp64": fma64, "fp32": fma32},
                "centres_formed": n_used if fmm else stats["n_centres"]}
        kt = known_traffic(dom, w["name"], args.precision)
        if kt:
            roof["traffic"], roof["traffic_source"] = kt
        # the flop model is a lower bound (logarithms, square roots and FP32
        # conversions are charged nothing); ncu's FP64-pipe utilisation of the
        # same kernel is the measured bound
        kp = known_pipe(dom, w["name"], args.precision)
        if kp:
            roof["fp64_pipe_utilisation_ncu"], roof["fp64_pipe_source"] = kp
        # the same fraction for every timed stage (flop model over its event time)
        roof["frac_by_stage"] = {
            k: round(1e3 * (flops[k][0] / (FP64_PEAK_TFLOPS * 1e12) +
                            flops[k][1] / (FP32_PEAK_TFLOPS * 1e12)) / per[k], 4)
            for k in per if k in flops and per[k] > 0}

    # the coefficients of every centre (alpha_out on the device): the QBX local
    # expansion formed at all 2 n centres, not only at those some target uses
    all_c = None
    if fmm:
        alpha_dev = torch.empty((lp.n_centres, 2 * w["p"] + 1), dtype=torch.complex128,
                                device=dev)
        out3 = torch.empty_like(out)
        step_all = lambda: lp.eval(sigma_S=sS, sigma_D=sD, cS=w["cS"], cD=w["cD"], out=out3,
                                   alpha_out=alpha_dev, precision=prec, stream=sp)
        ms3, _ = timed_steps(step_all, max(3, args.steps // 4), 2, stream, flush, ws, dev, lp)
        k3 = max(3, args.steps // 4)
        all_c = {"value": job_throughput(n_t, ws, k3, ms3), "unit": UNIT,
                 "ms_per_step": ms3 / k3, "centres_per_s": ws * lp.n_centres * k3 / (ms3 / 1e3),
                 "n_centres": lp.n_centres}
        del alpha_dev

    # end-to-end through the C ABI with pinned host buffers (copies inside the timed region)
    hS = torch.from_numpy(np.ascontiguousarray(w["sigma_S"])).pin_memory() if sS is not None else None
    hD = torch.from_numpy(np.ascontiguousarray(w["sigma_D"])).pin_memory() if sD is not None else None
    hout = torch.empty(n_t, dtype=torch.complex128).pin_memory()
    for _ in range(2):
        lp.eval(sigma_S=hS, sigma_D=hD, cS=w["cS"], cD=w["cD"], out=hout, precision=prec,
                stream=sp)
    torch.cuda.synchronize()
    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        lp.eval(sigma_S=hS, sigma_D=hD, cS=w["cS"], cD=w["cD"], out=hout, precision=prec,
                stream=sp)
        e2e_s.append(time.perf_counter() - a)
    e2e_ms = max_over_ranks(1e3 * sum(e2e_s), ws, dev)
    h2d = 16 * g.n * ((1 if hS is not None else 0) + (1 if hD is not None else 0))
    e2e = {"value": job_throughput(n_t, ws, args.steps, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16 * n_t}
    per64 = per if prec == qbx.QBX_FP64 else per_other
    m2l_tc = m2l_tensor_roofline(lp, per64["m2l"]) if fmm and "m2l" in per64 else None
    res = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
               warmup=args.warmup, ms_per_step=total_ms / args.steps, higher_is_better=True,
               scaling="weak", vs_baseline=None,
               dtype="f64" if prec == qbx.QBX_FP64 else "f32+f64",
               data="synthetic",
               rel_err_mixed_vs_fp64=err_mixed,
               config={"workload": WORKLOADS[args.config] % w["name"],
                       "mode": args.mode, "precision": args.precision, "n_targets": n_t,
                       "n_qbx_targets": stats["n_qbx_targets"],
                       "box_orders": [int(x) for x in lp.box_orders()] if fmm else None,
                       "n_boxes": stats["n_boxes"], "tree_build_s": tree_s,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if ws > 1 else "single"},
               roofline=roof, m2l_tensor_roofline=m2l_tc, per_kernel_ms=per,
               gpu_launches=launches,
               clocks=clk.summary(), e2e=e2e, equal_accuracy=eq, all_centres=all_c,
               **comparison)
    lp.close()
    return res


def run_batch(args, w, ws, rank, local):
    """The 256-curve batch: one LayerPotential per curve with its plan chosen by
    qbx_autotune, all evaluated by one qbx_batch_eval (one CUDA graph)."""
    import torch
    from paper_1602_05301_gb300 import qbx

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g = w["geom"]
    noff = g.node_offset()
    prec = qbx.QBX_MIXED if args.precision == "mixed" else qbx.QBX_FP64
    t0 = time.perf_counter()
    probs, chosen = [], []
    for c in range(g.n_curves):
        G = g.as_dict(c)
        lp = qbx.LayerPotential(G, w["p"], sides=1)
        n = G["node_xy"].shape[0]
        _, plan, _ = lp.autotune_tol(G["node_xy"], np.arange(n), np.ones(n, np.int8),
                                     p_fmm=w["p_fmm"], tol=1e-6 if args.precision == "mixed"
                                     else 1e-10, precision=prec, reps=2)
        probs.append(lp)
        chosen.append(plan)
    plan_s = time.perf_counter() - t0
    b = qbx.Batch(probs, n_streams=16)
    sS = torch.from_numpy(np.ascontiguousarray(w["sigma_S"])).to(dev)
    sD = torch.from_numpy(np.ascontiguousarray(w["sigma_D"])).to(dev)
    out = torch.empty(b.n_targets, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    class _L:  # launches are not counted per handle inside the graph
        @staticmethod
        def stats():
            return {"launches": 0}

    step = lambda: b.eval(sigma_S=sS, sigma_D=sD, cS=1.0, cD=1.0, out=out, precision=prec,
                          stream=stream.cuda_stream)
    with ClockSampler(local) as clk:
        total_ms, _ = timed_steps(step, args.steps, args.warmup, stream, flush, ws, dev, _L)
    n_t = b.n_targets
    value = job_throughput(n_t, ws, args.steps, total_ms)
    # e2e: host densities and results (the batch stages them through its buffers)
    hS, hD = np.ascontiguousarray(w["sigma_S"]), np.ascontiguousarray(w["sigma_D"])
    hout = np.empty(n_t, np.complex128)
    b.eval(sigma_S=hS, sigma_D=hD, cS=1.0, cD=1.0, out=hout, precision=prec)
    e2e_s = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        a = time.perf_counter()
        b.eval(sigma_S=hS, sigma_D=hD, cS=1.0, cD=1.0, out=hout, precision=prec)
        e2e_s.append(time.perf_counter() - a)
    e2e_ms = max_over_ranks(1e3 * sum(e2e_s), ws, dev)
    res = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
               warmup=args.warmup, ms_per_step=total_ms / args.steps, higher_is_better=True,
               scaling="weak", vs_baseline=None,
               dtype="f64" if prec == qbx.QBX_FP64 else "f32+f64", data="synthetic",
               config={"workload": WORKLOADS[4] % w["name"], "precision": args.precision,
                       "n_curves": g.n_curves, "n_sources": int(g.n), "n_targets": n_t,
                       "plans": {"direct": sum(c["mode"] == 0 for c in chosen),
                                 "fmm": sum(c["mode"] == 1 for c in chosen),
                                 "fmm_n_max": sorted(set(c["n_max"] for c in chosen
                                                         if c["mode"] == 1)),
                                 "fmm_p_fmm": sorted(set(c["p_fmm"] for c in chosen
                                                         if c["mode"] == 1)),
                                 "cuda_core_m2l": sum(c["engine"] == 2 for c in chosen),
                                 "l2qbxl_g": sorted(set(c["g"] for c in chosen))},
                       "autotuner": "qbx_autotune_tol, tolerance 1e-6 (mixed) / 1e-10 (fp64) "
                                    "against the most accurate plan",
                       "plan_and_autotune_s": plan_s,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if ws > 1 else "single"},
               roofline=None, gpu_launches=None, clocks=clk.summary(),
               e2e={"value": job_throughput(n_t, ws, args.steps, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": 32 * int(g.n), "d2h_bytes_per_step": 16 * n_t})
    b.close()
    for lp in probs:
        lp.close()
    return res


# ---------------------------------------------------------------- oracle (CPU) timing
def oracle_sample(w, assoc, budget_s=12.0, seed=0, max_src_pairs=None):
    """Times the FP64 oracle on a stratified sample of targets (the workload's
    direct/QBX mix; a QBX target costs its centre's coefficients plus the
    evaluation, a direct target its Gauss sum). Every sampled target is summed
    over every m-th source, m = 1 unless a single target over all sources would
    take much of the budget (max_src_pairs caps the source count per target);
    the work per target is linear in the sources, so its time is scaled by m.
    Returns (targets/s, threads, description)."""
    from oracle import oracle
    g = w["geom"]
    rng = np.random.default_rng(seed)
    qbx_t = np.nonzero(assoc >= 0)[0]
    dir_t = np.nonzero(assoc < 0)[0]
    frac_q = qbx_t.size / max(1, assoc.size)
    m = 1 if not max_src_pairs else max(1, -(-g.n // max_src_pairs))
    sl = slice(None, None, m)
    sxy, snr, sw = g.node_xy[sl], g.normal_xy[sl], g.weight[sl]
    sS = None if w["sigma_S"] is None else w["sigma_S"][sl]
    sD = None if w["sigma_D"] is None else w["sigma_D"][sl]
    cxy, _ = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, w["sides"])
    k = g.k[0]
    n_q = 1 if g.n > 100000 else 4
    n_d = 4 if g.n > 100000 else 32
    elapsed, t_q, t_d, nq_done, nd_done = 0.0, 0.0, 0.0, 0, 0
    while elapsed < budget_s:
        if qbx_t.size:
            tq = rng.choice(qbx_t, min(n_q, qbx_t.size), replace=False)
            a = time.perf_counter()
            al = oracle.qbx_coefficients(sxy, snr, sw, k, cxy[assoc[tq]], w["p"], sS, sD,
                                         w["cS"], w["cD"])
            oracle.qbx_evaluate(w["tgt_xy"][tq], np.arange(tq.size, dtype=np.int32),
                                cxy[assoc[tq]], al, w["p"], k)
            dt = time.perf_counter() - a
            t_q += dt * m
            nq_done += tq.size
            elapsed += dt
        if dir_t.size:
            td = rng.choice(dir_t, min(n_d, dir_t.size), replace=False)
            a = time.perf_counter()
            oracle.direct_potential(sxy, snr, sw, k, w["tgt_xy"][td], sS, sD, w["cS"], w["cD"])
            dt = time.perf_counter() - a
            t_d += dt * m
            nd_done += td.size
            elapsed += dt
    per_q = t_q / max(1, nq_done)
    per_d = t_d / max(1, nd_done)
    per_t = frac_q * per_q + (1 - frac_q) * per_d
    desc = ("%d QBX + %d direct targets (of %d; QBX fraction %.4f), each summed over every "
            "%s source of %d (time scaled by %d, the work being linear in the sources), %.1f s "
            "of oracle time, extrapolated to the full target mix"
            % (nq_done, nd_done, assoc.size, frac_q, "%d-th" % m if m > 1 else "", g.n, m,
               elapsed))
    return 1.0 / per_t, oracle.num_threads(), desc


def gpu_assoc_free(w):
    """Association for the CPU-only reference arm: the oracle's own brute force,
    run on the targets that a k-d tree finds within the largest association
    radius of some centre (the others are direct: the workloads have no target
    within h/4 of a panel outside every disk, which the GPU plan checks)."""
    from oracle import oracle
    from scipy.spatial import cKDTree
    g = w["geom"]
    cxy, crad = oracle.centres(g.node_xy, g.normal_xy, g.panel_of_node, g.panel_h, w["sides"])
    r_max = (1.0 + w["eps_assoc"]) * crad.max() * (1.0 + 1e-9)
    d, _ = cKDTree(cxy).query(w["tgt_xy"], k=1, distance_upper_bound=r_max)
    cand = np.isfinite(d)
    if w["on_surface_node"] is not None:
        cand |= w["on_surface_node"] >= 0
    idx = np.nonzero(cand)[0]
    cot = np.full(w["tgt_xy"].shape[0], -1, np.int32)
    osn = None if w["on_surface_node"] is None else w["on_surface_node"][idx]
    oss = None if w["on_surface_side"] is None else w["on_surface_side"][idx]
    c, _ = oracle.associate(w["tgt_xy"][idx], g.node_xy, g.panel_of_node, g.panel_h, cxy, crad,
                            w["eps_assoc"], osn, oss)
    cot[idx] = c
    return cot


def run_reference(args, w):
    from oracle import oracle
    oracle.build()
    assoc = gpu_assoc_free(w)
    vals = []
    desc = ""
    per_step_budget = max(2.0, min(12.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        v, cores, desc = oracle_sample(w, assoc, budget_s=per_step_budget, seed=i,
                                       max_src_pairs=1 << 18)
        if i >= args.warmup:
            vals.append(v)
    value = float(np.mean(vals))
    return dict(metric=METRIC, value=value, unit=UNIT, n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * w["tgt_xy"].shape[0] / value,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config={"workload": "%s (oracle: direct Global QBX, FP64 CPU)" % w["name"],
                        "mode": "direct", "precision": "fp64"},
                cpu_baseline={"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                              "sample": desc},
                e2e={"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                     "d2h_bytes_per_step": 0})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--mode", default="fmm", choices=["fmm", "direct"])
    ap.add_argument("--n-max", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-equal-accuracy", action="store_true")
    ap.add_argument("--size-scale", type=float, default=1.0,
                    help="shrink the 200-ellipse workload (ellipses, panels and targets "
                         "times this factor) for profiling captures; 1 = the full workload")
    ap.add_argument("--only-headline", action="store_true",
                    help="time the headline evaluations only (for profiler launch lists)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the starfish and batch workloads of the default line")
    ap.add_argument("--config", type=int, default=CONFIG_NUM, choices=[2, 3, 4, 5],
                    help="workload (5: the default line, 200 ellipses; 2, 3: starfish k = 10, "
                         "50; 4: the 256-curve batch)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    from qbx_workloads import make_config
    if args.size_scale != 1.0:
        if args.config != 5 or not 0.0 < args.size_scale <= 1.0:
            ap.error("--size-scale applies to --config 5 with a factor in (0, 1]")
        f = args.size_scale
        w = make_config(5, n_ellipses=max(1, int(round(200 * f))),
                        total_panels=max(64, int(round(65536 * f))),
                        n_uniform=int(round(900_000 * f)), n_near=int(round(100_000 * f)))
        args.no_extras = True
    else:
        w = make_config(args.config)

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, w)), flush=True)
        return
    import torch
    if ws > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1602_05301_gb300 import build as b
    if rank == 0:
        b.build()
    if ws > 1:
        torch.distributed.barrier()
    res = run_batch(args, w, ws, rank, local) if args.config == 4 else run_ours(args, w, ws, rank, local)
    if args.only_headline:
        args.no_extras = args.no_cpu_baseline = True
    if rank == 0 and ws == 1 and not args.no_extras and args.config == CONFIG_NUM:
        # the other workloads of the same metric, as extra keys of the line
        res["extra_workloads"] = {}
        for num in (2, 4):
            a2 = argparse.Namespace(**vars(args))
            a2.config, a2.no_equal_accuracy = num, True
            a2.steps = max(3, args.steps // 2)
            w2 = make_config(num)
            r2 = run_batch(a2, w2, ws, rank, local) if num == 4 else run_ours(a2, w2, ws, rank, local)
            keep = ("value", "unit", "ms_per_step", "dtype", "rel_err_mixed_vs_fp64", "config",
                    "fp64", "roofline", "per_kernel_ms", "e2e", "clocks", "gpu_launches",
                    "all_centres")
            res["extra_workloads"][w2["name"]] = {k: r2[k] for k in keep if k in r2}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.config != 4:
        from paper_1602_05301_gb300 import qbx
        from oracle import oracle
        lp = qbx.LayerPotential(w["geom"].as_dict(), w["p"], sides=w["sides"])
        assoc = lp.build(w["tgt_xy"], w["on_surface_node"], w["on_surface_side"])
        lp.close()
        v, cores, desc = oracle_sample(w, assoc, budget_s=10.0, max_src_pairs=1 << 18)
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": desc}
        n_all = oracle.num_threads()
        oracle.set_num_threads(1)
        v1, cores1, desc1 = oracle_sample(w, assoc, budget_s=10.0, seed=1, max_src_pairs=1 << 14)
        oracle.set_num_threads(n_all)
        res["cpu_baseline_1core"] = {"value": v1, "unit": UNIT, "cores": cores1, "kind": "oracle",
                                     "sample": desc1}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
