"""Benchmark of the regularised TE domain-integral-equation solver on one GB300.

Workload (N = 1): the 512 x 512 core-shell scatterer (plasma-like core eps -2+0.1i,
radius 1.5; dielectric shell eps 20+0.5i to radius 2.5; side 8 wavelengths,
h = 1/64; 524288 complex unknowns), unit TE plane wave at psi = 0.

Step = one full solve of A_R A P^-1 v = A_R b to relative residual 1e-6:
restarted GMRES(30), deflation of the 20 largest-magnitude eigenvalues, complex64
products inside each cycle and an FP64 restart residual, FP64 Arnoldi and least
squares.  The operator set-up (Green's-tensor spectrum) and the deflation build
happen before the timed region; the build is timed separately (as the paper times
its eigs run separately).

value = regularised DIE products (A_R A applications) per second over the timed
solves.  Extra keys report the solve time against plain FP64 GMRES(30) on A on the
same GPU, products per second of the bare regularised product, the roofline of the
dominant kernel and the CPU oracle's throughput on this machine's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 512
RESTART = 30
R_DEFL = 20
TOL = 1e-6
METRIC = "regularized DIE matvecs/s + GMRES solve time to 1e-6 residual vs plain FP64, %HBM roofline"
UNIT = "regularized matvecs/s"
WORKLOAD = "core-shell 512x512 (eps -2+0.1i core R1.5, 20+0.5i shell R2.5, side 8), A_R A P^-1 GMRES(30) r=20 tol 1e-6"
L2_NOTE = "working set > L2: Krylov basis 31 x 8.4 MB + deflation basis 20 x 8.4 MB per solve"


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(p, budget_s: float = 12.0, max_products: int = 200):
    """Regularised products per second of the CPU oracle (scipy.fft FP64, all cores)."""
    from oracle import fftmv
    from paper_1104_4263_gb300 import workloads as W
    cores = os.cpu_count() or 1
    op = fftmv.FFTOperator(p.eps_r, p.h, workers=cores)
    x = W.random_vector(W.rng_for(2, 7), p.n1, p.n2)
    op.apply_regularized(x)
    t0 = time.perf_counter()
    k = 0
    while k < max_products and time.perf_counter() - t0 < budget_s:
        x = op.apply_regularized(x)
        x /= abs(x).max()
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{k} regularised FP64 FFT products (scipy.fft, workers={cores}) of the {p.n1}x{p.n2} core-shell operator"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    from paper_1104_4263_gb300 import workloads as W
    from oracle import fftmv
    p = W.config2(N_GRID)
    cores = os.cpu_count() or 1
    op = fftmv.FFTOperator(p.eps_r, p.h, workers=cores)
    x = W.random_vector(W.rng_for(2, 8), p.n1, p.n2)
    per_step = 4
    for _ in range(args.warmup):
        for _ in range(per_step):
            x = op.apply_regularized(x)
            x /= abs(x).max()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            x = op.apply_regularized(x)
            x /= abs(x).max()
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " [CPU oracle: regularised products only]"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} regularised FP64 FFT products per step (scipy.fft, workers={cores})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--max-iters", type=int, default=20000)
    ap.add_argument("--plain-seconds", type=float, default=45.0, help="time cap of the plain FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    from paper_1104_4263_gb300 import die, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        if pg is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    p = W.config2(args.n)
    psi = 2 * math.pi * rank / 8                       # replicas: one incidence angle per rank
    t0 = time.perf_counter()
    op = die.Operator(p.eps_r, p.h)
    t_setup = time.perf_counter() - t0
    b = op.plane_wave(psi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D = die.Deflation(op, R_DEFL, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    torch.cuda.synchronize()
    t_defl = time.perf_counter() - t0

    def solve(x=None):
        return op.solve(b, x, restart=RESTART, tol=TOL, max_iters=args.max_iters, regularized=True,
                        inner=die.DIE_FP32_INNER, deflation=D)

    for _ in range(args.warmup):
        x, rep = solve()
    barrier()
    reps = []
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, die.KernelTimer() as kt:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            x, rep = solve()
            reps.append(rep)
        ev1.record(stream)
        barrier()
    dt = ev0.elapsed_time(ev1) / 1e3
    dt = max_over_ranks(dt)
    products = sum(r["iters"] for r in reps)
    products_all = max_over_ranks(products) * world if world > 1 else products
    value = products_all / dt
    solve_s = dt / args.steps

    # end to end through the public API: pinned host b -> device, solve, x -> pinned host
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(b)
    e2e_reps = []
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        db.copy_(hb, non_blocking=True)
        xd, r2 = op.solve(db, restart=RESTART, tol=TOL, max_iters=args.max_iters, regularized=True,
                          inner=die.DIE_FP32_INNER, deflation=D)
        hx.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_reps.append(r2)
    e2e_dt = max_over_ranks(time.perf_counter() - t0)
    e2e_products = sum(r["iters"] for r in e2e_reps) * world
    nbytes = b.numel() * b.element_size()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * solve_s, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c64 products / f64 Krylov",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [p.n1, p.n2], "unknowns": 2 * p.N, "restart": RESTART,
                      "deflated": D.r, "tol": TOL, "parallelism": f"replicas x{world}", "l2": L2_NOTE}}
    if rank != 0:
        if pg is not None:
            pg.barrier()
            pg.destroy_process_group()
        return 0
    out["e2e"] = {"value": e2e_products / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                  "d2h_bytes_per_step": nbytes}
    launches = sum(v["launches"] for v in kt.result.values())
    out["gpu_launches"] = launches
    out["gmres"] = {"solve_s": solve_s, "iters": reps[-1]["iters"], "cycles": reps[-1]["cycles"],
                    "n_reorth": reps[-1]["n_reorth"],
                    "rel_res_solved": reps[-1]["rel_res_solved"], "rel_res_orig": reps[-1]["rel_res_orig"],
                    "status": reps[-1]["status"], "deflation_build_s": t_defl, "operator_setup_s": t_setup,
                    "deflation_converged": D.converged}
    out["kernels"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in kt.result.items()}
    out["clocks"] = clk.summary()

    # dominant kernel and its roofline
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64_peak = 152 * 4 * 2070e6 / 1e12         # TFLOP/s: 152 SMs x 2 DFMA/clk x 2.07 GHz
    top = max(kt.result.items(), key=lambda kv: kv[1]["ms"])
    out["roofline"] = roofline(top[0], top[1], p, op, reps, kt.result, hbm_peak, fp64_peak, peaks)

    # bare regularised product rate (complex64 and FP64), L2 flushed between launches
    out["matvec"] = matvec_rates(op, p, die, torch)

    if not args.no_plain:
        out["plain_fp64"] = plain_fp64(op, b, args.plain_seconds, solve_s)
    if not args.no_cpu:
        try:
            out["cpu_baseline"] = cpu_oracle_rate(p)
        except Exception as e:  # noqa: BLE001
            out["cpu_baseline"] = {"unavailable": str(e)}
    print(json.dumps(out))
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def roofline(name, stat, p, op, reps, allk, hbm_peak, fp64_peak, peaks):
    """Algorithmic bytes (or flops) per launch / average launch time for kernel class `name`."""
    N = p.N
    M1, M2 = op.M1, op.M2
    avg_s = stat["ms"] / stat["launches"] / 1e3
    res = {"kernel": name, "launches": stat["launches"], "avg_us": avg_s * 1e6}
    mean_nv = None
    if name == "cols_green":
        Q = (M1 // 2 + 1) * (M2 // 2 + 1)
        bytes_ = 2 * (2 * M1 * p.n2 * 8) + 3 * Q * 8          # read + write W (c64) + quarter spectra
        res.update({"bound": "hbm", "achieved": bytes_ / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "algorithmic_bytes": bytes_})
    elif name in ("rows_fwd", "rows_inv", "rows_inv_fwd"):
        per = {"rows_fwd": (2 * N * 16 + N * 8) + 2 * M1 * p.n2 * 8,
               "rows_inv": 2 * M1 * p.n2 * 8 + 2 * N * 8 + 2 * N * 16,
               "rows_inv_fwd": 2 * M1 * p.n2 * 8 + 2 * N * 16 + N * 8 + 2 * N * 8 + 2 * M1 * p.n2 * 8}[name]
        res.update({"bound": "hbm", "achieved": per / avg_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "algorithmic_bytes": per})
    else:
        # FP64 Krylov sweeps: 8 flops per (basis vector, element) per sweep; mean basis size
        iters = sum(r["iters"] for r in reps)
        cycles = sum(r["cycles"] for r in reps)
        m = RESTART
        mean_j = (m + 1) / 2.0
        nvec = {"dots": mean_j + 1, "cgs_update_dots": 2 * mean_j, "cgs_update_norm": mean_j + 1,
                "defl_update": R_DEFL}.get(name, 1)
        flops = 8 * nvec * 2 * N
        res.update({"bound": "alu", "achieved": flops / avg_s / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                    "algorithmic_flops": flops, "note": "FP64 peak = 152 SMs x 2 DFMA/clk x 2.07 GHz"})
        mean_nv = nvec
    res["frac"] = res["achieved"] / res["peak"]
    res["traffic"] = None
    res["peak_source"] = "MEASURED_PEAKS.json" if peaks else "fallback"
    return res


def matvec_rates(op, p, die, torch):
    """Bare regularised products per second (c64 and FP64), L2 flushed before each launch."""
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for prec, dt, name in ((die.DIE_FP32_INNER, torch.complex64, "c64"), (die.DIE_FP64, torch.complex128, "c128")):
        o = op if prec == die.DIE_FP64 else die.Operator(p.eps_r, p.h, prec=prec)
        x = torch.randn(2, p.n2, p.n1, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            o.apply_regularized(x, y)
        reps = 20
        ms = 0.0
        s = torch.cuda.current_stream()
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            o.apply_regularized(x, y)
            e1.record(s)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        out[name] = {"regularized_per_s": reps / (ms / 1e3), "us_per_product": 1e3 * ms / reps,
                     "l2": "flushed (256 MB write) before each product"}
    return out


def plain_fp64(op, b, cap_s, solve_s):
    """Plain FP64 GMRES(30) on A u = b, capped in wall time."""
    import torch
    x = None
    t0 = time.perf_counter()
    total_iters, status, rel = 0, None, None
    chunk = 600
    while time.perf_counter() - t0 < cap_s:
        x, rep = op.solve(b, x, restart=RESTART, tol=TOL, max_iters=chunk)
        total_iters += rep["iters"]
        rel = rep["rel_res_solved"]
        status = rep["status"]
        if rep["converged"]:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    res = {"solve_s": dt, "iters": total_iters, "rel_res": rel, "converged": status == "DIE_OK"}
    if status == "DIE_OK":
        res["speedup"] = dt / solve_s
    else:
        res["speedup_lower_bound"] = dt / solve_s
        res["note"] = f"plain FP64 GMRES({RESTART}) did not reach {TOL} within {cap_s:.0f} s"
    return res


if __name__ == "__main__":
    sys.exit(main())
