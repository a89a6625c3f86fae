"""Benchmark of the regularised TE domain-integral-equation solver on GB300.

Workload (N = 1): the 512 x 512 core-shell scatterer -- plasma-like core eps -2+0.1i,
radius 1.5; dielectric shell eps 20+0.5i to radius 2.5; side 8 wavelengths, h = 1/64;
524288 complex unknowns -- lit by a unit TE plane wave.

Timed step: one call of gmres_solve on A_R A P^-1 v = A_R b from x0 = 0 -- GMRES(30),
deflation of the 20 largest-magnitude eigenvalues of A_R A, complex64 products and
complex64 P^-1 inside each cycle, FP64 Arnoldi / least squares / restart residual --
for a budget of 1500 Arnoldi steps (50 restart cycles).  With these settings the
solve does not reach 1e-6 on this object (it stalls near 1e-1 after 2e4 steps), so
the step is a fixed amount of the solver's work and the residual it reaches is
reported.  Operator set-up and the deflation build (Krylov-Schur, tol 1e-4) run
before the timed region; the build is timed separately.

value = regularised DIE products (applications of A_R A) per second over the timed
steps.  Other keys: the same through the public API with host buffers (e2e); plain
FP64 GMRES(30) on A for the same step budget; time-to-tolerance against plain FP64 on
problems that converge (the paper's Section 4 test squares with the Table 2
fair-memory settings, and the 32^2 cylinder); the bare regularised product rate, alone
and batched over 8 right-hand sides (matvec); 4 and 8 incidence angles solved one after
another and concurrently (batch_solve); Arnoldi steps per second on the batched
workload's grid sizes, one solve and 8 concurrent angles, each with cycles launched
kernel by kernel and as CUDA graphs (small_grids); 64 systems of 16 mixed-size
scatterers solved one after another and together (many_systems); the roofline of the
dominant kernel; the CPU oracle on this machine's cores.

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
STEP_ITERS = 1500
PROF_STEPS = 2
METRIC = "regularized DIE matvecs/s + GMRES solve time to 1e-6 residual vs plain FP64, %HBM roofline"
UNIT = "regularized matvecs/s"
WORKLOAD = ("core-shell 512x512 (eps -2+0.1i core R1.5, 20+0.5i shell R2.5, side 8): A_R A P^-1, GMRES(30), r=20, "
            "FP32 products + FP64 Krylov, 1500 Arnoldi steps per step")
L2_NOTE = "working set > L2 (Krylov basis 31 x 8.4 MB, deflation basis 20 x 4.2 MB)"
# ncu DRAM bytes (read + write) of one launch of the FP64 projection kernel on this
# workload: 13 basis vectors with their Re - Im planes, and the norm of w, over
# 2N = 524288, from one capture of the committed profile driver (bench.py
# --profile-driver; the kernel is unchanged since).  Its traffic grows with the vectors
# read, so it is scaled to the bench's average launch by the algorithmic bytes.
# DRAM bytes of the five passes of one complex64 regularised product at 512^2 (reads; no
# DRAM writes were counted during the passes: the row spectra stay in L2)
NCU_PRODUCT = {"dram_bytes": (6.315520 + 14.774016 + 14.725632 + 14.769408 + 12.608512) * 1e6, "n": 524288,
               "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:\"k1_fast|k2_fast2|"
                         "k3k1_fast|k3_fast\" -c 5 on bench.py --profile-driver (its first complex64 product)"}
NCU_DOTS = {"dram_bytes": 175.365632e6 + 0.137216e6, "nv": 13, "n": 524288,
            "source": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:proj3 -s 10 -c 3 on "
                      "bench.py --profile-driver (the 13-vector launch; groups of eight vectors)"}


def fp64_peak(die):
    """FP64 peak of this GPU: the library's FMA-chain probe (die_fp64_peak), and the nominal
    SM count x 2 DFMA/clk x max SM clock beside it."""
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    measured = die.fp64_peak_tflops()
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", str(torch.cuda.current_device())], capture_output=True, text=True, timeout=20)
        mhz = float(out.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        pass
    return {"measured_tflops": measured, "sms": props.multi_processor_count,
            "nominal_tflops": props.multi_processor_count * 4 * mhz * 1e6 / 1e12, "max_sm_mhz": mhz}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
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
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_arnoldi_rate(n: int, steps: int, workers: int):
    """Arnoldi steps per second of the oracle's GMRES(30) on the regularised operator A_R A
    of the n x n core-shell workload (scipy.fft FP64 products with `workers` threads,
    modified Gram-Schmidt in numpy): `steps` steps from x0 = 0, after one untimed product.
    One step applies A_R A once, the unit of the GPU line.  The oracle's deflation (ARPACK
    eigs of the 20 largest eigenvalues) is left out: at 512^2 it takes far longer than the
    sample budget."""
    from oracle import fftmv, gmres
    from paper_1104_4263_gb300 import workloads as W
    p = W.config2(n)
    op = fftmv.FFTOperator(p.eps_r, p.h, workers=workers)
    from oracle import dense
    b = dense.plane_wave(p.n1, p.n2, p.h, 0.0)
    bt = op.apply_R(b)
    t0 = time.perf_counter()
    res = gmres.gmres(op.apply_regularized, bt, RESTART, 1e-14, steps)
    dt = time.perf_counter() - t0
    return res.iters / dt, res.iters, dt


def cpu_oracle_rate(n: int = N_GRID, steps_all: int = 40, steps_one: int = 8):
    """The CPU baseline in the GPU line's unit: the oracle's regularised GMRES(30) Arnoldi
    steps per second on all host cores, and on one thread (a child process with the BLAS
    and FFT thread counts set to 1)."""
    cores = os.cpu_count() or 1
    rate, k, dt = oracle_arnoldi_rate(n, steps_all, cores)
    one = None
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
                f"print(json.dumps(bench.oracle_arnoldi_rate({n}, {steps_one}, 1)))")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        v = json.loads(r.stdout.strip().splitlines()[-1])
        one = {"value": v[0], "arnoldi_steps": v[1], "seconds": v[2], "threads": 1}
    except Exception as e:  # noqa: BLE001
        one = {"unavailable": f"{type(e).__name__}: {e}"}
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": (f"{k} Arnoldi steps of the oracle's GMRES({RESTART}) on A_R A of the {n}x{n} core-shell "
                       f"(scipy.fft FP64, workers={cores}; MGS in numpy), {dt:.1f} s; deflation omitted"),
            "one_thread": one}


def reference_arm(args):
    """The CPU oracle on this machine's cores, in the GPU line's unit: Arnoldi steps of the
    oracle's regularised GMRES(30) on the 512^2 core-shell per second (one bounded sample
    of steps per timed step)."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    cores = os.cpu_count() or 1
    per_step = 8
    for _ in range(args.warmup):
        oracle_arnoldi_rate(N_GRID, 2, cores)
    total_steps, total_s = 0, 0.0
    for _ in range(args.steps):
        _, k, dt = oracle_arnoldi_rate(N_GRID, per_step, cores)
        total_steps += k
        total_s += dt
    value = total_steps / total_s
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ("core-shell 512x512: A_R A, GMRES(30) Arnoldi steps of the CPU oracle "
                                "(scipy.fft FP64, MGS; deflation omitted)")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"{per_step} oracle Arnoldi steps per timed step (scipy.fft, workers={cores})"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
    return 0


# ------------------------------------------------------------------ work model per kernel class
def product_bytes(p, op, s, out_s=None, defl_r=0):
    """Algorithmic bytes of one regularised product A_R A (five passes K1 K2 K3K1 K2 K3)
    with element size s: each pass reads its inputs and writes its outputs once; the
    transposed row spectra W (2 x M1 x n2) go through HBM between passes, the Green
    spectra are the quarter planes (3 x Q1 x Q2).  defl_r > 0: the first row pass also
    applies the deflation (reads r complex64 basis vectors and the FP64 Arnoldi vector,
    writes it back normalised and stores z)."""
    N, n = p.N, 2 * p.N
    out_s = out_s or s
    Wb = 2 * op.M1 * p.n2 * s
    Q = (op.M1 // 2 + 1) * (op.M2 // 2 + 1)
    k1 = n * s + N * s + Wb
    if defl_r:
        k1 = defl_r * n * 8 + 2 * n * 16 + n * 8 + N * s + Wb
    k2 = 2 * Wb + 3 * Q * s
    k3k1 = Wb + n * s + N * s + n * s + Wb
    k3 = Wb + n * s + n * out_s
    return {"rows_fwd": k1, "cols_green": 2 * k2, "rows_inv_fwd": k3k1, "rows_inv": k3}


def work_model(cls, p, op, r, steps_per_cycle, cycles, products, fp64_products):
    """Algorithmic work of all launches of a kernel class in the timed region:
    ('hbm', bytes) or ('alu', FP64 flops).  Products: the deflated complex64 ones inside
    the cycles (complex128 output), and the FP64 restart residuals; each counted at its
    own element size."""
    n = 2 * p.N
    if cls in ("rows_fwd", "cols_green", "rows_inv_fwd", "rows_inv"):
        c64 = product_bytes(p, op, 8, out_s=16, defl_r=r)[cls]
        c128 = product_bytes(p, op, 16)[cls]
        return "hbm", products * c64 + fp64_products * c128
    if cls == "dots32":                     # cf of v_0, once per cycle
        return "hbm", cycles * (r * n * 8 + n * 8)
    if cls == "defl_update":                # FP64 P^-1 in the update of x, once per cycle
        return "hbm", cycles * (r * n * 16 + 2 * n * 16)
    m = steps_per_cycle
    if cls == "dots_bytes":
        # step j: j+1 basis vectors (16 B) and their Re - Im planes (8 B), w read once;
        # per cycle the residual norm and the FP64 deflation projections (r vectors + x)
        per_cycle = sum((j + 1) * 24 + 16 for j in range(m)) + 16 + 16 * r + 16
        return "hbm", cycles * per_cycle * n + 16 * n
    if cls == "dots":
        # step j of a cycle: j+1 projections + the norm of w; per cycle one norm of the
        # residual, one FP64 deflation projection set (r) for the update of x
        per_cycle = sum((j + 1) * 8 + 4 for j in range(m)) + 4 + 8 * r
        return "alu", cycles * per_cycle * n + 4 * n
    if cls == "cgs_update_norm":
        per_cycle = sum((j + 1) * 8 + 4 for j in range(m))
        return "alu", cycles * per_cycle * n
    return None, None


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--step-iters", type=int, default=STEP_ITERS)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 and time-to-tol comparisons")
    ap.add_argument("--single-system", action="store_true",
                    help="skip the sections that solve several systems at once (host threads)")
    ap.add_argument("--profile-driver", action="store_true",
                    help="short fixed run for ncu captures: one complex64 regularised product, then one "
                         "30-step FP32-inner regularised GMRES cycle without and one with deflation (r=20)")
    ap.add_argument("--profile-fno", action="store_true",
                    help="short fixed run for ncu captures of the tensor-core GEMMs: one forward and one backward "
                         "pass of the 128^2 network on a batch of 4")
    ap.add_argument("--paper-table2", action="store_true",
                    help="the four systems of Table 2 on the three Section 4 squares (one JSON line)")
    ap.add_argument("--paper-table1", action="store_true",
                    help="Table 1: the TM systems A and A P^-1 on the three Section 4 squares (one JSON line)")
    ap.add_argument("--paper-sweeps", action="store_true",
                    help="Section 5 restart sweeps (restart r/2, 2r, 10r against r, 3r, 11r) over object size and "
                         "permittivity (one JSON line)")
    ap.add_argument("--paper-sinusoidal", action="store_true",
                    help="Section 5's sinusoidal 4-wavelength object: A with restart 1620 against A_R A P^-1 with "
                         "r = 180 and restart 1440 (one JSON line)")
    ap.add_argument("--config3", action="store_true",
                    help="the batched workload: 64 random scatterers x 8 angles (512 right-hand sides) to 1e-6, "
                         "one after another and concurrently with graph cycles (one JSON line)")
    ap.add_argument("--config5", action="store_true",
                    help="the 2048^2 composite of 400 random cylinders: plain FP64 GMRES(40) and GMRES(80) against "
                         "A_R A P^-1 (r = 40) GMRES(40) in FP64 and FP32-inner, a fixed step budget (one JSON line)")
    ap.add_argument("--budget", type=int, default=1000, help="--config5: Arnoldi steps per solve")
    ap.add_argument("--learned", action="store_true",
                    help="learned preconditioner: solver-generated pairs on 128^2 random fields, training on the "
                         "GPU, flexible GMRES with the network vs the regularised + deflated method on held-out "
                         "fields (one JSON line)")
    ap.add_argument("--pairs", type=int, default=20000, help="--learned: training pairs")
    ap.add_argument("--epochs", type=int, default=8, help="--learned: training epochs")
    ap.add_argument("--held-out", type=int, default=32, help="--learned: held-out fields")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_driver:
        return profile_driver(args)
    if args.profile_fno:
        return profile_fno(args)
    if args.paper_table2:
        return paper_table2(args)
    if args.learned:
        return learned_bench(args)
    if args.paper_table1:
        return paper_table1(args)
    if args.paper_sweeps:
        return paper_sweeps(args)
    if args.paper_sinusoidal:
        return paper_sinusoidal(args)
    if args.config5:
        return config5_budget(args)
    if args.config3:
        import torch

        from paper_1104_4263_gb300 import die, workloads as W
        print(json.dumps({"config3": config3_rates(die, W, torch)}))
        return 0

    import numpy as np
    import torch

    from paper_1104_4263_gb300 import die, replicas, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = W.config2(args.n)
    t0 = time.perf_counter()
    op = die.Operator(p.eps_r, p.h)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    tune = op.autotune(force=True)         # tile height of the complex64 row passes
    tune["seconds"] = time.perf_counter() - t0
    b = op.plane_wave(replicas.angle_for_rank(rank))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D = die.Deflation(op, R_DEFL, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    torch.cuda.synchronize()
    t_defl = time.perf_counter() - t0

    def step(bb=b):
        return op.solve(bb, restart=RESTART, tol=TOL, max_iters=args.step_iters, regularized=True,
                        inner=die.DIE_FP32_INNER, deflation=D, graph=True)

    for _ in range(args.warmup):
        step()
    barrier()
    reps = []
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            reps.append(step()[1])
        ev1.record(stream)
        barrier()
    dt_local = ev0.elapsed_time(ev1) / 1e3
    products_local = sum(r["iters"] for r in reps)
    products, dt = replicas.combine(products_local, dt_local, dist)
    value = products / dt
    # per-kernel times: CUDA events around every library launch, in PROF_STEPS further
    # steps identical to the timed ones (kept out of the timed region: the events add
    # host work per launch)
    prof_reps = []
    with die.KernelTimer() as kt:
        for _ in range(PROF_STEPS):
            prof_reps.append(step()[1])
    prof_products = sum(r["iters"] for r in prof_reps)
    prof_cycles = sum(r["cycles"] for r in prof_reps)

    # end to end through the public API: pinned host b -> device, solve, x -> pinned host
    hb = b.cpu().pin_memory()
    hx = torch.empty_like(hb).pin_memory()
    db = torch.empty_like(b)
    barrier()
    t0 = time.perf_counter()
    e2e_products = 0
    for _ in range(args.steps):
        db.copy_(hb, non_blocking=True)
        xd, r2 = step(db)
        hx.copy_(xd, non_blocking=True)
        torch.cuda.synchronize()
        e2e_products += r2["iters"]
    e2e_units, e2e_dt = replicas.combine(e2e_products, time.perf_counter() - t0, dist)
    nbytes = b.numel() * b.element_size()

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    last = reps[-1]
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [p.n1, p.n2], "unknowns": 2 * p.N, "restart": RESTART,
                      "deflated": D.r, "step_arnoldi_steps": args.step_iters,
                      "parallelism": f"replicas x{world} (one incidence angle per GPU)", "l2": L2_NOTE,
                      "tile_rows": tune["tile_rows"], "cycles": "CUDA graphs (gmres_opts.graph)"}}
    out["autotune"] = tune
    out["e2e"] = {"value": e2e_units / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                  "d2h_bytes_per_step": nbytes}
    # library kernels per step (counted in the identical profiled steps) x timed steps
    out["gpu_launches"] = int(round(sum(v["launches"] for v in kt.result.values()) / PROF_STEPS * args.steps))
    out["gmres"] = {"arnoldi_steps_per_step": last["iters"], "cycles": last["cycles"], "n_reorth": last["n_reorth"],
                    "rel_res_solved_after_step": last["rel_res_solved"], "rel_res_orig_after_step": last["rel_res_orig"],
                    "reached_tol": last["converged"], "tol": TOL, "step_s": dt / args.steps,
                    "us_per_arnoldi_step": 1e6 * dt / products, "deflation_build_s": t_defl,
                    "deflation_converged": D.converged, "operator_setup_s": t_setup}
    out["clocks"] = clk.summary()

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    fp64 = fp64_peak(die)
    FP64_PEAK_TFLOPS = fp64["measured_tflops"]
    out["fp64_peak"] = fp64
    cycles = prof_cycles
    fp64_products = cycles                 # one FP64 restart residual per cycle (x0 = 0 skips the first)
    kernels = {"_note": f"CUDA events around each launch over {PROF_STEPS} extra steps identical to the timed ones"}
    best = None
    for cls, st in kt.result.items():
        ent = {"launches": st["launches"], "ms": round(st["ms"], 3)}
        bound, work = work_model(cls, p, op, D.r, RESTART, cycles, prof_products, fp64_products)
        if bound == "hbm":
            ent.update({"bound": "hbm", "GBps": work / (st["ms"] / 1e3) / 1e9})
            ent["frac"] = ent["GBps"] / hbm_peak
        elif bound == "alu":
            ent.update({"bound": "alu", "TFLOPs_fp64": work / (st["ms"] / 1e3) / 1e12})
            ent["frac"] = ent["TFLOPs_fp64"] / FP64_PEAK_TFLOPS
        kernels[cls] = ent
        if bound and (best is None or st["ms"] > kt.result[best]["ms"]):
            best = cls
    out["kernels"] = kernels
    if best:
        k = kernels[best]
        bound, work = work_model(best, p, op, D.r, RESTART, cycles, prof_products, fp64_products)
        per_launch = work / k["launches"]
        avg_s = k["ms"] / k["launches"] / 1e3
        if bound == "hbm":
            out["roofline"] = {"bound": "hbm", "achieved": per_launch / avg_s / 1e9, "peak": hbm_peak,
                               "unit": "GB/s", "frac": (per_launch / avg_s / 1e9) / hbm_peak, "traffic": None,
                               "kernel": best, "algorithmic_bytes_per_launch": per_launch,
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"}
        else:
            out["roofline"] = {"bound": "alu", "achieved": per_launch / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                               "unit": "TFLOP/s", "frac": (per_launch / avg_s / 1e12) / FP64_PEAK_TFLOPS,
                               "traffic": None, "kernel": best, "algorithmic_flops_per_launch": per_launch,
                               "peak_source": (f"FP64 FMA probe of this run (die_fp64_peak, {fp64['sms']} SMs; "
                                               f"nominal {fp64['nominal_tflops']:.3f} TFLOP/s)")}
            if best == "dots" and NCU_DOTS and 2 * p.N == NCU_DOTS["n"]:
                _, tot_bytes = work_model("dots_bytes", p, op, D.r, RESTART, cycles, prof_products, fp64_products)
                alg_bytes = tot_bytes / k["launches"]
                captured_alg = (NCU_DOTS["nv"] * 24 + 16) * NCU_DOTS["n"]
                out["roofline"]["traffic"] = NCU_DOTS["dram_bytes"] * alg_bytes / captured_alg
                out["roofline"]["algorithmic_bytes_per_launch"] = alg_bytes
                out["roofline"]["traffic_source"] = (NCU_DOTS["source"] + ", scaled to the average launch by the "
                                                     "algorithmic bytes")

    _extra(out, "matvec", lambda: matvec_rates(op, p, die, torch))
    if isinstance(out.get("matvec"), dict) and "c64" in out["matvec"]:
        mv = out["matvec"]["c64"]
        out["roofline_matvec"] = {"bound": "hbm", "achieved": mv["GBps"], "peak": hbm_peak, "unit": "GB/s",
                                  "frac": mv["GBps"] / hbm_peak,
                                  "traffic": NCU_PRODUCT["dram_bytes"] if 2 * p.N == NCU_PRODUCT["n"] else None,
                                  "traffic_source": NCU_PRODUCT["source"],
                                  "kernel": "complex64 regularised product (5 passes, one call)",
                                  "algorithmic_bytes_per_launch": mv["algorithmic_bytes"],
                                  "us_per_product": mv["us_per_product"],
                                  "note": "L2 flushed before each product; CUDA events on the launching stream"}
    _extra(out, "fp64_same_budget", lambda: fp64_same_budget(op, b, args.step_iters, dt / args.steps, torch))
    if not args.single_system:
        _extra(out, "batch_solve", lambda: [batch_solve_rates(op, D, die, torch, nrhs=k) for k in (4, 8)])
        _extra(out, "small_grids", lambda: small_grid_rates(die, W, torch))
        _extra(out, "many_systems", lambda: many_rates(die, W, torch))
    _extra(out, "te_mag", lambda: te_mag_rates(die, W, torch))
    if not args.no_compare:
        _extra(out, "plain_fp64_same_budget", lambda: plain_fp64(op, b, args.step_iters, dt / args.steps, last))
        _extra(out, "time_to_tol", lambda: time_to_tol(die, W, torch))
        _extra(out, "config2_to_tol", lambda: config2_to_tol(op, b, D, die, torch))
    if not args.no_cpu:
        try:
            out["cpu_baseline"] = cpu_oracle_rate(args.n)
        except Exception as e:  # noqa: BLE001
            out["cpu_baseline"] = {"unavailable": str(e)}
    print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _extra(out: dict, key: str, fn):
    """An informational section of the JSON line, measured after the timed region: a
    failure in it is recorded under its key instead of losing the line."""
    try:
        out[key] = fn()
    except Exception as e:  # noqa: BLE001
        out[key] = {"error": f"{type(e).__name__}: {e}"}


def profile_driver(args):
    """Fixed short run on the 512^2 core-shell for kernel captures (launch order: the
    complex64 product's K1 K2 K3K1 K2 K3, then GMRES kernels without, then with deflation)."""
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    p = W.config2(args.n)
    op32 = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    x = torch.ones(2, p.n2, p.n1, dtype=torch.complex64, device="cuda")
    op32.apply_regularized(x)
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    _, r1 = op.solve(b, restart=RESTART, tol=TOL, max_iters=RESTART, regularized=True, inner=die.DIE_FP32_INNER)
    D = die.Deflation(op, R_DEFL, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    _, r2 = op.solve(b, restart=RESTART, tol=TOL, max_iters=RESTART, regularized=True, inner=die.DIE_FP32_INNER,
                     deflation=D)
    torch.cuda.synchronize()
    print(json.dumps({"profile_driver": "ok", "steps": [r1["iters"], r2["iters"]]}))
    return 0


def profile_fno(args):
    """One forward and one backward pass of the default 128^2 network (batch 4)."""
    import torch

    from paper_1104_4263_gb300 import learned
    net = learned.default_network(128, max_batch=4)
    x = torch.randn(4, 6, 128, 128, device="cuda")
    y = net.forward(x)
    net.zero_grads()
    net.backward(torch.randn_like(y))
    torch.cuda.synchronize()
    print(json.dumps({"profile_fno": "ok", "params": net.n_params}))
    return 0


def matvec_rates(op, p, die, torch):
    """Bare regularised products per second (complex64 and FP64), L2 flushed before each."""
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for prec, dt, name in ((die.DIE_FP32_INNER, torch.complex64, "c64"), (die.DIE_FP64, torch.complex128, "c128")):
        o = op if prec == die.DIE_FP64 else die.Operator(p.eps_r, p.h, prec=prec)
        x = torch.randn(2, p.n2, p.n1, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            o.apply_regularized(x, y)
        reps = 20
        s = torch.cuda.current_stream()
        times = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            o.apply_regularized(x, y)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        # the median product: single products right after a flush vary by several percent
        # (the flush leaves dirty lines that the product's accesses evict)
        ms = reps * sorted(times)[reps // 2]
        ms_mean = sum(times)
        if name == "c64":   # the same products batched over 8 right-hand sides (e.g. incidence angles)
            nb = 8
            xb = torch.randn(nb, 2, p.n2, p.n1, dtype=dt, device="cuda")
            yb = torch.empty_like(xb)
            for _ in range(3):
                o.apply_batch(xb, yb, regularized=True)
            tb = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                o.apply_batch(xb, yb, regularized=True)
                e1.record(s)
                torch.cuda.synchronize()
                tb.append(e0.elapsed_time(e1))
            msb = reps * sorted(tb)[reps // 2]
            nbytes_b = nb * sum(product_bytes(p, o, 8).values())
            out["c64_batch8"] = {"regularized_per_s": nb * reps / (msb / 1e3), "us_per_product": 1e3 * msb / reps / nb,
                                 "GBps": nbytes_b / (msb / reps / 1e3) / 1e9,
                                 "hbm_frac": nbytes_b / (msb / reps / 1e3) / 1e9 / hbm_peak(),
                                 "note": "8 right-hand sides per call (dieop_apply_batch), L2 flushed before each call; median of 20"}
        s_el = 8 if name == "c64" else 16
        nbytes = sum(product_bytes(p, o, s_el).values())
        gbs = nbytes / (ms / reps / 1e3) / 1e9
        out[name] = {"regularized_per_s": reps / (ms / 1e3), "us_per_product": 1e3 * ms / reps,
                     "us_per_product_mean": 1e3 * ms_mean / reps,
                     "algorithmic_bytes": nbytes, "GBps": gbs, "hbm_frac": gbs / hbm_peak(),
                     "l2": "flushed (256 MB write) before each product; median of 20 products"}
    return out


def hbm_peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError):
        return 6800.0


def batch_solve_rates(op, D, die, torch, nrhs: int = 4, iters: int = 300):
    """The timed step's solver on nrhs incidence angles: nrhs sequential gmres_solve calls
    against one gmres_solve_batch call (concurrent contexts), same step budget each."""
    B = torch.stack([op.plane_wave(2 * math.pi * k / nrhs) for k in range(nrhs)]).contiguous()
    kw = dict(restart=RESTART, tol=TOL, max_iters=iters, regularized=True, inner=die.DIE_FP32_INNER, deflation=D)
    op.solve_batch(B, **kw)                       # contexts allocated, kernels warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = sum(op.solve(B[k].clone(), **kw)[1]["iters"] for k in range(nrhs))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, reps = op.solve_batch(B, **kw)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    steps = sum(r["iters"] for r in reps)
    return {"nrhs": nrhs, "arnoldi_steps_each": iters, "sequential_per_s": seq / t_seq,
            "concurrent_per_s": steps / t_bat, "speedup": (steps / t_bat) / (seq / t_seq),
            "unit": UNIT, "note": "incidence angles 2 pi k / nrhs; wall time around the host calls"}


def small_grid_rates(die, W, torch, sizes=(64, 96, 128, 256, 512), iters: int = 300, reps: int = 3,
                     nrhs: int = 8):
    """Arnoldi steps per second on the Gaussian-field scatterers of the batched workload
    (the first of each grid size), regularised, FP32-inner, GMRES(30), a fixed budget of
    `iters` steps per solve: one solve at a time with each cycle launched kernel by kernel
    or as one CUDA graph (gmres_opts.graph), and nrhs incidence angles solved concurrently
    (gmres_solve_batch), again direct or as graphs."""
    probs = {}
    for q in W.config3(64):
        probs.setdefault(q.n1, q)
    out = []
    for n in sizes:
        if n not in probs:
            continue
        q = probs[n]
        op = die.Operator(q.eps_r, q.h)
        op.autotune()                      # per-size tile height (timed once per size)
        b = op.plane_wave(0.0)
        B = torch.stack([op.plane_wave(2 * math.pi * k / nrhs) for k in range(nrhs)]).contiguous()
        kw = dict(restart=RESTART, tol=1e-14, max_iters=iters, regularized=True, inner=die.DIE_FP32_INNER)
        res = {}
        for graph in (False, True):
            op.solve(b.clone(), graph=graph, **kw)       # context allocated, kernels warm, graphs captured
            op.solve_batch(B, graph=graph, **kw)
        for graph in (False, True):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps = sum(op.solve(b.clone(), graph=graph, **kw)[1]["iters"] for _ in range(reps))
            torch.cuda.synchronize()
            res[("single", graph)] = steps / (time.perf_counter() - t0)
            t0 = time.perf_counter()
            steps = sum(sum(r["iters"] for r in op.solve_batch(B, graph=graph, **kw)[1]) for _ in range(reps))
            torch.cuda.synchronize()
            res[("batch", graph)] = steps / (time.perf_counter() - t0)
        out.append({"n": n, "unknowns": 2 * n * n,
                    "single_direct": res[("single", False)], "single_graph": res[("single", True)],
                    f"batch{nrhs}_direct": res[("batch", False)], f"batch{nrhs}_graph": res[("batch", True)]})
        del op
    return {"unit": "Arnoldi steps/s (regularised products in the solver)", "sizes": out,
            "note": (f"{iters} steps per solve, {reps} repetitions; batch: {nrhs} incidence angles 2 pi k / {nrhs} "
                     "solved concurrently; wall time around the host calls")}


def many_rates(die, W, torch, count: int = 16, n_angles: int = 4, iters: int = 200):
    """The batched workload's first `count` scatterers (mixed grid sizes) under n_angles
    incidence angles each: the count x n_angles systems solved one after another
    (gmres_solve) and all together (gmres_solve_many, cycles direct and as graphs);
    regularised, FP32-inner, GMRES(30), a fixed budget of `iters` Arnoldi steps each."""
    probs = W.config3(64)[:count]
    ops, bs = [], []
    for q in probs:
        op = die.Operator(q.eps_r, q.h)
        op.autotune()                      # per-size tile height (timed once per size)
        for j in range(n_angles):
            ops.append(op)
            bs.append(op.plane_wave(2 * math.pi * j / n_angles))
    kw = dict(restart=RESTART, tol=1e-14, max_iters=iters, regularized=True, inner=die.DIE_FP32_INNER)
    for k in range(0, len(ops), n_angles):          # contexts allocated, kernels warm, graphs captured
        ops[k].solve(bs[k].clone(), **kw)
    die.solve_many(ops, bs, **kw)
    die.solve_many(ops, bs, graph=True, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = sum(op.solve(b.clone(), **kw)[1]["iters"] for op, b in zip(ops, bs))
    torch.cuda.synchronize()
    rates = {"sequential": seq / (time.perf_counter() - t0)}
    for name, graph in (("many_direct", False), ("many_graph", True)):
        t0 = time.perf_counter()
        _, reps = die.solve_many(ops, bs, graph=graph, **kw)
        torch.cuda.synchronize()
        rates[name] = sum(r["iters"] for r in reps) / (time.perf_counter() - t0)
    sizes = sorted({q.n1 for q in probs})
    return {"systems": len(ops), "scatterers": count, "angles": n_angles, "grid_sizes": sizes,
            "arnoldi_steps_each": iters, "unit": "Arnoldi steps/s (regularised products in the solver)", **rates,
            "speedup_many_graph": rates["many_graph"] / rates["sequential"],
            "note": "wall time around the host calls; gmres_solve_many runs up to 16 systems at once"}


def config2_to_tol(op, b, D32, die, torch, k: int = 1000, budget: int = 2000):
    """The metric's second half on the 512^2 core-shell: GMRES to 1e-6 under Section 5's
    fair-memory rule with k = 1000 vectors -- plain FP64 GMRES(k) on A against GMRES(k - r)
    on A_R A P^-1 (r = 20) with FP64 products and with FP32-inner products -- for a budget
    of `budget` Arnoldi steps each.  On this object none reaches 1e-6 (the core's segment
    [1, -2 + 0.1i] of Eq. (3.20) passes 0.033 from the origin, 0.017 after Eq. (5.3)): the
    residual reached and the seconds per step are the comparison."""
    marks = (100, 300, 1000, 2000)
    out = {"fair_memory_vectors": k, "r": D32.r, "tol": TOL, "budget_steps": budget}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D64 = die.Deflation(op, R_DEFL, tol=1e-4, regularized=True, inner=die.DIE_FP64)
    torch.cuda.synchronize()
    t_b64 = time.perf_counter() - t0
    for name, kw in (("plain_fp64", dict(restart=k)),
                     ("reg_defl_fp64", dict(restart=k - D64.r, regularized=True, deflation=D64)),
                     ("reg_defl_mixed", dict(restart=k - D32.r, regularized=True, deflation=D32,
                                             inner=die.DIE_FP32_INNER))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = op.solve(b, tol=TOL, max_iters=budget, history=budget, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h = rep["history"]
        out[name] = {"restart": kw["restart"], "seconds": dt, "iters": rep["iters"], "converged": rep["converged"],
                     "rel_res_solved": rep["rel_res_solved"], "rel_res_orig": rep["rel_res_orig"],
                     "ms_per_step": 1e3 * dt / max(rep["iters"], 1), "n_reorth": rep["n_reorth"],
                     "history": {m: float(h[m - 1]) for m in marks if m <= len(h)}}
    out["deflation_build_s"] = {"fp64": t_b64}
    out["note"] = ("residual estimates of the solved system at the marked steps; none of the three reaches 1e-6 "
                   "(the same stagnation as the oracle's GMRES on the object at 64^2 and 128^2)")
    out["core_shell_64"] = core_shell_small_to_tol(die, torch)
    return out


def core_shell_small_to_tol(die, torch, n: int = 64, k: int = 1500):
    """The closest member of the core-shell family the method solves to 1e-6: the same
    permittivities and cell size h = 1/64 on a 64^2 grid (a one-wavelength box), where
    unrestarted GMRES converges (the oracle: about 700 steps on A_R A, 1500 on A).  Fair
    memory k = 1500 vectors: plain FP64 GMRES(k) against A_R A P^-1 GMRES(k - r) in FP64 and
    FP32-inner, r = 5 (the eigenvalues beyond the Section 5 radius at this size)."""
    from paper_1104_4263_gb300 import workloads as W
    p = W.config2(n)
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    rows = {}
    for name, inner in (("plain_fp64", None), ("reg_defl_fp64", die.DIE_FP64), ("reg_defl_mixed", die.DIE_FP32_INNER)):
        tb, D, kw = 0.0, None, dict(restart=k)
        if inner is not None:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            D = die.Deflation(op, 5, tol=1e-4, regularized=True, inner=inner)
            torch.cuda.synchronize()
            tb = time.perf_counter() - t0
            kw = dict(restart=k - D.r, regularized=True, deflation=D, inner=inner)
        op.solve(b, tol=TOL, max_iters=50, **kw)              # context and kernels warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = op.solve(b, tol=TOL, max_iters=6000, **kw)
        torch.cuda.synchronize()
        rows[name] = {"restart": kw["restart"], "seconds": time.perf_counter() - t0, "iters": rep["iters"],
                      "converged": rep["converged"], "rel_res_orig": rep["rel_res_orig"], "deflation_build_s": tb}
    base = rows["plain_fp64"]["seconds"]
    for v in rows.values():
        v["speedup_vs_plain_fp64"] = base / v["seconds"] if v["seconds"] > 0 else None
    return {"grid": [n, n], "unknowns": 2 * p.N, "tol": TOL, **rows}


def fp64_same_budget(op, b, step_iters, step_s, torch):
    """The headline configuration in its FP64 form: A_R A P^-1 with an FP64 deflation
    build (r = 20) and FP64 products inside the cycles, GMRES(30), the same step budget."""
    from paper_1104_4263_gb300 import die
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D = die.Deflation(op, R_DEFL, tol=1e-4, regularized=True, inner=die.DIE_FP64)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, rep = op.solve(b, restart=RESTART, tol=TOL, max_iters=step_iters, regularized=True, inner=die.DIE_FP64,
                      deflation=D, graph=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"arnoldi_steps": rep["iters"], "seconds": dt, "regularized_per_s": rep["iters"] / dt,
            "rel_res_solved": rep["rel_res_solved"], "rel_res_orig": rep["rel_res_orig"],
            "deflation_build_s": tb, "seconds_ratio_vs_step": dt / step_s,
            "note": "FP64 products and FP64 deflation inside the cycles; same budget as the timed (FP32-inner) step"}


def te_mag_rates(die, W, torch):
    """The TE system with magnetic contrast (E1, E2, H3; three planes, runtime-plan kernels):
    regularised products per second at 512^2 (FP64 and complex64, back to back), and time to
    1e-6 on a magneto-dielectric core-shell at 128^2 (eps 4 + 0.2i core, 9 + 0.3i shell,
    mu_r = 2 + 0.1i in both, side 2 wavelengths): plain FP64 GMRES(40) against A_R A P^-1
    (r = 10, complex64 deflation build) FP32-inner GMRES(30)."""
    import numpy as np
    out = {}
    p = W.config2(512)
    mu = np.where(np.abs(p.eps_r - 1.0) > 0, 2.0 + 0.1j, 1.0).astype(np.complex128)
    for prec, dt, name in ((die.DIE_FP64, torch.complex128, "c128"), (die.DIE_FP32_INNER, torch.complex64, "c64")):
        op = die.Operator(p.eps_r, p.h, prec=prec, pol=die.DIE_TE_MAG, mu_r=mu)
        x = torch.randn(3, p.n2, p.n1, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            op.apply_regularized(x, y)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record(s)
        for _ in range(reps):
            op.apply_regularized(x, y)
        e1.record(s)
        torch.cuda.synchronize()
        out[f"product_512_{name}_us"] = 1e3 * e0.elapsed_time(e1) / reps
    q = W.core_shell(128, side=2.0, r_core=0.35, r_shell=0.7, eps_core=4.0 + 0.2j, eps_shell=9.0 + 0.3j)
    mu = np.where(np.abs(q.eps_r - 1.0) > 0, 2.0 + 0.1j, 1.0).astype(np.complex128)
    op = die.Operator(q.eps_r, q.h, pol=die.DIE_TE_MAG, mu_r=mu)
    b = op.plane_wave(0.0)
    op.solve(b, restart=40, tol=TOL, max_iters=40)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, ra = op.solve(b, restart=40, tol=TOL, max_iters=20000)
    torch.cuda.synchronize()
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    D = die.Deflation(op, 10, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    kw = dict(restart=30, tol=TOL, regularized=True, inner=die.DIE_FP32_INNER, deflation=D)
    op.solve(b, **dict(kw, max_iters=30))                 # context allocated, kernels warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rr = op.solve(b, max_iters=20000, **kw)
    torch.cuda.synchronize()
    tr = time.perf_counter() - t0
    out["core_shell_128"] = {"unknowns": 3 * q.N, "tol": TOL,
                             "plain_fp64": {"restart": 40, "iters": ra["iters"], "s": ta, "converged": ra["converged"]},
                             "reg_defl_mixed": {"restart": 30, "r": D.r, "iters": rr["iters"], "s": tr,
                                                "converged": rr["converged"], "rel_res_orig": rr["rel_res_orig"],
                                                "deflation_build_s": tb},
                             "speedup_online": ta / tr if tr > 0 else None, "speedup_with_build": ta / (tr + tb)}
    return out


def config3_rates(die, W, torch, tol: float = 1e-6, max_iters: int = 3000):
    """The batched workload: 64 Gaussian-field scatterers on grids drawn from {64, ..., 512},
    8 incidence angles each (512 right-hand sides), complex64 products with FP64 refinement
    (regularised, FP32-inner GMRES(30)), every system to `tol` (at most `max_iters` steps).
    Right-hand sides solved per second one after another (gmres_solve) and all together
    (gmres_solve_many, cycles as CUDA graphs); the two runs' Arnoldi step counts are
    compared system by system."""
    probs = W.config3(64)
    ops, bs = [], []
    for q in probs:
        op = die.Operator(q.eps_r, q.h)
        op.autotune()                      # per-size tile height (timed once per size)
        for psi in q.psi:
            ops.append(op)
            bs.append(op.plane_wave(psi))
    kw = dict(restart=RESTART, tol=tol, max_iters=max_iters, regularized=True, inner=die.DIE_FP32_INNER)
    for k in range(0, len(ops), 8):                       # contexts allocated, kernels warm
        ops[k].solve(bs[k].clone(), **dict(kw, max_iters=30))
    die.solve_many(ops[:16], bs[:16], graph=True, **dict(kw, max_iters=30))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [op.solve(b.clone(), **kw)[1] for op, b in zip(ops, bs)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, reps = die.solve_many(ops, bs, graph=True, **kw)
    torch.cuda.synchronize()
    t_many = time.perf_counter() - t0
    same = sum(a["iters"] == r["iters"] for a, r in zip(seq, reps))
    sizes = sorted({q.n1 for q in probs})
    return {"scatterers": len(probs), "right_hand_sides": len(ops), "grid_sizes": sizes, "tol": tol,
            "converged": sum(r["converged"] for r in reps), "arnoldi_steps": sum(r["iters"] for r in reps),
            "sequential_rhs_per_s": len(ops) / t_seq, "many_graph_rhs_per_s": len(ops) / t_many,
            "speedup": t_seq / t_many, "sequential_s": t_seq, "many_s": t_many,
            "same_step_counts": same,
            "note": "gmres_solve_many runs up to 16 systems at once; wall time around the host calls"}


def plain_fp64(op, b, step_iters, step_s, last):
    """Plain FP64 GMRES(30) on A u = b for the same Arnoldi-step budget."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = op.solve(b, restart=RESTART, tol=TOL, max_iters=step_iters, graph=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"arnoldi_steps": rep["iters"], "seconds": dt, "rel_res": rep["rel_res_solved"],
            "seconds_ratio_vs_step": dt / step_s,
            "note": (f"A u = b, FP64 products and Krylov, GMRES({RESTART}); same step budget as the timed step, "
                     f"which reached {last['rel_res_solved']:.3g} on A_R A P^-1 ({last['rel_res_orig']:.3g} on A)")}


def time_to_tol(die, W, torch):
    """Solve time to tolerance, plain FP64 GMRES on A vs regularised + deflated FP32-inner
    GMRES on A_R A P^-1, on problems that converge: the three test squares of the paper's
    Section 4 (side = one wavelength, 61 x 61 cells, h = 1/60) with the Table 2 fair-memory
    settings (A: restart 40; A_R A P^-1: r deflated and restart 40 - r), tol 1e-8; and
    the 32^2 cylinder (plain GMRES(20), tol 1e-8)."""
    rows = []
    cases = [("eps 16", W.paper_squares()[0], 14), ("eps -16+1.5i", W.paper_squares()[1], 30),
             ("eps 16 with 2.5+20i core", W.paper_squares()[2], 14)]
    for name, p, r in cases:
        op = die.Operator(p.eps_r, p.h)
        b = op.plane_wave(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ra = op.solve(b, restart=40, tol=1e-8, max_iters=60000)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        t0 = time.perf_counter()
        D = die.Deflation(op, r, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, rr = op.solve(b, restart=40 - r, tol=1e-8, max_iters=60000, regularized=True,
                         inner=die.DIE_FP32_INNER, deflation=D)
        torch.cuda.synchronize()
        tr = time.perf_counter() - t0
        rows.append({"case": name, "grid": [p.n1, p.n2], "r": r,
                     "plain_fp64": {"restart": 40, "s": ta, "iters": ra["iters"], "converged": ra["converged"],
                                    "rel_res": ra["rel_res_solved"]},
                     "reg_defl_mixed": {"restart": 40 - r, "s": tr, "iters": rr["iters"], "converged": rr["converged"],
                                        "rel_res_orig": rr["rel_res_orig"], "deflation_build_s": tb},
                     "speedup_online": ta / tr if tr > 0 else None,
                     "speedup_with_build": ta / (tr + tb) if tr + tb > 0 else None})
    p = W.config1(32)
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rc = op.solve(b, restart=20, tol=1e-8, max_iters=20000)
    torch.cuda.synchronize()
    rows.append({"case": "cylinder eps 4, 32x32, plain FP64 GMRES(20)", "s": time.perf_counter() - t0,
                 "iters": rc["iters"], "converged": rc["converged"]})
    return rows


# Table 2 (TE, fair memory, tol 1e-8): per scatterer and system, the deflated count r,
# restart, the paper's iterations and speed-up over A (Matlab on the paper's 3N system;
# context for the ratios, not a target).
PAPER_TABLE2 = {
    "eps 16": {"A": (0, 40, 15258, 1.0), "AP^-1": (6, 34, 14002, 1.1), "A_R A": (0, 40, 4030, 2.5),
               "A_R A P^-1": (14, 26, 3626, 3.0)},
    "eps -16+1.5i": {"A": (0, 40, 1708, 1.0), "AP^-1": (7, 33, 1659, 1.1), "A_R A": (0, 40, 1021, 1.1),
                     "A_R A P^-1": (30, 10, 534, 2.4)},
    "eps 16 with 2.5+20i core": {"A": (0, 40, 11823, 1.0), "AP^-1": (3, 37, 13156, 0.9), "A_R A": (0, 40, 3032, 2.6),
                                 "A_R A P^-1": (14, 26, 2911, 3.0)},
}


def paper_table2(args):
    """The four systems of Table 2 (A, A P^-1, A_R A, A_R A P^-1) on the three test squares
    of Section 4 (61 x 61, h = 1/60), with the table's r and restart, tol 1e-8, FP64
    throughout as in the paper, plus A_R A P^-1 in the FP32-inner form.  Solve times
    exclude the deflation builds (reported beside them).  Prints one JSON line."""
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    names = list(PAPER_TABLE2)
    out = []
    for name, p in zip(names, W.paper_squares()):
        op = die.Operator(p.eps_r, p.h)
        b = op.plane_wave(0.0)
        rows = {}
        variants = [(sys_, reg, defl, die.DIE_FP64) for sys_, reg, defl in
                    (("A", False, False), ("AP^-1", False, True), ("A_R A", True, False), ("A_R A P^-1", True, True))]
        variants.append(("A_R A P^-1", True, True, die.DIE_FP32_INNER))
        for sys_, reg, defl, inner in variants:
            r, restart, paper_iters, paper_speedup = PAPER_TABLE2[name][sys_]
            D, tb = None, 0.0
            if defl:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                D = die.Deflation(op, r, tol=1e-4, regularized=reg, inner=inner)
                torch.cuda.synchronize()
                tb = time.perf_counter() - t0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = op.solve(b, restart=restart, tol=1e-8, max_iters=100000, regularized=reg, inner=inner,
                              deflation=D)
            torch.cuda.synchronize()
            key = sys_ + (" (FP32-inner)" if inner == die.DIE_FP32_INNER else "")
            rows[key] = {"r": r, "restart": restart, "iters": rep["iters"], "s": time.perf_counter() - t0,
                         "deflation_build_s": tb, "converged": rep["converged"],
                         "rel_res_orig": rep["rel_res_orig"], "paper_iters": paper_iters,
                         "paper_speedup": paper_speedup}
        ta = rows["A"]["s"]
        for v in rows.values():
            v["speedup"] = ta / v["s"] if v["s"] > 0 else None
        out.append({"case": name, "grid": [p.n1, p.n2], "systems": rows})
    print(json.dumps({"paper_table2": out, "tol": 1e-8,
                      "note": "2N unknowns (E1, E2) here against the paper's 3N: compare speed-ups, not counts"}))
    return 0


# Table 1 (TM, fair memory, tol 1e-8): per scatterer the paper's (iterations, seconds) for
# A with restart 40 and for A P^-1 with r = 28 and restart 12, and the speed-up.
PAPER_TABLE1 = {
    "eps 16": {"A": (7311, 168.0), "AP^-1": (4230, 78.0), "speedup": 2.2},
    "eps -16+1.5i": {"A": (27, 0.7), "AP^-1": (14, 0.5), "speedup": 1.4},
    "eps 16 with 2.5+20i core": {"A": (1000, 23.0), "AP^-1": (749, 14.0), "speedup": 1.6},
}


def paper_table1(args):
    """The two TM systems of Table 1 (A with restart 40; A P^-1 deflating the 28 largest
    eigenvalues of A, restart 12) on the three test squares of Section 4 (61 x 61,
    h = 1/60), tol 1e-8, FP64 throughout.  Solve seconds exclude the deflation build."""
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    out = []
    for name, p in zip(PAPER_TABLE1, W.paper_squares()):
        op = die.Operator(p.eps_r, p.h, pol=die.DIE_TM)
        b = op.plane_wave(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ra = op.solve(b, restart=40, tol=1e-8, max_iters=200000)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        t0 = time.perf_counter()
        D = die.Deflation(op, 28, tol=1e-4, regularized=False)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, rd = op.solve(b, restart=12, tol=1e-8, max_iters=200000, deflation=D)
        torch.cuda.synchronize()
        td = time.perf_counter() - t0
        ref = PAPER_TABLE1[name]
        out.append({"case": name, "grid": [p.n1, p.n2],
                    "A": {"restart": 40, "iters": ra["iters"], "s": ta, "converged": ra["converged"],
                          "paper_iters": ref["A"][0]},
                    "AP^-1": {"r": 28, "restart": 12, "iters": rd["iters"], "s": td, "converged": rd["converged"],
                              "deflation_build_s": tb, "paper_iters": ref["AP^-1"][0]},
                    "speedup": ta / td if td > 0 else None, "paper_speedup": ref["speedup"]})
    print(json.dumps({"paper_table1": out, "tol": 1e-8,
                      "note": "TM (E3) unknowns N here; the paper's counts are for its own discretisation"}))
    return 0


def _timed_solve(op, b, torch, **kw):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = op.solve(b, **kw)
    torch.cuda.synchronize()
    return rep, time.perf_counter() - t0


# Section 5's speed-ups read from the text (Figs. 6-7): restart rule -> (min, max) over the sweep
PAPER_SWEEP_SIZE = {"r/2": (None, 2.4), "2r": (2.1, 5.1), "10r": (8.7, 46.6)}
PAPER_SWEEP_EPS = {"2r": (1.8, 4.1), "10r": (1.6, 11.4)}


def paper_sweeps(args, sizes=(1.0, 1.6, 2.2), eps_values=(10.0, 15.0, 20.0), tol: float = 1e-8,
                 max_iters: int = 60000):
    """Section 5's fair-memory experiments on lossless squares at 15 points per medium
    wavelength: for each object, r = the eigenvalues of A_R A outside the deflation radius
    (r = 0 in the deflation build), then for each memory rule restart(A_R A P^-1) = r/2, 2r,
    10r against restart(A) = r, 3r, 11r, both solved to tol in FP64 (the paper's Matlab
    double).  Sizes a/lambda at eps 16; permittivities at a/lambda = 1."""
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    rules = (("r/2", 0.5, 1.0), ("2r", 2.0, 3.0), ("10r", 10.0, 11.0))

    def one(p):
        op = die.Operator(p.eps_r, p.h)
        b = op.plane_wave(0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D = die.Deflation(op, 0, tol=1e-4, regularized=True, r_max=128)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        r = D.r
        row = {"grid": p.n1, "r": r, "deflation_build_s": tb}
        for name, fp, fa in rules:
            kp, ka = max(1, int(round(fp * r))), max(1, int(round(fa * r)))
            ra, ta = _timed_solve(op, b, torch, restart=min(ka, 2048), tol=tol, max_iters=max_iters)
            rp, tp = _timed_solve(op, b, torch, restart=min(kp, 2048), tol=tol, max_iters=max_iters,
                                  regularized=True, deflation=D)
            row[name] = {"restart_A": ka, "restart_ARAP": kp, "A": {"iters": ra["iters"], "s": ta,
                         "converged": ra["converged"]}, "ARAP": {"iters": rp["iters"], "s": tp,
                         "converged": rp["converged"], "rel_res_orig": rp["rel_res_orig"]},
                         "speedup": ta / tp if tp > 0 else None}
        return row

    size_rows = [dict(a_over_lambda=a, **one(W.lossless_square(a, 16.0))) for a in sizes]
    eps_rows = [dict(eps=e, **one(W.lossless_square(1.0, e))) for e in eps_values]
    print(json.dumps({"paper_sweeps": {"size": size_rows, "permittivity": eps_rows, "tol": tol,
                                       "paper_speedups_size": PAPER_SWEEP_SIZE,
                                       "paper_speedups_permittivity": PAPER_SWEEP_EPS,
                                       "note": "FP64 throughout; 2N unknowns (E1, E2) against the paper's 3N"}}))
    return 0


def paper_sinusoidal(args, tol: float = 1e-8, max_iters: int = 60000):
    """Section 5's continuous-permittivity example (233 x 233, a = 4 wavelengths): A with
    restart 1620 against A_R A P^-1 with r = 180 and restart 1440, FP64, tol 1e-8; the
    paper's Matlab run took 162692 s and 11620 s (+ 775 s of eigs), a 14x (13.1x) speed-up."""
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    p = W.sinusoidal()
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    D = die.Deflation(op, 180, tol=1e-4, regularized=True)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    rp, tp = _timed_solve(op, b, torch, restart=1440, tol=tol, max_iters=max_iters, regularized=True, deflation=D)
    ra, ta = _timed_solve(op, b, torch, restart=1620, tol=tol, max_iters=max_iters)
    print(json.dumps({"paper_sinusoidal": {
        "grid": [p.n1, p.n2], "unknowns": 2 * p.N, "r": D.r, "deflation_converged": D.converged,
        "deflation_build_s": tb,
        "A": {"restart": 1620, "iters": ra["iters"], "s": ta, "converged": ra["converged"],
              "rel_res": ra["rel_res_solved"]},
        "ARAP": {"restart": 1440, "iters": rp["iters"], "s": tp, "converged": rp["converged"],
                 "rel_res_orig": rp["rel_res_orig"]},
        "speedup_online": ta / tp if tp > 0 else None, "speedup_with_build": ta / (tp + tb),
        "paper": {"A_s": 162692, "ARAP_s": 11620, "eigs_s": 775, "speedup_online": 14.0, "speedup_with_build": 13.1},
        "tol": tol}}))
    return 0


def config5_budget(args, r: int = 40, restart: int = 40):
    """The large composite: 400 seeded cylinders (radius 0.2-0.6 wavelength, eps_r in
    {-6 + 0.5i, 2, 9, 30 + 1i}) on a 2048^2 grid of side 32 wavelengths (8.4 M unknowns).
    Plain FP64 GMRES(40) and, under Section 5's memory rule, GMRES(40 + r) on A, against
    A_R A P^-1 with the r = 40 largest-magnitude eigenvalues deflated, GMRES(40), with FP64
    products and with complex64 products (FP64 Krylov and restarts), each for `--budget`
    Arnoldi steps toward 1e-6.  Reported: residual of the solved system at marked steps,
    seconds, and the steps and seconds each form needs to reach the residual plain FP64
    GMRES(40) ends at."""
    import numpy as np
    import torch

    from paper_1104_4263_gb300 import die, workloads as W
    budget = args.budget
    marks = [m for m in (100, 300, 1000, 2000, 5000) if m <= budget]
    t0 = time.perf_counter()
    p = W.random_cylinders()
    t_gen = time.perf_counter() - t0
    op = die.Operator(p.eps_r, p.h)
    b = op.plane_wave(0.0)
    out = {"grid": [p.n1, p.n2], "unknowns": 2 * p.N, "cylinders": 400, "tol": TOL, "budget_steps": budget,
           "restart": restart, "input_seconds": t_gen}
    builds = {}
    for name, inner in (("fp32_inner", die.DIE_FP32_INNER), ("fp64", die.DIE_FP64)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D = die.Deflation(op, r, tol=1e-4, regularized=True, inner=inner)
        torch.cuda.synchronize()
        builds[name] = (D, time.perf_counter() - t0)
    out["deflation_build_s"] = {k: v[1] for k, v in builds.items()}
    out["deflation_converged"] = {k: v[0].converged for k, v in builds.items()}
    runs = (("plain_fp64", dict(restart=restart)),
            ("plain_fp64_fair_memory", dict(restart=restart + r)),
            ("reg_defl_fp64", dict(restart=restart, regularized=True, deflation=builds["fp64"][0])),
            ("reg_defl_mixed", dict(restart=restart, regularized=True, deflation=builds["fp32_inner"][0],
                                    inner=die.DIE_FP32_INNER)))
    hist = {}
    for name, kw in runs:
        op.solve(b, tol=TOL, **dict(kw, max_iters=kw["restart"]))   # context allocated, kernels warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = op.solve(b, tol=TOL, max_iters=budget, history=budget, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        h = np.asarray(rep["history"])
        hist[name] = (h, dt)
        out[name] = {"restart": kw["restart"], "seconds": dt, "iters": rep["iters"], "converged": rep["converged"],
                     "rel_res_solved": rep["rel_res_solved"], "rel_res_orig": rep["rel_res_orig"],
                     "ms_per_step": 1e3 * dt / max(rep["iters"], 1), "n_reorth": rep["n_reorth"],
                     "history": {m: float(h[m - 1]) for m in marks if m <= len(h)}}
    target = float(hist["plain_fp64"][0][-1])
    out["plain_fp64_final_residual"] = target
    for name, (h, dt) in hist.items():
        hit = np.nonzero(h <= target)[0]
        if hit.size:
            steps = int(hit[0]) + 1
            out[name]["steps_to_plain_final"] = steps
            out[name]["seconds_to_plain_final"] = dt * steps / len(h)
    base = out["plain_fp64"].get("seconds_to_plain_final")
    for name in hist:
        s_ = out[name].get("seconds_to_plain_final")
        if base and s_:
            out[name]["speedup_to_plain_final"] = base / s_
    out["note"] = ("seconds_to_plain_final = the solve's seconds x the fraction of its steps taken until its "
                   "residual first reached plain FP64 GMRES(40)'s final residual; the deflation build is extra")
    print(json.dumps({"config5": out}))
    return 0


def _learned_summary(rows):
    """Means, convergence counts and residual geomeans of learned.evaluate's rows."""
    def mean(key, sub):
        v = [r[sub][key] for r in rows]
        return sum(v) / len(v)
    summary = {
        "held_out_fields": len(rows),
        "without_network": {"mean_iters": mean("iters", "without_network"), "mean_s": mean("s", "without_network"),
                            "converged": sum(r["without_network"]["converged"] for r in rows)},
        "with_network": {"mean_iters": mean("iters", "with_network"), "mean_s": mean("s", "with_network"),
                         "converged": sum(r["with_network"]["converged"] for r in rows),
                         "used_fallback": sum(r["with_network"]["used_fallback"] for r in rows)},
        "mean_initial_guess_rel_res": sum(r["initial_guess_rel_res"] for r in rows) / len(rows),
        "mean_deflation_build_s": sum(r["deflation_build_s"] for r in rows) / len(rows),
    }
    summary["initial_guess_only"] = {"mean_iters": mean("iters", "initial_guess_only"),
                                     "mean_s": mean("s", "initial_guess_only"),
                                     "converged": sum(r["initial_guess_only"]["converged"] for r in rows)}
    gm = lambda sub: math.exp(sum(math.log(max(r[sub]["rel_res_orig"], 1e-300)) for r in rows) / len(rows))
    for sub in ("without_network", "with_network", "initial_guess_only"):
        summary[sub]["geomean_final_rel_res"] = gm(sub)
        summary[sub]["fields_lower_than_without"] = sum(r[sub]["rel_res_orig"] < r["without_network"]["rel_res_orig"]
                                                        for r in rows)
    summary["iteration_ratio"] = summary["without_network"]["mean_iters"] / max(summary["with_network"]["mean_iters"], 1)
    summary["time_ratio"] = summary["without_network"]["mean_s"] / max(summary["with_network"]["mean_s"], 1e-9)
    return summary


def learned_bench(args):
    """The learned preconditioner end to end (see paper_1104_4263_gb300/learned.py): pairs,
    training, evaluation; one JSON line."""
    import torch

    from paper_1104_4263_gb300 import learned
    torch.cuda.set_device(0)
    data = learned.make_dataset(args.pairs)
    net = learned.default_network(128, max_batch=16)
    err0 = learned.relative_error(net, data)
    losses, t_train = learned.train(net, data, epochs=args.epochs)
    err1 = learned.relative_error(net, data)
    rows = learned.evaluate(net, args.held_out)
    summary = _learned_summary(rows)
    # the same network on held-out fields of the same generator with Re eps_r in [1, 16]
    # (no negative permittivity), where the method without it converges
    rows_pos = learned.evaluate(net, args.held_out, re_lo=1.0)
    summary_pos = _learned_summary(rows_pos)
    print(json.dumps({"learned": {
        "grid": 128, "network": {"layers": 4, "modes": 16, "width": 32, "hidden": 128, "params": net.n_params,
                                 "arithmetic": "BF16 tcgen05 GEMMs, FP32 accumulation"},
        "pairs": {"count": len(data.kinds), "solve": data.kinds.count("solve"), "product": data.kinds.count("product"),
                  "generation_s": data.gen_s},
        "training": {"epochs": len(losses), "loss_per_epoch": losses, "seconds": t_train,
                     "rel_error_before": err0, "rel_error_after": err1},
        "evaluation": summary, "rows": rows,
        "evaluation_positive_eps": summary_pos, "rows_positive_eps": rows_pos,
        "tol": 1e-6, "note": ("FGMRES(30) with the network as x0 and right preconditioner for up to 600 steps, "
                              "then the method without it; the network's x0 alone followed by that method; and "
                              "the method alone: regularised + deflated (r = 8) FP32-inner GMRES(100), all to 1e-6 "
                              "on ||b - A u|| / ||b|| within 8000 Arnoldi steps")}}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
