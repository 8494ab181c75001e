"""Benchmark: full-TDDFT PCG iterations on the chromophore-sized synthetic workload.

One step = one preconditioned-CG iteration (tddft_pcg_step) on k = 10 state pairs: traces and
Q (Sec. III C), multi-state gradient, inner-CG preconditioner (Eq. precond), conjugation, one
batched operator application on the search directions (Eq. operator_RPA: L -> P map, Kohn-Sham
difference products, response density, FFT Hartree + LDA kernel, potential integrals, coupling
products), the sum-functional line step and sign flip + Gram-Schmidt (Eq. ortho).

Metric: operator applies (state pairs) per second over whole iterations, counting the k applies
of each iteration and the k of every periodic re-application. The end-to-end figure runs
tddft_apply on pinned host buffers (host->device and device->host copies inside the timed
region). `--impl reference` times the FP64 CPU oracle on a bounded sample of one application.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under torch.distributed.run,
one independent replica per GPU (the single-system path has no data-parallel split).

Other lines (one JSON line each, not the default):
  --batched S     S uneven systems solved at once (tddft_create_batch / tddft_solve_batch);
  --scaling N,..  operator applies on the core + shell series (synthetic.scaling_recipe) at the
                  given atom counts, with time per unit of algorithmic work.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDDFT operator applies/s; time to k states at 1e-5 Ha, learned vs plain PCG"
UNIT = "applies/s"
WORKLOAD = ("chromophore-140: 140 pseudo-atoms in a 30 A cell, 120^3 grid (0.25 A), 4 phi + 9 chi "
            "per atom, 8 A localisation radius, 12 A kernel cutoff, k=10 states, synthetic seeded")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--config", default="chromophore", choices=["chromophore", "small"])
    ap.add_argument("--precond", default="exact", choices=["exact", "iter", "none"],
                    help="preconditioner of the timed PCG steps (exact: Eq. precond solved in its "
                         "eigenbases; iter: the paper's inner CG to 1e-4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes of the grid kernels")
    ap.add_argument("--no-iter-line", action="store_true",
                    help="skip the extra timing of PCG steps with the paper's inner-CG preconditioner")
    ap.add_argument("--learned-train-atoms", type=int, default=150,
                    help="atoms of the two training systems of the time-to-k comparison")
    ap.add_argument("--learned-eval-atoms", type=int, default=200,
                    help="atoms of the unseen system the time-to-k comparison solves")
    ap.add_argument("--learned-precision", default="mixed", choices=["fp64", "mixed"],
                    help="precision of the time-to-solution comparison of the preconditioners")
    ap.add_argument("--no-time-to-k", action="store_true",
                    help="skip the separate time-to-solution report (not part of the timed steps)")
    ap.add_argument("--batched", type=int, default=0,
                    help="instead of the default line: solve this many uneven systems at once (systems/s)")
    ap.add_argument("--batch-max-atoms", type=int, default=300)
    ap.add_argument("--batch-seed", type=int, default=3)
    ap.add_argument("--batch-tol", type=float, default=1e-5, help="residual (Ha) each batched system converges to")
    ap.add_argument("--batch-workers", type=int, default=8, help="processes generating the systems")
    ap.add_argument("--batch-pool-atoms", type=int, default=150,
                    help="systems from this size up are generated in the main process (pooled table sums)")
    ap.add_argument("--scaling", default="",
                    help="comma-separated atom counts of the core + shell series: time operator applies "
                         "on each (one JSON line with the series)")
    ap.add_argument("--scaling-k", type=int, default=4)
    ap.add_argument("--scaling-dense", action="store_true",
                    help="the series with dense products instead of the truncated form")
    ap.add_argument("--scaling-cpu-max-atoms", type=int, default=500,
                    help="largest member whose oracle sample runs (dense products grow as N^3)")
    return ap.parse_args()


def recipe(name):
    from paper_1507_08157_gb300 import synthetic as sy
    return sy.CONFIG_CHROMOPHORE if name == "chromophore" else sy.CONFIG_SMALL


def workload_name(args):
    if args.config == "small":
        return "small-8: 8 pseudo-atoms, 16 A cell, 48^3 grid, 4 phi + 4 chi per atom, 7 A radius, no truncation"
    return WORKLOAD


# ------------------------------------------------------------------------------------------------
# N replicas (one per GPU): the job's time is the slowest rank's, its rate all ranks' units over it
def max_over_ranks(ms, world, device):
    """The largest of the ranks' timed-region lengths (every rank takes part)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units processed by all ranks per second of the slowest rank's timed region."""
    return units_per_rank * world / (ms_max / 1000.0)


# ------------------------------------------------------------------------------------------------
# GPU clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                clk, mx, util = float(f[1]), float(f[2]), float(f[4])
            except ValueError:
                continue
            smax = mx
            if util > 0:
                sm.append(clk)
            for name, v in zip(names, f[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return os.cpu_count(), model or "unknown"


def blas_threads(n):
    """Set the thread count of the BLAS numpy loaded (OpenBLAS or MKL) through its own call;
    returns False when no such call is found."""
    import ctypes
    ok = False
    try:
        with open("/proc/self/maps") as f:
            libs = {l.split()[-1] for l in f if ".so" in l and ("blas" in l.lower() or "mkl" in l.lower())}
    except OSError:
        libs = set()
    for path in libs:
        try:
            lib = ctypes.CDLL(path)
        except OSError:
            continue
        for sym in ("openblas_set_num_threads", "openblas_set_num_threads64_", "scipy_openblas_set_num_threads",
                    "scipy_openblas_set_num_threads64_", "MKL_Set_Num_Threads"):
            fn = getattr(lib, sym, None)
            if fn is not None:
                fn(ctypes.c_int(n))
                ok = True
    return ok


def cpu_oracle_sample(sys_, target_s=15.0):
    """Time the FP64 oracle's operator application on a bounded sample and scale it to one
    state-pair application: all matrix products and one FFT Poisson solve in full, the response
    density and potential integrals on the chi functions of the first m atoms (their cost is
    linear in the chi atoms covered), scaled by natoms / m."""
    from oracle import grid as ogrid
    from oracle import operator as oop
    from paper_1507_08157_gb300 import synthetic as sy
    op = oop.Operator(sys_)
    Pp, Pq = sy.random_kernels(sys_, 1, 9)
    t0 = time.perf_counter()
    Pc, Hc, Hv, Pv = op.Pc, op.Hc, op.Hv, op.Pv
    _ = Pc @ Hc @ Pp[0] - Pp[0] @ Hv @ Pv
    fq = Pc @ Hc @ Pq[0] - Pq[0] @ Hv @ Pv
    rho_full = np.zeros((1, sys_.n, sys_.n, sys_.n))
    V = op.response_potential(rho_full)
    _ = fq + 2.0 * Pc @ np.zeros_like(Pq[0]) @ Pv
    t_fixed = time.perf_counter() - t0
    chi_sub = ogrid.BoxedSet(sys_.chi, sys_.n)
    groups = chi_sub.groups
    m, spent = 0, 0.0
    while m < len(groups) and spent < target_s:
        chi_sub.groups = groups[m:m + 1]
        t1 = time.perf_counter()
        ogrid.response_density(chi_sub, op.phi, Pq)
        ogrid.potential_integrals(chi_sub, op.phi, V, sys_.dV)
        spent += time.perf_counter() - t1
        m += 1
    per_apply = t_fixed + spent * len(groups) / max(m, 1)
    cores, model = host_cpu()
    return {"value": 1.0 / per_apply, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
            "estimate": m < len(groups), "timed_s": t_fixed + spent,
            "sample": (f"one state-pair application: matrix products and FFT Poisson solve in full, "
                       f"grid contractions on the chi functions of {m} of {len(groups)} atoms "
                       f"({spent:.1f} s), scaled linearly; numpy/scipy float64, BLAS threads = all cores")}


def cpu_oracle_one_thread(sys_, target_s=6.0):
    """The same bounded sample with the BLAS on one thread (the grid contractions of the oracle
    are single-threaded numpy either way)."""
    if not blas_threads(1):
        return None
    try:
        r = cpu_oracle_sample(sys_, target_s=target_s)
    finally:
        blas_threads(os.cpu_count() or 1)
    return {"value": r["value"], "unit": UNIT, "cores": 1, "sample": r["sample"].replace("all cores", "1")}


# ------------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1507_08157_gb300 import synthetic as sy
    s = sy.generate(recipe(args.config))
    vals, timed = [], []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_sample(s, target_s=3.0)
        if i >= args.warmup:
            vals.append(r["value"])
            timed.append(r["timed_s"])
    v = float(np.mean(vals))
    cores, model = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * args.k / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args), "states": args.k, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
                             "sample": r["sample"]},
            "estimate": ("each step times a bounded sample of one application and scales its grid "
                         "contractions to the whole system: value and ms_per_step are extrapolated")
                        if r["estimate"] else None,
            "timed_s_per_step": float(np.mean(timed)),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_time_to_k(tddft, sy, torch, stream, s, k, autotune, tol=1e-5):
    """Time to the lowest k states at a 1e-5 Ha residual in mixed precision on the benchmark's
    system, from the seeded random start, with the exact preconditioner and with the paper's
    inner CG (Eq. precond to 1e-4). The response kernels are not truncated here: at the
    throughput workload's 12 A cutoff the synthetic system's PCG stalls near 1e-2 Ha (its density
    kernels decay slowly), so there is no converged answer to time."""
    import dataclasses
    su = dataclasses.replace(s, kernel_cutoff=0.0)
    out = {"workload": "the benchmark's chromophore-140 system, response kernels untruncated", "k": k,
           "precision": "mixed", "tol_Ha": tol}
    for pre in ("exact", "iter"):
        c = tddft.Context(su, precision="mixed", stream=stream.cuda_stream, tol=tol, max_iter=600, precond=pre)
        if autotune:
            c.autotune(k)
        st = c.state(sy.initial_guess(su, k, 0))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, res, it, rc = st.solve()
        torch.cuda.synchronize()
        out[pre] = {"s": time.perf_counter() - t0, "iterations": int(it), "status": int(rc),
                    "resid_max": float(np.max(res)), "omega": [float(x) for x in om]}
        st.close()
        c.close()
    return out


def learned_vs_plain(tddft, sy, torch, stream, k=10, train_atoms=16, eval_atoms=24, tol=1e-5, precision="fp64"):
    rows = ([], [], [])
    for seed in (31, 32):
        s = sy.generate(sy.small_density_recipe(train_atoms, seed))
        c = tddft.Context(s, precision=precision, stream=stream.cuda_stream)
        st = c.state(sy.initial_guess(s, k, seed))
        for it in range(30):
            st.step()
            if it % 3 == 2:
                for acc, t in zip(rows, c.samples(st)):
                    acc.append(t)
        st.close()
        c.close()
    X, T, W = (torch.cat(a).contiguous() for a in rows)
    n_b = T.shape[1]
    n_f = X.shape[1] - n_b
    net = tddft.Mlp(n_b, n_f, 256)
    net.set(sy.mlp_init(n_f, 256, n_b * n_b, 33))
    steps, batch = 2000, 512
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l0, l1 = net.train(X, T, steps, batch, 1e-3, sy.minibatch_order(X.shape[0], steps, batch, 34), W)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    s = sy.generate(sy.small_density_recipe(eval_atoms, 35))
    Y0 = sy.initial_guess(s, k, 35)
    out = {}
    for pre in ("iter", "adaptive", "exact", "learned", "none"):
        c = tddft.Context(s, precision=precision, precond="iter" if pre == "adaptive" else pre, tol=tol,
                          max_iter=1000, stream=stream.cuda_stream, precond_adaptive=pre == "adaptive")
        if pre == "learned":
            c.set_mlp(net)
        st = c.state(Y0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        om, res, it, rc = st.solve()
        torch.cuda.synchronize()
        out[pre] = {"s": time.perf_counter() - t0, "iterations": it, "status": int(rc),
                    "omega_Ha": [float(x) for x in om], "stats": st.stats()}
        st.close()
        c.close()
    net.close()
    dw = max(abs(a - b) for a, b in zip(out["learned"]["omega_Ha"], out["iter"]["omega_Ha"]))
    r = s.recipe
    return {"workload": f"c1-density systems: train 2 x {train_atoms} atoms ({X.shape[0]} rows, {steps} Adam "
                        f"steps of {batch}), evaluate an unseen {eval_atoms}-atom system, "
                        f"{r.cell_ang:.1f} A cell, {r.ngrid}^3 grid, 4 phi + 4 chi per atom",
            "k": k, "precision": precision, "tol_Ha": tol,
            "plain_pcg_s": out["iter"]["s"], "plain_iterations": out["iter"]["iterations"],
            "plain_inner_cg_iterations": out["iter"]["stats"][2],
            "plain_adaptive_tol_s": out["adaptive"]["s"], "plain_adaptive_tol_iterations": out["adaptive"]["iterations"],
            "plain_adaptive_tol_inner_cg_iterations": out["adaptive"]["stats"][2],
            "learned_pcg_s": out["learned"]["s"], "learned_iterations": out["learned"]["iterations"],
            "learned_fallbacks": out["learned"]["stats"][1],
            "exact_precond_s": out["exact"]["s"], "exact_precond_iterations": out["exact"]["iterations"],
            "unpreconditioned_s": out["none"]["s"], "unpreconditioned_iterations": out["none"]["iterations"],
            "status": [out[p]["status"] for p in ("iter", "adaptive", "exact", "learned", "none")],
            "max_domega_exact_vs_plain_Ha": max(abs(a - b) for a, b in zip(out["exact"]["omega_Ha"],
                                                                            out["iter"]["omega_Ha"])),
            "max_domega_learned_vs_plain_Ha": dw, "train_s": train_s, "train_loss": [l0, l1]}


# DRAM bytes (read + write) per tc_gemm_kernel launch in a timed PCG step of the default workload,
# mean over the step's 16 launches, from one capture of this build:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
#       -k regex:tc_gemm_kernel --csv python bench.py --steps 1 --warmup 1 --no-cpu-baseline
#       --no-time-to-k --no-iter-line --no-autotune
GEMM_TRAFFIC_PER_LAUNCH = 82.0e6


def stage_rooflines(prof, peaks, args):
    """Per stage of the timed steps: the time its algorithmic work takes at the measured peaks
    (roof_ms = the larger of flops at the stage's compute peak and bytes at the HBM copy rate),
    against the measured time; and the same summed over the stages that have a roof (the small
    float64 algebra has none: it is latency, not throughput)."""
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    mixed = args.precision == "mixed"
    compute_peak = {"gemm": bf16 * 1.1 / 2.25 if mixed else 1.25,
                    "response_density": bf16 if mixed else 1.25,
                    "potential_integrals": bf16 if mixed else 1.25}
    out, roof_sum, ms_sum = {}, 0.0, 0.0
    for name, (launches, ms_, flops, bytes_) in prof.items():
        if not launches or name == "small_fp64":
            continue
        t_flop = flops / (compute_peak[name] * 1e12) * 1e3 if name in compute_peak else 0.0
        t_byte = bytes_ / (hbm * 1e9) * 1e3
        roof_ms = max(t_flop, t_byte)
        out[name] = {"ms": round(ms_, 4), "roof_ms": round(roof_ms, 4), "frac": round(roof_ms / max(ms_, 1e-12), 4),
                     "bound": "tensor" if t_flop >= t_byte and name in compute_peak else "hbm"}
        roof_sum += roof_ms
        ms_sum += ms_
    small = prof.get("small_fp64", (0, 0.0))[1]
    summed = {"roof_ms": round(roof_sum, 4), "measured_ms": round(ms_sum, 4),
              "frac": round(roof_sum / max(ms_sum, 1e-12), 4), "small_fp64_ms_excluded": round(small, 4),
              "peaks": {"tf32_tflops": round(bf16 * 1.1 / 2.25, 1), "f16_tflops": bf16, "hbm_gbs": hbm},
              "note": "gemm flops are 2MNK of each product (the float32-accurate split issues three MMAs); "
                      "float64 stages against the nominal 1.25 TFLOP/s"}
    return out, summed


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1507_08157_gb300 import synthetic as sy
    from paper_1507_08157_gb300 import tddft

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tddft.load()
    s = sy.generate(recipe(args.config))
    stream = torch.cuda.current_stream()
    ctx = tddft.Context(s, precision=args.precision, stream=stream.cuda_stream, tol=1e-5, precond=args.precond)
    k = args.k
    # tile shapes of the grid kernels picked by the library's autotuner (outside the timed region)
    tuning = ctx.autotune(k) if args.precision == "mixed" and not args.no_autotune else None
    st = ctx.state(sy.initial_guess(s, k, 0))
    for _ in range(args.warmup):
        st.step()
    reapply = ctx.options.reapply_every
    it0 = args.warmup
    extra = sum(1 for i in range(it0, it0 + args.steps) if reapply > 0 and (i + 1) % reapply == 0)
    applies = k * (args.steps + extra)

    def barrier():
        if world > 1:
            dist.barrier()

    ctx.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            om, res = st.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    prof = ctx.profile_read()
    ctx.profile(False)
    ms_max = max_over_ranks(ms, world, "cuda")
    value = whole_job_rate(applies, world, ms_max)

    # end to end: tddft_apply from pinned host buffers, copies inside the timed region
    Pp, Pq = sy.random_kernels(s, k, 3)
    hPp = torch.from_numpy(Pp).pin_memory()
    hPq = torch.from_numpy(Pq).pin_memory()
    hfp = torch.empty_like(hPp).pin_memory()
    hfq = torch.empty_like(hPq).pin_memory()
    dPp, dPq = hPp.cuda(), hPq.cuda()
    for _ in range(2):
        ctx.apply(hPp, hPq, hfp, hfq)
    barrier()
    t0 = time.perf_counter()
    n_e2e = max(3, args.steps // 2)
    for _ in range(n_e2e):
        ctx.apply(hPp, hPq, hfp, hfq)
    e2e_s = time.perf_counter() - t0
    # device-resident operator only (context figure)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_e2e):
        ctx.apply(dPp, dPq)
    e1.record(stream)
    torch.cuda.synchronize()
    apply_only = k * n_e2e / (e0.elapsed_time(e1) / 1000.0)
    e2e = {"value": k * n_e2e * world / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hPp.numel() * 8 * 2), "d2h_bytes_per_step": int(hfp.numel() * 8 * 2)}

    # roofline of the dominant stage
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, dms, dfl, dby) = dom
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    clock = clk.summary()
    sm_mhz = clock["sm_max_mhz"] or 2070.0
    if name in ("fft_poisson_fxc", "vector", "trace"):
        achieved = dby / (dms / 1000.0) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "kernel": name,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s"}
    elif name == "gemm" and args.precision == "mixed" and os.environ.get("TDDFT_NO_TC") != "1":
        # tcgen05 kind::tf32 (three-term split); peak = measured sustained bf16 x nominal tf32/bf16
        bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
        peak = bf16 * (1.1 / 2.25)
        achieved = dfl / (dms / 1000.0) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": name,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained x 1.1/2.25 (tf32/bf16 nominal)",
                "note": "achieved counts 2MNK per product; the three-term split issues 3 MMAs per product",
                "frac_of_fp32_accurate_peak": achieved / (peak / 3.0)}
    elif (name in ("potential_integrals", "response_density") and args.precision == "mixed"
          and os.environ.get("TDDFT_NO_TC") != "1" and os.environ.get("TDDFT_NO_GRID_TC") != "1"):
        # tcgen05 kind::f16 grid contractions: the roof is the larger of the algorithmic bytes at
        # the HBM rate and the algorithmic flops at the f16 (= bf16) tensor rate
        tpk = peaks.get("bf16_tflops_sustained", 1700.0)
        hpk = peaks.get("hbm_gbs", 6800.0)
        t_flop, t_byte = dfl / (tpk * 1e12), dby / (hpk * 1e9)
        if t_byte >= t_flop:
            achieved = dby / (dms / 1000.0) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": hpk, "unit": "GB/s",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
        else:
            achieved = dfl / (dms / 1000.0) / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (f16 and bf16 dense rates are equal)"}
        roof.update({"frac": achieved / roof["peak"], "traffic": None, "kernel": name,
                     "roof_ms": {"bytes_at_hbm": 1e3 * t_byte, "flops_at_tensor": 1e3 * t_flop,
                                 "measured_per_call": dms / max(launches, 1)},
                     "note": "algorithmic work: 2 k pair_points flops (pairs of nonzero chi and phi values "
                             "at each grid point) and the tables, grids and outputs read or written once"})
    else:
        # CUDA-core float32 (mixed) or float64 contraction: ALU bound.
        lanes = 128 if args.precision == "mixed" else 2
        peak = 152 * lanes * 2 * sm_mhz * 1e6 / 1e12
        achieved = dfl / (dms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": name,
                "peak_source": f"152 SMs x {lanes} lanes x 2 flop x {sm_mhz:.0f} MHz"}
    gpu_launches = sum(v[0] for v in prof.values()) + 4 * prof.get("fft_poisson_fxc", (0,))[0]
    stages = {n: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / max(ms, 1e-9), 4)}
              for n, v in prof.items() if v[0]}
    stage_roofs, summed = stage_rooflines(prof, peaks, args)
    if roof.get("kernel") == "gemm" and roof.get("bound") == "tensor":
        roof["traffic"] = GEMM_TRAFFIC_PER_LAUNCH
        roof["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum per tc_gemm_kernel launch, mean "
                                "over the 16 launches of one timed PCG step (one ncu capture of this build)")

    # the same PCG steps with the paper's preconditioner (inner CG on Eq. precond to 1e-4), when
    # the timed steps used another one: both are reported
    iter_line = None
    if rank == 0 and not args.no_iter_line and args.precond != "iter":
        ctx_i = tddft.Context(s, precision=args.precision, stream=stream.cuda_stream, tol=1e-5, precond="iter")
        if tuning is not None:
            ctx_i.autotune(k)
        st_i = ctx_i.state(sy.initial_guess(s, k, 0))
        for _ in range(args.warmup):
            st_i.step()
        n_i = max(3, args.steps // 2)
        extra_i = sum(1 for i in range(args.warmup, args.warmup + n_i) if reapply > 0 and (i + 1) % reapply == 0)
        ctx_i.profile(True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(n_i):
            st_i.step()
        f1.record(stream)
        torch.cuda.synchronize()
        ms_i = f0.elapsed_time(f1)
        prof_i = ctx_i.profile_read()
        iter_line = {"precond": "iter (inner CG on Eq. precond to 1e-4, the paper's)", "steps": n_i,
                     "ms_per_step": ms_i / n_i, "applies_per_s": k * (n_i + extra_i) / (ms_i / 1000.0),
                     "inner_cg_iterations": st_i.stats()[2],
                     "stages_ms_per_step": {n_: round(v[1] / n_i, 3) for n_, v in prof_i.items() if v[0]}}
        st_i.close()
        ctx_i.close()

    # time to k states at 1e-5 Ha, learned vs plain PCG (mixed precision by default): the model is
    # trained on rows from plain-PCG runs on two 150-atom systems of the small workload's recipe
    # and density, then the solvers start from the same vectors on an unseen 200-atom system
    time_to_k = time_to_k_mixed = None
    if rank == 0 and not args.no_time_to_k:
        if args.config == "chromophore" and args.precision == "mixed":
            time_to_k_mixed = mixed_time_to_k(tddft, sy, torch, stream, s, k, tuning is not None)
        time_to_k = learned_vs_plain(tddft, sy, torch, stream, train_atoms=args.learned_train_atoms,
                                     eval_atoms=args.learned_eval_atoms, precision=args.learned_precision)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": workload_name(args), "states": k, "precision": args.precision,
                           "precond": args.precond,
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "inputs larger than L2 (function tables > 1 GB per pass)",
                           "applies_per_step": applies / args.steps},
                "e2e": e2e, "apply_only": {"value": apply_only, "unit": UNIT},
                "roofline": roof, "stages": stages, "stage_rooflines": stage_roofs,
                "summed_roofline": summed, "gpu_launches": int(gpu_launches),
                "clocks": {k_: clock[k_] for k_ in ("sm_mhz", "sm_max_mhz", "reasons")},
                "time_to_k": time_to_k, "time_to_k_mixed": time_to_k_mixed, "precond_iter": iter_line,
                "autotune": tuning,
                "omega_last": [float(x) for x in om], "resid_last": [float(x) for x in res]}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_sample(s)
            line["cpu_baseline"]["one_thread"] = cpu_oracle_one_thread(s)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _generate(recipe_):
    from paper_1507_08157_gb300 import synthetic as sy
    return sy.generate(recipe_)


def run_batched(args):
    """Many independent systems of uneven size solved at once (tddft_create_batch /
    tddft_solve_batch): atom counts log-uniform in [20, max], atoms in a cube at 0.1 atoms / A^3
    with 2R + 1 A of vacuum, 0.25 A grids, 4 phi + 4 chi (s, p) per atom of 7 A radius, 1 to 8
    states each. Mixed precision, converged to the method's 1e-5 Ha residual (--batch-tol) within
    600 iterations. The systems are generated on the
    host in a spawn process pool, a chunk at a time, before any of them is solved; the timed
    region is the concurrent solve of all systems (wall clock, device synchronised on both
    sides), from states already created."""
    import multiprocessing as mp
    import torch
    from paper_1507_08157_gb300 import synthetic as sy
    recs = sy.batch_recipes(args.batched, args.batch_seed, n_max=args.batch_max_atoms)
    order = sorted(range(len(recs)), key=lambda i: -recs[i][0].natoms)
    workers = max(1, args.batch_workers)
    pool = mp.get_context("spawn").Pool(workers)    # started before the first GPU call
    torch.cuda.set_device(0)
    from paper_1507_08157_gb300 import tddft
    tddft.load()
    tol = args.batch_tol
    ctxs, states, meta = [], [], []
    t_gen = t_create = 0.0
    # large systems are generated one at a time in this process, whose generator spreads their
    # table sums over a process pool of its own (a pool worker cannot start one); the rest go to
    # the worker pool a chunk at a time
    big = [i for i in order if recs[i][0].natoms >= args.batch_pool_atoms]
    rest = [i for i in order if recs[i][0].natoms < args.batch_pool_atoms]
    chunks = [[i] for i in big] + [rest[c:c + workers] for c in range(0, len(rest), workers)]
    try:
        for chunk in chunks:
            t0 = time.perf_counter()
            if len(chunk) == 1 and recs[chunk[0]][0].natoms >= args.batch_pool_atoms:
                systems = [sy.generate(recs[chunk[0]][0])]
            else:
                systems = pool.map(_generate, [recs[i][0] for i in chunk])
            t1 = time.perf_counter()
            cs = tddft.create_batch(systems, precision="mixed", tol=tol, max_iter=600, precond=args.precond)
            for i, c, sys_ in zip(chunk, cs, systems):
                k = recs[i][1]
                states.append(c.state(sy.initial_guess(sys_, k, i)))
                meta.append((i, sys_.natoms, k))
                c.sys = None                              # the device holds the system now
            ctxs.extend(cs)
            del systems
            t_gen += t1 - t0
            t_create += time.perf_counter() - t1
    finally:
        pool.close()
        pool.join()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, iters, status = tddft.solve_batch(states, nthreads=16)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ok = int(np.sum(status == tddft.OK))
    per = [{"atoms": a, "k": k, "iters": int(iters[j]), "status": int(status[j]),
            "omega_min": float(res[j][0][0]), "resid_max": float(np.max(res[j][1]))}
           for j, (i, a, k) in enumerate(meta)]
    for j, p_ in enumerate(per):
        if p_["status"] != tddft.OK:
            p_["error"] = states[j].ctx.last_error()
    line = {"metric": "systems solved per second (batched, uneven sizes)", "value": len(states) / wall,
            "unit": "systems/s", "n_gpus": 1, "higher_is_better": True, "impl": "ours",
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched: {len(states)} systems, {min(m[1] for m in meta)}-"
                                   f"{max(m[1] for m in meta)} atoms (log-uniform, seed {args.batch_seed}), "
                                   "0.1 atoms/A^3 cube + 2R + 1 A vacuum, 0.25 A grid, 4 phi + 4 chi per atom, "
                                   f"7 A radius, 1-8 states, mixed precision, {args.precond} preconditioner, "
                                   f"residual {tol:g} Ha, at most 600 iterations",
                       "systems": len(states), "atoms_total": int(sum(m[1] for m in meta)),
                       "states_total": int(sum(m[2] for m in meta)), "host_threads": 16},
            "wall_s": wall, "converged": ok, "iters_total": int(np.sum(iters)),
            "generate_s": t_gen, "create_s": t_create, "per_system": per}
    print(json.dumps(line), flush=True)


def _loglog_slope(x, y):
    """Least-squares slope of log y against log x."""
    lx, ly = np.log(np.asarray(x, dtype=float)), np.log(np.asarray(y, dtype=float))
    return float(np.polyfit(lx, ly, 1)[0]) if len(lx) > 1 else None


def run_scaling(args):
    """Operator applies on the linear-scaling series (synthetic.scaling_recipe: a 140-atom core
    and a solvent-like shell at 0.1 atoms / A^3, 4 phi + 9 chi per atom, R = 8 A, 0.25 A grid,
    every density matrix truncated at 15 A), k states, mixed precision, in the truncated form of
    Sec. IV (tddft_create_sparse: cluster-blocked matrices, block-sparse tensor-core products).
    Per size: device-resident applies timed with CUDA events after warm-up, the per-stage times of
    the library's profiler, and the time per unit of algorithmic work W (flops: 2 k pair_points
    for each grid contraction, 2 n_I n_K n_J over the atom-block triples that contribute to each
    block-sparse product), so that time / W stays flat when the time grows with the work; the line
    ends with the fitted exponents of time, of the grid stages' time and of W against N, and of
    time against W."""
    import torch
    from paper_1507_08157_gb300 import synthetic as sy
    from paper_1507_08157_gb300 import tddft
    torch.cuda.set_device(0)
    tddft.load()
    stream = torch.cuda.current_stream()
    k = args.scaling_k
    series = []
    for natoms in [int(x) for x in args.scaling.split(",") if x.strip()]:
        rec = sy.scaling_recipe(natoms)
        t0 = time.perf_counter()
        s = sy.generate(rec)
        t1 = time.perf_counter()
        ctx = tddft.Context(s, precision="mixed", stream=stream.cuda_stream, precond="none",
                            sparse=not args.scaling_dense)
        t2 = time.perf_counter()
        ctx.sys = None                                  # the device holds the system now
        pair_points, table_values = ctx.work()
        tuning = None if args.no_autotune else ctx.autotune(k)
        rng = np.random.default_rng(3)
        shape = (k, ctx.nnz) if ctx.sparse else (k, ctx.nc, ctx.nv)
        dPp = torch.from_numpy(rng.standard_normal(shape)).cuda()
        dPq = torch.from_numpy(rng.standard_normal(shape)).cuda()
        cpu = None
        if not args.no_cpu_baseline and natoms <= args.scaling_cpu_max_atoms:
            cpu = cpu_oracle_sample(s)
        nnz = ctx.nnz if ctx.sparse else ctx.nc * ctx.nv
        del s
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(args.warmup):
            ctx.apply(dPp, dPq)
        torch.cuda.synchronize()
        # at least about a second of timed applies, so that the clock sampler sees the load
        per = (time.perf_counter() - w0) / max(args.warmup, 1)
        steps = max(args.steps, int(math.ceil(1.0 / max(per, 1e-3))))
        ctx.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                ctx.apply(dPp, dPq)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        prof = ctx.profile_read()
        ctx.profile(False)
        flops = sum(v[2] for v in prof.values()) / steps
        vscf_ms = sum(prof.get(n_, (0, 0.0))[1] for n_ in ("response_density", "potential_integrals",
                                                            "fft_poisson_fxc")) / steps
        series.append({
            "atoms": natoms, "cell_ang": rec.cell_ang, "grid": rec.ngrid,
            "n_chi": ctx.nc, "n_phi": ctx.nv, "kernel_values": nnz,
            "kernel_fill": nnz / float(ctx.nc * ctx.nv),
            "pair_points": pair_points, "table_values": table_values,
            "ms_per_apply": ms, "applies_per_s": k / (ms / 1000.0), "timed_applies": steps,
            "vscf_ms_per_apply": vscf_ms,
            "work_tflop_per_apply": flops / 1e12, "ns_per_mflop": 1e6 * ms / max(flops / 1e6, 1e-30),
            "stages_ms": {n: round(v[1] / steps, 3) for n, v in prof.items() if v[0]},
            "generate_s": t1 - t0, "create_s": t2 - t1, "cpu_baseline": cpu,
            "autotune": [{k_: r[k_] for k_ in ("stage", "kind", "chi_chunk", "phi_chunk", "ms", "chosen")}
                         for r in tuning] if tuning else None,
            "clocks": {k_: clk.summary()[k_] for k_ in ("sm_mhz", "sm_max_mhz", "reasons")}})
        print(json.dumps({"partial": series[-1]}), flush=True)
        ctx.close()
        del dPp, dPq
        torch.cuda.empty_cache()
    atoms = [r["atoms"] for r in series]
    line = {"metric": "operator applies/s and time per unit of work vs atom count", "unit": UNIT,
            "n_gpus": 1, "higher_is_better": True, "impl": "ours", "dtype": "f32", "data": "synthetic",
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "linear-scaling series: 140-atom core + shell at 0.1 atoms/A^3, 4 phi + 9 chi "
                                   "per atom, 8 A radius, 0.25 A grid, every density matrix truncated at 15 A "
                                   f"({'dense products' if args.scaling_dense else 'truncated form, block-sparse products'}), "
                                   f"k={k}, mixed precision",
                       "l2": "inputs larger than L2 (function tables of several GB)"},
            "series": series,
            "exponent_time_vs_atoms": _loglog_slope(atoms, [r["ms_per_apply"] for r in series]),
            "exponent_vscf_time_vs_atoms": _loglog_slope(atoms, [r["vscf_ms_per_apply"] for r in series]),
            "exponent_work_vs_atoms": _loglog_slope(atoms, [r["work_tflop_per_apply"] for r in series]),
            "exponent_time_vs_work": _loglog_slope([r["work_tflop_per_apply"] for r in series],
                                                   [r["ms_per_apply"] for r in series]),
            "exponent_time_per_work_vs_atoms": _loglog_slope(atoms, [r["ns_per_mflop"] for r in series]),
            "work_note": "work = 2 k pair_points per grid contraction + 2 n_I n_K n_J over the contributing "
                         "atom-block triples of every block-sparse product (padding and pattern cuts "
                         "inside cluster blocks excluded)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.scaling:
        run_scaling(args)
        return
    if args.batched > 0:
        run_batched(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
