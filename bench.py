"""Benchmark of the CNP DG operator hot path on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl native|reference]

A step is one pass of the hot path over one synthetic state of the workload
(inputs resident in HBM): R(u), J(u)v and J(u)^T w of the FP64-accurate
operator in both of its arithmetics (native FP64, and double-float on the FP32
pipe), the single-precision J(u)v of the mixed-precision inner solve, one
block-Jacobi apply (FP32-stored inverses), the c_m recovery and one device
inner product. `value` is the metric's quantity: the FP64-accurate J(u)v in
GDOF/s (unknown degrees of freedom per second of one application, in the faster
of the two arithmetics, both parity-tested against the oracle at 1e-12),
summed over ranks; the FP64, double-float and FP32 J v rates, the fraction of
the HBM roofline and the FP64 vs mixed solve times are top-level keys, and the
whole step's blend under `step_blend_GDOF_s`. Each operator is timed with
CUDA events on the launching stream; between steps a 512 MB buffer is written
to flush the 129 MB L2 (outside the events). The block-Jacobi setup, FGMRES and
Newton rows run in a full solve of the cube16_p3 workload after the timed
steps, FP64 and mixed precision, with block-Jacobi and with the two-level
preconditioner, reported under `solve`; the batched operating-point sweep of
the plate reactor at 0.1-0.8 V (continuation in the applied potential,
graph-captured Krylov cycles) is reported under `batched_solve`.

Extra keys: per-operator throughput (`ops`), the roofline of the dominant kernel
(`roofline`), the CPU oracle on a bounded sample (`cpu_baseline`), the same
metric end to end through the C ABI with host buffers (`e2e`), SM clocks sampled
during the timed region (`clocks`) and the number of kernel launches (`gpu_launches`).

`--impl reference` times the CPU oracle (the plain FP64 reference
implementation of the same operator) on a bounded sample of the same workload,
on the host cores; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ENP DG Jv GDOF/s at p=3 hex, FP64 vs mixed; % of HBM roofline; solve time"
DEFAULT_WORKLOAD = "channel64_p3"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 issue rate of GB300: 2 FMA per clock per SM (measured 1.20 TFLOP/s with an
# FMA loop at 1.99 GHz; 152 SMs x 2 x 2 flop x 2.07 GHz = 1.26 TFLOP/s nominal).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# A double-float multiply-add of a sum-factorised contraction takes 12 FP32
# instructions (TwoProd with the cross terms: 4, TwoSum: 6, error sum: 2): its
# issue-limited rate in FP64-equivalent flops.
DF32_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12

# DRAM traffic per launch of a kernel from one ncu capture, keyed by the hash
# of the sources that kernel is built from (stale -> reported null): the
# operator kernels from the operator headers, the block apply from the solver.
TRAFFIC = {
    ("5d4d7cdd78a5", "jvp_df32", "channel64_p3"): 699.86e6,  # face + element kernel
    ("5d4d7cdd78a5", "jvp_f32", "channel64_p3"): 243.07e6,   # face + element kernel
    ("33fe528c30dc", "bj_apply_f32", "channel64_p3"): 4933.98e6,
}

KERNEL_SOURCES = {
    "operator": ("enp_operator.cuh", "enp_operator3d.cuh", "enp_common.cuh"),
}


def _function_text(src, signature):
    """The text of the definition that starts at `signature` (through its
    closing brace at column 0)."""
    i = src.index(signature)
    return src[i:src.index("\n}\n", i) + 3]


def _solver_apply_text():
    """The block apply's own source: its kernel and its host launcher."""
    with open(os.path.join(ROOT, "paper_2112_09271_gb300", "csrc", "enp_solver.cu")) as fh:
        src = fh.read()
    return (_function_text(src, "__global__ void bj_apply_kernel(") +
            _function_text(src, "static cudaError_t bj_apply_plain(enp_handle h, const TV* x, TV* y) {"))


def _kernel_hash(kind=None):
    """Hash of the sources a kernel family is built from: 'operator' (the
    operator headers), 'solver' (the block-apply kernel and its launcher), or
    both (None)."""
    h = hashlib.sha1()
    if kind in (None, "operator"):
        for f in KERNEL_SOURCES["operator"]:
            with open(os.path.join(ROOT, "paper_2112_09271_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    if kind in (None, "solver"):
        h.update(_solver_apply_text().encode())
    return h.hexdigest()[:12]


def _family(op_name):
    return "solver" if op_name.startswith("bj_") else "operator"



def contraction_flops(dim, p, nf, mode):
    """Floating-point operations (2 per multiply-add) of the sum-factorised
    contractions of one element for one operator application (mode 'res', 'jvp'
    or 'vjp'): the volume, and the dim faces the element owns (every face once),
    each with the traces of both sides and the test contractions of both sides,
    all counted as interior. Pointwise physics is excluded."""
    n, q = p + 1, p + 2
    if dim == 3:
        interp = q * n ** 3 + q * q * n * n + q ** 3 * n + 3 * q ** 4
        trace = n ** 3 + 2 * (q * n * n + q * q * n)
        ftest = 2 * (q * q * n + q * n * n) + n ** 3
    else:
        interp = q * n * n + q * q * n + 2 * q ** 3
        trace = n * n + 2 * q * n
        ftest = 2 * q * n + n * n
    nv = 1 if mode == "res" else 2
    vol = nf * (nv * interp + interp)
    faces = dim * nf * (2 * nv * trace + 2 * ftest)
    return 2 * (vol + faces)


def algorithmic_bytes_per_dof(mode, word):
    """Each vector read or written once, geometry and velocity computed on the
    fly: R reads u and writes r; J v and J^T w read u and v (or w) and write
    the result."""
    return {"res": 2, "jvp": 3, "vjp": 3}[mode] * word


def read_peaks():
    try:
        with open(PEAKS_PATH) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path):
        self.path = path
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(prob, budget_s=12.0):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload's elements: J(u)v rows (the metric's operator) of randomly chosen
    elements, in batches that grow until about budget_s seconds of CPU time are
    spent."""
    import oracle
    import workloads as W
    orc = oracle.Oracle(prob)
    u, v = W.random_state(prob, 2), W.random_vector(prob, 3)
    rng = np.random.default_rng(0)
    n_el = min(64, prob.E)
    t_ops, dofs, n_total = 0.0, 0, 0
    while t_ops < budget_s:
        el = rng.choice(prob.E, n_el, replace=False)
        t0 = time.perf_counter()
        orc.jvp(u, v, elems=el)
        dt = time.perf_counter() - t0
        t_ops += dt
        n_total += n_el
        dofs += n_el * prob.n_fields * prob.Np
        want = n_el * (budget_s - t_ops) / max(dt, 1e-4)
        n_el = int(max(1, min(prob.E, want, 8 * n_el)))
    return {"value": dofs / t_ops / 1e9, "unit": "GDOF/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"J(u)v rows of {n_total} randomly chosen elements (with "
                      f"repeats) of {prob.name} ({prob.E} elements), {t_ops:.1f} s of CPU time"}


def SOLVE_VARIANTS(enp):
    """(label, two-level preconditioner, Newton options) of the full solves.
    `arith` is the arithmetic of the FP64 residual and J v (native FP64 or
    double-float); `guess` starts from the initial guess of Sec. 4.3 instead
    of Phi = 0."""
    f64 = dict(bj_storage=enp.BJ_F64, mixed=False)
    mix = dict(bj_storage=enp.BJ_BF16, mixed=True)
    df = dict(f64, arith=enp.ARITH_DF32)
    return [("fp64", 0, f64), ("mixed", 0, mix), ("fp64_two_level", 1, f64),
            ("fp64_df32_two_level", 1, df),
            ("fp64_df32_two_level_pc32", 1, dict(df, bj_storage=enp.BJ_F32)),
            ("mixed_two_level", 1, mix), ("mixed_two_level_lag3", 1, dict(mix, pc_lag=3)),
            ("mixed_two_level_sweep", 1, dict(mix, sweep=1)),
            ("mixed_two_level_paper_guess", 1, dict(mix, guess=1))]


CHANNEL_SOLVE_VARIANTS = ("fp64_df32_two_level", "fp64_df32_two_level_pc32", "mixed_two_level",
                          "mixed_two_level_paper_guess")


def run_solves(enp, W, name, labels=None, reference="fp64"):
    """Newton with backtracking line search and preconditioned FGMRES(50)
    (inner rtol 1e-3, as in the paper) from c = c_in, Phi = 0 to
    ||R|| <= 1e-10 ||R_0||: FP64 throughout (native, or double-float arithmetic
    for the residual and J v), then mixed (FP32 inner operator and Krylov
    vectors, BF16 block inverses assembled in FP32) with the FP64 outer
    residual; each with block-Jacobi alone and with the two-level
    preconditioner (block-Jacobi plus the coarse element-mean potential
    correction); and from the initial guess of Sec. 4.3 (c = c_in, Phi from the
    charge equation at constant c, inner rtol 1e-2), its time included. Wall
    time on the device, and each solution's distance from the `reference`
    one."""
    import torch
    prob = W.config(name)
    op = enp.Operator(prob)
    for code in (enp.ARITH_F64, enp.ARITH_DF32):
        op.set_arithmetic(code)
        op.autotune()
    u0 = np.zeros((prob.n_fields, prob.E, prob.Np))
    for k in range(1, prob.n_fields):
        u0[k] = prob.c_in[k - 1]
    out, sols = {"workload": name, "n_dof": prob.n_dof, "rtol": 1e-10}, {}
    for label, two, kw in SOLVE_VARIANTS(enp):
        if labels is not None and label not in labels:
            continue
        kw = dict(kw)
        op.set_sweep(kw.pop("sweep", 0))
        op.set_arithmetic(kw.pop("arith", enp.ARITH_F64))
        guess = kw.pop("guess", 0)
        op.set_preconditioner(two)
        u = torch.tensor(u0.reshape(-1), device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gst = None
        if guess:
            gst = op.initial_guess(u, rtol=1e-8, krylov_rtol=1e-2, krylov_restart=50,
                                   raise_on_fail=False, **kw)
        st = op.newton_solve(u, max_it=30, rtol=1e-10, krylov_restart=50, krylov_max_it=4000,
                             krylov_rtol=1e-3, raise_on_fail=False, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sols[label] = u.cpu().numpy()
        out[label] = {"seconds": dt, "newton_iterations": st["iterations"],
                      "krylov_iterations": st["krylov_iterations"],
                      "setups": st["setups"], "setup_seconds": st["setup_seconds"],
                      "krylov_seconds": st["krylov_seconds"],
                      "converged": bool(st["converged"]),
                      "final_relative_residual": st["residual_norm"] / st["initial_norm"]}
        if gst is not None:
            out[label]["initial_guess"] = {
                "newton_iterations": gst["iterations"],
                "krylov_iterations": gst["krylov_iterations"],
                "converged": bool(gst["converged"])}
    op.set_arithmetic(enp.ARITH_F64)
    ref = sols[reference]
    others = [k for k in sols if k != reference]
    for label in others:
        out[label + "_vs_" + reference + "_relative_error"] = float(
            np.linalg.norm(sols[label] - ref) / np.linalg.norm(ref))
    if "mixed" in sols:
        out["speedup_mixed_over_fp64"] = out[reference]["seconds"] / out["mixed"]["seconds"]
    best = min(others, key=lambda k: out[k]["seconds"])
    out["best"] = best
    out["speedup_best_over_" + reference] = out[reference]["seconds"] / out[best]["seconds"]
    return out


def run_batched_solve(enp, W, name, batch=8, volts=(0.1, 0.8),
                      labels=("fp64", "mixed", "mixed_device_loop", "mixed_sweep",
                              "mixed_paper_guess"), pc_lag=1, shared_blocks=-1, storage="f32",
                      restart=50):
    """The operating-point sweep of the plate reactor (Sec. 5.2): `batch`
    applied cathode potentials from volts[0] to volts[1] (anode at 0), all
    solved in one batched Newton run per stage, with continuation in the
    applied potential (Butler-Volmer exponents reach e^31 at 0.8 V, beyond the
    reach of Newton from a plain guess), the two-level preconditioner and FGMRES
    restart cycles replayed from a captured CUDA graph (`_device_loop`: every
    Newton iteration one graph launch with device-side loops over the cycles,
    the line search and the steps). FP64 and mixed (FP32
    inner operator, FP32 block inverses); initial guess c = c_in,
    Phi = phi_app / 2 at the first stage, or (`_paper_guess`) the initial guess
    of Sec. 4.3 at the first stage's potentials (Phi from the charge equation
    at c = c_in, inner rtol 1e-2, its time included); the last stage to 1e-10
    relative."""
    import torch
    prob = W.config(name)
    phis = 38.92 * np.linspace(volts[0], volts[1], batch)  # F/RT at 298.15 K
    target = np.array([[ph, 0.0, 0.0, 0.0] for ph in phis])
    op = enp.Operator(prob, batch=batch)
    op.autotune()
    op.set_preconditioner(1)
    op.set_shared_blocks(shared_blocks)
    bj_mixed = enp.BJ_BF16 if storage == "bf16" else enp.BJ_F32
    step0 = 0.125
    u0 = W.reactor_initial_state(prob, phis * step0)
    out = {"workload": name, "batch": batch, "volts": list(volts), "n_dof_per_point": prob.n_dof,
           "pc_lag": pc_lag, "shared_blocks": shared_blocks, "mixed_storage": storage,
           "restart": restart,
           "rtol_last_stage": 1e-10, "continuation": "lambda from 0.125, x1.5 after a converged "
           "stage (max 0.25), /2 after a failed one; intermediate stages to 1e-6 in 10 iterations"}
    sols = {}
    kws = {"fp64": dict(bj_storage=enp.BJ_F64, mixed=False),
           "mixed": dict(bj_storage=bj_mixed, mixed=True),
           "mixed_sweep": dict(bj_storage=bj_mixed, mixed=True),
           "mixed_paper_guess": dict(bj_storage=bj_mixed, mixed=True),
           "mixed_device_loop": dict(bj_storage=bj_mixed, mixed=True, device_loop=True),
           "mixed_device_loop_sweep": dict(bj_storage=bj_mixed, mixed=True, device_loop=True)}
    for label in labels:
        op.set_sweep(1 if label.endswith("_sweep") else 0)
        u = torch.tensor(u0, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gst = None
        if label.endswith("_paper_guess"):
            op.set_phi_app(target * step0)
            gst = op.initial_guess(u, rtol=1e-8, krylov_rtol=1e-2, graph=True,
                                   raise_on_fail=False, **kws[label])
        st = op.newton_continuation(u, target, step0=step0, graph=True, raise_on_fail=False,
                                    pc_lag=pc_lag, krylov_restart=restart, **kws[label])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sols[label] = u.cpu().numpy()
        last = st["last"]
        out[label] = {"seconds": dt, "points_per_second": batch / dt,
                      "reached_lambda": st["lambda"], "stages": st["stages"],
                      "failed_stages": st["failed_stages"],
                      "newton_iterations": st["newton_iterations"],
                      "krylov_iterations": st["krylov_iterations"],
                      "converged": st["status"] == 0,
                      "last_stage_relative_residual": last["residual_norm"] / last["initial_norm"],
                      "last_stage_residual_norm": last["residual_norm"]}
        if gst is not None:
            out[label]["initial_guess"] = {"newton_iterations": gst["iterations"],
                                           "krylov_iterations": gst["krylov_iterations"],
                                           "converged": bool(gst["converged"])}
    if "fp64" in sols:
        ref = sols["fp64"]
        for lab in sols:
            if lab != "fp64":
                out[lab + "_vs_fp64_relative_error"] = float(
                    np.linalg.norm(sols[lab] - ref) / np.linalg.norm(ref))
                out["speedup_" + lab + "_over_fp64"] = out["fp64"]["seconds"] / out[lab]["seconds"]
    return out


def run_fgmres_profile(enp, W, args):
    """Whole FGMRES(50) restart cycles (50 iterations each: rtol 0) on the solve
    workload with the two-level preconditioner, FP64 or FP32 (`--only
    fgmres_f64|fgmres_f32`): `warmup` untimed cycles, then `steps` timed ones;
    the per-iteration time of the Krylov loop (J v, preconditioner, CGS2)."""
    import torch
    prob = W.config(args.solve_workload)
    op = enp.Operator(prob)
    op.autotune()
    op.set_preconditioner(1)
    f32 = args.only == "fgmres_f32"
    u = torch.tensor(W.random_state(prob, 2), device="cuda")
    op.block_jacobi_setup(u, enp.BJ_F32 if f32 else enp.BJ_F64)
    dt = torch.float32 if f32 else torch.float64
    ul = u.to(dt)
    b = torch.tensor(W.random_vector(prob, 6), device="cuda").to(dt)
    x = torch.zeros_like(b)
    its, t = 0, 0.0
    for i in range(args.warmup + args.steps):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.fgmres_solve(ul, b, x, restart=50, max_it=50, rtol=0.0, raise_on_fail=False)
        torch.cuda.synchronize()
        if i >= args.warmup:
            t += time.perf_counter() - t0
            its += st["iterations"]
    return {"only": args.only, "workload": prob.name, "n_dof": prob.n_dof,
            "iterations": its, "ms_per_iteration": 1e3 * t / its, "kernel_hash": _kernel_hash()}


def run_precond_profile(enp, W, args):
    """Block-Jacobi against the downwind block Gauss-Seidel sweep (`--only
    precond_f32`) on the solve workload, FP32 inverses and the two-level
    correction: the time of one preconditioner application to an FP32 vector
    (CUDA events, L2 flushed before each) and one FP32 FGMRES(50) linear solve
    to 1e-4 at the reactor's initial state for 0.45 V (a random state on other
    workloads)."""
    import torch
    prob = W.config(args.solve_workload)
    op = enp.Operator(prob)
    op.autotune()
    op.set_preconditioner(1)
    if prob.name.startswith("reactor"):
        u = torch.tensor(W.reactor_initial_state(prob, [0.45 * 38.92]), device="cuda")
    else:
        u = torch.tensor(W.random_state(prob, 2), device="cuda")
    x = torch.tensor(W.random_vector(prob, 6), device="cuda").float()
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {"only": args.only, "workload": prob.name, "n_dof": prob.n_dof,
           "fgmres": "FP32, restart 50, rtol 1e-4", "kernel_hash": _kernel_hash()}
    for sweep in (0, 1):
        op.set_sweep(sweep)
        op.block_jacobi_setup(u, enp.BJ_F32)
        ms = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            op.block_jacobi_apply_f32(x, out=y)
            e1.record()
            torch.cuda.synchronize()
            if i >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        z = torch.zeros_like(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.fgmres_solve(u.float(), x, z, restart=50, max_it=5000, rtol=1e-4,
                             raise_on_fail=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["sweep" if sweep else "block_jacobi"] = {
            "apply_ms": float(np.median(ms)), "fgmres_iterations": st["iterations"],
            "fgmres_seconds": dt, "ms_per_iteration": 1e3 * dt / max(1, st["iterations"]),
            "converged": st["converged"] == 1,
            # the true residual of the FP32 iterate (an FP32 J v), relative to b
            "relative_residual": st["relative_residual"]}
    return out


def run_reference(args, rank, world):
    import workloads as W
    if rank != 0:
        return
    prob = W.config(args.workload)
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_baseline(prob, budget_s=budget / 4)
    vals, t0 = [], time.perf_counter()
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(prob, budget_s=budget)
        vals.append(cb["value"])
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GDOF/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "n_dof": prob.n_dof, "p": prob.p,
                       "elements": prob.E, "fields": prob.n_fields, "l2": "sampled rows (CPU)",
                       "value": "FP64 J(u)v rows of the oracle, GDOF/s"},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--solve-workload", default="cube16_p3")
    ap.add_argument("--reactor-workload", default="reactor_n2_p2",
                    help="workload of the batched 0.1-0.8 V sweep (reactor192_p2: the full "
                         "plate reactor, mixed precision only, about 13 minutes)")
    ap.add_argument("--reactor-only", default=None,
                    help="comma-separated labels of the batched sweep (fp64, mixed, "
                         "mixed_device_loop, mixed_sweep, mixed_paper_guess): run only the "
                         "batched 0.1-0.8 V sweep of --reactor-workload and print its record")
    ap.add_argument("--reactor-pc-lag", type=int, default=1,
                    help="preconditioner rebuilds every this many Newton iterations in the sweep")
    ap.add_argument("--reactor-shared-blocks", type=int, default=-1,
                    help=">= 0: one set of block inverses (of this operating point) for the "
                         "whole batch in the sweep (the memory strategy at p = 4)")
    ap.add_argument("--reactor-storage", default="f32", choices=["f32", "bf16"],
                    help="block-inverse storage of the mixed sweeps")
    ap.add_argument("--reactor-restart", type=int, default=50, help="FGMRES restart of the sweep")
    ap.add_argument("--reactor-parts", type=int, default=1,
                    help="solve the 8 operating points as this many consecutive batches (each "
                         "with its own per-point block inverses: the memory strategy at p = 4)")
    ap.add_argument("--channel-solve", type=int, default=0,
                    help="1: also solve channel64_p3 (3 species, 6.3M DOFs) to 1e-10, FP64 "
                         "(double-float arithmetic) and mixed (FP32 inner, BF16 inverses)")
    ap.add_argument("--only", default=None,
                    help="time one operator alone (for profiling): residual_f64, jvp_f64, "
                         "vjp_f64, residual_df32, jvp_df32, vjp_df32, jvp_f32, bj_apply_f32, "
                         "bj_setup_f32 (block-Jacobi setup: FP32 block columns and inversion); "
                         "no autotune, solves or e2e; or "
                         "fgmres_f64 / fgmres_f32: FGMRES(50) cycles with the two-level "
                         "preconditioner on the solve workload; precond_f32: block-Jacobi "
                         "against the downwind sweep on the solve workload (one application, "
                         "one linear solve to 1e-4)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2112_09271_gb300 as enp
    from paper_2112_09271_gb300 import dist as pdist
    import workloads as W

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    enp.build()
    if args.reactor_only:
        if rank == 0:
            t0 = time.perf_counter()
            parts = max(1, args.reactor_parts)
            volts = np.linspace(0.1, 0.8, 8)
            recs = []
            for part in np.array_split(volts, parts):
                recs.append(run_batched_solve(enp, W, args.reactor_workload, batch=len(part),
                                              volts=(float(part[0]), float(part[-1])),
                                              labels=tuple(args.reactor_only.split(",")),
                                              pc_lag=args.reactor_pc_lag,
                                              shared_blocks=args.reactor_shared_blocks,
                                              storage=args.reactor_storage,
                                              restart=args.reactor_restart))
            rec = recs[0] if parts == 1 else {"parts": recs}
            rec["wall_seconds"] = time.perf_counter() - t0
            print(json.dumps({"reactor_only": rec}), flush=True)
        return
    if args.only in ("fgmres_f64", "fgmres_f32"):
        if rank == 0:
            print(json.dumps(run_fgmres_profile(enp, W, args)), flush=True)
        return
    if args.only == "precond_f32":
        if rank == 0:
            print(json.dumps(run_precond_profile(enp, W, args)), flush=True)
        return
    prob = W.config(args.workload)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    op = enp.Operator(prob, stream=stream)
    n = op.n
    u = torch.tensor(W.random_state(prob, 2), device="cuda")
    v = torch.tensor(W.random_vector(prob, 3), device="cuda")
    w = torch.tensor(W.random_vector(prob, 4), device="cuda")
    u32, v32 = u.float(), v.float()
    r, jv, jtw, z = (torch.empty_like(u) for _ in range(4))
    jv32 = torch.empty_like(u32)
    cm = torch.empty(prob.E * prob.Np, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tuned = {}
    if args.only:
        if args.only == "bj_apply_f32":
            op.block_jacobi_setup(u, enp.BJ_F32)
    else:
        # launch shape per operator and arithmetic, before any timing
        for ar, code in (("f64", enp.ARITH_F64), ("df32", enp.ARITH_DF32)):
            op.set_arithmetic(code)
            op.autotune()
            tuned[ar] = op.launch_shapes()
        op.set_arithmetic(enp.ARITH_F64)
        op.block_jacobi_setup(u, enp.BJ_F32)   # preconditioner set up once, outside the steps
    fp64_ops = ["residual_f64", "jvp_f64", "vjp_f64", "residual_df32", "jvp_df32", "vjp_df32"]
    ops = fp64_ops + ["jvp_f32", "bj_apply_f32", "recover_cm", "inner_product"]
    applications = fp64_ops + ["jvp_f32", "bj_apply_f32"]
    if args.only:
        ops, applications = [args.only], [args.only]
    op_l = 2 if prob.dim == 3 else 1   # hexahedra: a face launch, then an element launch
    launches = {nm: op_l for nm in fp64_ops + ["jvp_f32"]}
    launches.update({"bj_apply_f32": 1, "recover_cm": 1, "inner_product": 2,
                     "bj_setup_f32": 3})  # FP32 copy of u, block columns, inversion
    launches_per_step = sum(launches[nm] for nm in ops)
    ip_out = np.zeros(1)

    def run_op(name):
        if name in fp64_ops:
            op.set_arithmetic(enp.ARITH_DF32 if name.endswith("_df32") else enp.ARITH_F64)
        kind = name.rsplit("_", 1)[0]
        if name in fp64_ops and kind == "residual":
            op.residual(u, out=r)
        elif name in fp64_ops and kind == "jvp":
            op.jvp(u, v, out=jv)
        elif name in fp64_ops and kind == "vjp":
            op.vjp(u, w, out=jtw)
        elif name == "jvp_f32":
            op.jvp_f32(u32, v32, out=jv32)
        elif name == "bj_apply_f32":
            op.block_jacobi_apply(v, out=z)
        elif name == "bj_setup_f32":
            op.block_jacobi_setup(u, enp.BJ_F32)  # block columns + inversion (synchronises)
        elif name == "recover_cm":
            op.recover_cm(u, out=cm)
        else:
            # enp_inner_product synchronises (it returns a host value): timed as its
            # device reduction (two launches) plus the copy of one double
            ip_out[:] = op.inner_product(jv, jv)

    ev = {nm: [torch.cuda.Event(enable_timing=True) for _ in range(2)] for nm in ops}
    t_ops = {nm: 0.0 for nm in ops}

    def step(timed):
        for nm in ops:
            if timed:
                ev[nm][0].record(stream)
            run_op(nm)
            if timed:
                ev[nm][1].record(stream)

    for _ in range(args.warmup):
        step(False)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    import tempfile
    cdir = os.environ.get("ENP_CLOCKS_DIR", tempfile.gettempdir())
    sampler = ClockSampler(local, os.path.join(cdir, f"clocks_rank{rank}.csv"))
    sampler.start()
    time.sleep(0.3)
    total_ms = 0.0
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        s0.record(stream)
        step(True)
        s1.record(stream)
        s1.synchronize()
        total_ms += s0.elapsed_time(s1)
        for nm in ops:
            t_ops[nm] += ev[nm][0].elapsed_time(ev[nm][1])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms_step = pdist.max_over_ranks(total_ms / args.steps, device="cuda")
    per_op = {nm: {"ms": t_ops[nm] / args.steps,
                   "GDOF_s": n / (t_ops[nm] / args.steps * 1e-3) / 1e9} for nm in ops}
    if args.only:
        if rank == 0:
            print(json.dumps({"only": args.only, "ops": per_op,
                              "kernel_hash": _kernel_hash(_family(args.only))}),
                  flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    # the headline: the FP64-accurate J v, in the faster of its two arithmetics
    ms_jv = {ar: pdist.max_over_ranks(t_ops["jvp_" + ar] / args.steps, device="cuda")
             for ar in ("f64", "df32")}
    head = min(ms_jv, key=ms_jv.get)
    head_op = "jvp_" + head
    value = world * n / (ms_jv[head] * 1e-3) / 1e9
    blend = world * n * len(applications) / (ms_step * 1e-3) / 1e9
    op.set_arithmetic(enp.ARITH_DF32 if head == "df32" else enp.ARITH_F64)

    # roofline of the headline kernel pair (face + element launch of J v): bound by
    # the arithmetic pipe it runs on; its HBM fraction alongside
    fl = contraction_flops(prob.dim, prob.p, prob.n_fields, "jvp") * prob.E * op.batch
    dom_s = ms_jv[head] * 1e-3
    hbm, hbm_kind = read_peaks()
    hbm_bytes = algorithmic_bytes_per_dof("jvp", 8) * n
    kh = _kernel_hash("operator")
    traffic = TRAFFIC.get((kh, head_op, prob.name))
    if head == "df32":
        peak = DF32_PEAK_TFLOPS
        peak_kind = ("derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 12 FP32 instructions per "
                     "double-float multiply-add x 2 flop")
        kname = f"face3d_kernel + op3d_kernel <p={prob.p},NF={prob.n_fields},jvp,df> (double-float)"
    else:
        peak = FP64_PEAK_TFLOPS
        peak_kind = "derived: 152 SMs x 2 FP64 FMA/clk x 2.07 GHz (measured FMA loop 1.20)"
        kname = f"face3d_kernel + op3d_kernel <p={prob.p},NF={prob.n_fields},jvp,double>"
    achieved = fl / dom_s / 1e12
    hbm_frac = hbm_bytes / dom_s / 1e9 / hbm
    roof = {"bound": "alu", "kernel": kname + " (one operator application = the two launches, "
                                              "timed together)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_kind": peak_kind, "traffic": traffic,
            "hbm_achieved_GBs": hbm_bytes / dom_s / 1e9, "hbm_peak_GBs": hbm,
            "hbm_frac": hbm_frac, "hbm_peak_kind": hbm_kind,
            "flops_per_launch": fl, "flops_kind": "sum-factorised contraction flops of the "
            "volume and the faces each element owns (pointwise physics excluded)",
            "algorithmic_bytes_per_launch": hbm_bytes}
    nb = prob.n_fields * prob.Np
    bj_bytes = prob.E * (nb * nb * 4 + 2 * nb * 8)  # FP32 inverse + FP64 x in, y out
    bj_s = t_ops["bj_apply_f32"] / args.steps * 1e-3
    roof_hbm = {"bound": "hbm", "kernel": "bj_apply_kernel<float,float,double>",
                "achieved": bj_bytes / bj_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bj_bytes / bj_s / 1e9 / hbm, "peak_kind": hbm_kind,
                "bytes_per_launch": bj_bytes,
                "traffic": TRAFFIC.get((_kernel_hash("solver"), "bj_apply_f32", prob.name))}
    f32_s = t_ops["jvp_f32"] / args.steps * 1e-3
    per_op["jvp_f32"]["fp32_TFLOPs"] = fl / op.batch / f32_s / 1e12
    per_op["jvp_f32"]["fp32_frac"] = fl / op.batch / f32_s / 1e12 / FP32_PEAK_TFLOPS
    per_op["jvp_f32"]["hbm_frac"] = algorithmic_bytes_per_dof("jvp", 4) * n / f32_s / 1e9 / hbm
    per_op["jvp_f32"]["traffic"] = TRAFFIC.get((kh, "jvp_f32", prob.name))
    for ar in ("f64", "df32"):
        t = t_ops["jvp_" + ar] / args.steps * 1e-3
        per_op["jvp_" + ar]["hbm_frac"] = hbm_bytes / t / 1e9 / hbm

    # end to end through the C ABI with host buffers, every step: H2D of u and v
    # (pinned), the FP64-accurate J v, D2H of the result
    hu, hv = (x.cpu().pin_memory() for x in (u, v))
    hj = torch.empty(n, dtype=torch.float64).pin_memory()
    du, dv = torch.empty_like(u), torch.empty_like(v)

    def e2e_step():
        du.copy_(hu, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        op.jvp(du, dv, out=jv)
        hj.copy_(jv, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_steps = max(3, args.steps // 2)
    s0.record(stream)
    for _ in range(e_steps):
        e2e_step()
    s1.record(stream)
    s1.synchronize()
    e2e_ms = pdist.max_over_ranks(s0.elapsed_time(s1) / e_steps, device="cuda")
    e2e = {"value": world * n / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8,
           "ms_per_step": e2e_ms, "arith": head}

    del flush
    solve = batched = solve_channel = None
    if rank == 0 and not args.no_solve:
        solve = run_solves(enp, W, args.solve_workload)
        full = args.reactor_workload.startswith("reactor192")
        batched = run_batched_solve(enp, W, args.reactor_workload,
                                    labels=("mixed", "mixed_device_loop", "mixed_sweep") if full
                                    else ("fp64", "mixed", "mixed_device_loop", "mixed_sweep",
                                          "mixed_paper_guess"))
        if args.channel_solve:
            solve_channel = run_solves(enp, W, "channel64_p3", labels=CHANNEL_SOLVE_VARIANTS,
                                       reference="fp64_df32_two_level")
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(prob)
    if rank == 0:
        solve_seconds = None
        if solve:
            solve_seconds = {k: solve[k]["seconds"] for k in solve
                             if isinstance(solve[k], dict) and "seconds" in solve[k]}
            solve_seconds["workload"] = solve["workload"]
        if solve_channel:
            solve_seconds = solve_seconds or {}
            solve_seconds["channel64_p3"] = {
                k: solve_channel[k]["seconds"] for k in solve_channel
                if isinstance(solve_channel[k], dict) and "seconds" in solve_channel[k]}
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 in/out; " + ("double-float (2 x f32) arithmetic" if head == "df32"
                                           else "f64 arithmetic"),
                "data": "synthetic",
                "config": {"workload": prob.name, "elements": prob.E, "p": prob.p,
                           "fields": prob.n_fields, "n_dof": prob.n_dof,
                           "n_dof_incl_cm": prob.n_dof // prob.n_fields * (prob.n_fields + 1),
                           "value": "FP64-accurate J(u)v, one application, GDOF/s (" + head +
                                    " arithmetic, the faster of f64 and df32)",
                           "step": "R, J v, J^T w in f64 and in df32 arithmetic, J v f32, "
                                   "block-Jacobi apply (FP32 inverses), c_m recovery, inner "
                                   "product",
                           "applications_per_step": len(applications),
                           "tile_shapes": {ar: {nm: {"elements_per_block": eb, "faces_per_block": fb}
                                                for nm, eb, fb in zip(["residual", "jvp", "vjp",
                                                                       "jvp_f32", "residual_f32"],
                                                                      t[0], t[1])}
                                           for ar, t in tuned.items()},
                           "l2": "flushed between steps (512 MB write)"},
                "jvp_GDOF_s": {"f64": n / (ms_jv["f64"] * 1e-3) / 1e9,
                               "df32": n / (ms_jv["df32"] * 1e-3) / 1e9,
                               "f32": per_op["jvp_f32"]["GDOF_s"]},
                "hbm_frac": hbm_frac, "solve_seconds": solve_seconds,
                "step_blend_GDOF_s": blend,
                "ops": per_op, "roofline": roof, "roofline_hbm": roof_hbm, "solve": solve,
                "solve_channel": solve_channel,
                "batched_solve": batched,
                "cpu_baseline": cb, "e2e": e2e,
                "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
                "kernel_hash": kh}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
