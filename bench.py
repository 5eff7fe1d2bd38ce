"""Benchmark of the FETI hot path on GB300: dual-operator applies/s and PCG time-to-tolerance.

Workload (default): all-floating FETI, linear elasticity (E = 1, nu = 0.3) on
the thick-walled tube r in [1, 1.5], length 2, 32 x 128 x 64 cells split into
P1 tetrahedra with nodes jittered by +-0.2 cells (274,560 nodes, 823,680
DOFs), recursive coordinate bisection with jittered cuts into 1024 uneven
subdomains, Dirichlet preconditioner, internal pressure 0.01, PCG to 1e-8
(synthetic inputs, seeded generator): the FP32-local against the FP64 form.

A step = one block of `n_apply` back-to-back dual-operator applies
(q = F v, z = M^-1 q) on device-resident vectors; value = applies/s over all
ranks.  The local operators F_i and S_i read per apply (GBs) exceed the 129 MB
L2, so no flush is needed between steps.  The whole solve (setup + projected
PCG to 1e-8 + recovery) is timed separately and reported in the same line.

--impl reference times the FP64 CPU oracle on the host cores on the same
workload and metric (the paper has no GPU code to run).
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

METRIC = "dual-operator F·λ+precond applies/s & PCG time to 1e-8, FP32-local vs FP64"
UNIT = "applies/s"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (every rank calls it); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes per F_i apply of the dominant FP32 kernel, from the ncu capture in
# profiles/k_symv3_f32_traffic_jittered_tube_16x64x32_128sub.md (128 subdomains
# of the same size mix, dram__bytes_read.sum + dram__bytes_write.sum of the
# second F_i launch = 1.075 x the algorithmic bytes there), scaled by the
# algorithmic bytes of the workload; only for the kernel variant captured.
TRAFFIC_RATIO = {"k_symv3_f32<32>": 1.075}


def cpu_baseline(prob, n_apply: int, budget_s: float = 20.0) -> dict:
    """The FP64 oracle's dual apply on the host cores (bounded sample)."""
    import numpy as np
    from oracle import feti as ofeti
    o = ofeti.FetiOracle(prob, "af", "dirichlet")
    o.assemble()
    o.factorize()
    v = np.random.default_rng(1).normal(size=o.n_lambda)
    t0 = time.perf_counter()
    done = 0
    while done < n_apply:
        q = o.apply_F(v)
        o.apply_prec(q)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} dual applies (F v then M^-1 q, dense LAPACK solves per subdomain) on the "
                      f"full workload after an untimed oracle setup; numpy/BLAS threads on {cores} cores"}


def run_reference(args, prob, workload_cfg):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import numpy as np
    from oracle import feti as ofeti
    t0 = time.perf_counter()
    o = ofeti.FetiOracle(prob, "af", "dirichlet")
    o.assemble()
    o.factorize()
    setup = time.perf_counter() - t0
    v = np.random.default_rng(1).normal(size=o.n_lambda)
    for _ in range(args.warmup):
        o.apply_prec(o.apply_F(v))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.apply_prec(o.apply_F(v))
    dt = time.perf_counter() - t0
    val = args.steps / dt
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_cfg,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one dual apply per step on the full workload; oracle setup "
                                       f"{setup:.1f} s untimed"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-apply", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="jcyl32", choices=["jcyl32", "cyl16", "cyl8", "jcyl16", "jcyl48"],
                    help="jcyl32: jittered tube, 1024 uneven subdomains (default); cyl16: the 64-subdomain "
                         "tube; cyl8: a 32-subdomain tube for profiler captures; jcyl16: jittered tube with "
                         "128 subdomains of the same size mix as jcyl32, for profiler captures; jcyl48: "
                         "jittered tube, 4096 uneven subdomains")
    ap.add_argument("--symmetric", default="auto", choices=["auto", "off", "force", "force_streamed", "force_cta"],
                    help="FP32 local applies: autotuner choice, full rows, or the symmetric panel kernel (pin it "
                         "for profiler runs, where serialised launches change the autotuner's timings)")
    ap.add_argument("--plain", type=int, default=1,
                    help="also time the plain FP64 form with one local-apply launch per subdomain (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--coarse", default="auto", choices=["auto", "dense", "sparse"],
                    help="coarse problem: dense inverse, supernodal sparse Cholesky, or automatic")
    ap.add_argument("--fp32-form", default="mixed", choices=["mixed", "f32factor"],
                    help="precision form of the timed FP32-local applies: FP64 factors rounded to FP32 operators "
                         "(mixed, default) or FP32 factorizations (f32factor: half the device memory, for profiler "
                         "captures); the applies run the same kernels")
    ap.add_argument("--f32factor", type=int, default=1,
                    help="also run the form with FP32 local factorizations and refined K^+ (0: skip)")
    ap.add_argument("--implicit", type=int, default=1, help="also measure the implicit FP64 local form (0: skip)")
    ap.add_argument("--block", type=int, default=1, help="also measure the 16-RHS block form (0: skip)")
    ap.add_argument("--block-fp64", type=int, default=1, help="include the FP64 16-RHS block leg (0: skip)")
    ap.add_argument("--elements", type=int, default=1,
                    help="also time the hyperelastic element kernel on the 256-subdomain tube (0: skip)")
    ap.add_argument("--elements-only", action="store_true",
                    help="only the element-kernel leg: for profiler captures")
    ap.add_argument("--apply-only", action="store_true",
                    help="setup only (no PCG solve) before the timed applies: for profiler captures")
    ap.add_argument("--solve-only", default=None, choices=["fp64", "mixed", "mixed_f32factor"],
                    help="one untimed solve, then one complete create + setup + solve of this precision "
                         "form inside the NVTX range 'timed': for profiler launch lists")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    from feti_inputs import mesh
    if args.workload == "cyl16":
        prob = mesh.config_problem("cyl16")
        wname = ("AF-FETI tube 16x64x32 cells P1 (35,904 nodes, 107,712 DOFs), 64 wedge subdomains, "
                 "Dirichlet preconditioner, FP64, PCG tol 1e-8")
    elif args.workload == "jcyl32":
        prob = mesh.config_problem("jcyl32")
        wname = ("AF-FETI jittered tube 32x128x64 cells P1 (274,560 nodes, 823,680 DOFs), 1024 uneven "
                 "subdomains (jittered RCB), Dirichlet preconditioner, PCG tol 1e-8")
    elif args.workload == "jcyl16":
        prob = mesh.config_problem("jcyl16")
        wname = ("AF-FETI jittered tube 16x64x32 cells P1 (35,904 nodes), 128 uneven subdomains (jittered RCB, "
                 "the subdomain size mix of the 1024-subdomain tube), Dirichlet preconditioner, PCG tol 1e-8 "
                 "(profiler-sized)")
    elif args.workload == "jcyl48":
        prob = mesh.config_problem("jcyl48")
        wname = ("AF-FETI jittered tube 48x192x96 cells P1 (912,576 nodes, 2,737,728 DOFs), 4096 uneven "
                 "subdomains (jittered RCB), Dirichlet preconditioner, PCG tol 1e-8")
    else:
        prob = mesh.cylinder_problem(8, 64, 16, (2, 8, 2))
        wname = ("AF-FETI tube 8x64x16 cells P1 (9,792 nodes), 32 wedge subdomains, Dirichlet "
                 "preconditioner, FP64, PCG tol 1e-8 (profiler-sized)")
    workload_cfg = {"workload": wname,
                    "n_subdomains": prob.n_parts, "n_dofs": 3 * prob.n_nodes, "method": "all-floating",
                    "precond": "dirichlet", "precision": "fp64", "l2": "inputs larger than L2 (the F_i and S_i read per apply exceed the 129 MB L2)",
                    "parallelism": "replicas" if args.gpus > 1 else "single"}
    if args.impl == "reference":
        run_reference(args, prob, workload_cfg)
        return

    import torch
    import torch.distributed as dist
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1508_02599_gb300 import FetiSolver

    stream = torch.cuda.Stream()            # a real stream: the library captures graphs on it
    torch.cuda.set_stream(stream)
    peaks, src = _peaks()
    fp64_peak = 1.259  # TFLOP/s: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz

    def measure(precision: str, batched: bool = True, n_apply: int = 0, steps: int = 0, local_form: str = "auto"):
        """Full solve once, then `steps` timed blocks of n_apply dual applies."""
        n_apply = n_apply or args.n_apply
        steps = steps or args.steps
        solver = FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, coarse=args.coarse,
                            stream=stream.cuda_stream, precision=precision, batched=batched,
                            symmetric=args.symmetric, local_form=local_form)
        if args.apply_only:
            solver.prepare()
            U, rep = np.zeros(3 * prob.n_nodes), {"t_pcg_ms": None, "iterations": 0, "outer_iterations": 0,
                                                  "cond_est": None, "t_setup_ms": None}
        else:
            U, rep = solver.solve()      # full hot path once: setup + PCG + recovery
        sizes = solver.sizes()
        sizes["coarse"] = solver.coarse_info()
        sizes["factor"] = solver.factor_info()
        nl = sizes["n_lambda"]
        g = torch.Generator(device="cuda").manual_seed(1234 + rank)
        v = torch.randn(nl, dtype=torch.float64, device="cuda", generator=g)
        q = torch.empty_like(v)
        z = torch.empty_like(v)
        for _ in range(args.warmup):
            solver.dual_apply(v, q, z, n_apply)
        clocks = ClockSampler(local)
        clocks.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        kern_ms = []
        torch.cuda.nvtx.range_push("timed")      # profiler filter: the timed applies only
        for _ in range(steps):
            solver.dual_apply(v, q, z, n_apply)
            kern_ms.append(solver.kernel_stats()["gemv_ms"])
        torch.cuda.nvtx.range_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = _max_over_ranks(ev0.elapsed_time(ev1), world, "cuda")
        clk = clocks.stop()
        ks = solver.kernel_stats()
        sched = solver.schedule()
        kern = statistics.mean(kern_ms)
        solver.close()
        return {"U": U, "rep": rep, "sizes": sizes, "ms": ms, "kern_ms": kern, "ks": ks, "clocks": clk, "sched": sched,
                "value": _job_rate(steps * n_apply, world, ms / 1e3), "steps": steps}

    def measure_block(precision: str, nrhs: int = 16):
        """Block form: nrhs load cases p_k ~ U[8, 16] x the reference pressure (seeded), one block
        PCG to 1e-8, then timed blocks of block dual applies (RHS-applies/s)."""
        rng = np.random.Generator(np.random.PCG64(16))
        scales = rng.uniform(8.0, 16.0, size=nrhs)
        solver = FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, coarse=args.coarse,
                            stream=stream.cuda_stream, precision=precision)
        U, rep = solver.solve_multi(scales)
        nl = solver.sizes()["n_lambda"]
        g = torch.Generator(device="cuda").manual_seed(99 + rank)
        V = torch.randn((nl, nrhs), dtype=torch.float64, device="cuda", generator=g)
        Q = torch.empty_like(V)
        Z = torch.empty_like(V)
        n_ap = max(1, args.n_apply // 8)
        for _ in range(args.warmup):
            solver.dual_apply_multi(V, Q, Z, nrhs, n_ap)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        kern = []
        for _ in range(args.steps):
            solver.dual_apply_multi(V, Q, Z, nrhs, n_ap)
            kern.append(solver.kernel_stats()["gemv_ms"])
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        ks = solver.kernel_stats()
        km = statistics.mean(kern)
        sched = solver.schedule()
        solver.close()
        return {"rhs_applies_per_s": nrhs * args.steps * n_ap / (ms / 1e3), "nrhs": nrhs,
                "gemm_schedule": sched["block_fp32_F"] if precision == "mixed" else None,
                "pcg_time_to_tol_ms": rep["t_pcg_ms"], "iterations": rep["iterations"],
                "outer_iterations": rep["outer_iterations"], "converged": rep["converged"],
                "gemm_kernel_ms": km, "gemm_gbs": ks["gemv_bytes"] / (km / 1e3) / 1e9,
                "gemm_tflops": ks["gemv_flops"] / (km / 1e3) / 1e12, "U": U, "scales": scales}

    def measure_elements():
        """Element tangents + internal forces of the two-fibre hyperelastic model (Table 1) on the
        24x96x48-cell tube (663,552 tets), at a 5 % radial expansion (fibres stretched, active)."""
        ep = mesh.config_problem("cyl24_hgo")
        U = np.zeros((ep.n_nodes, 3))
        U[:, :2] = 0.05 * ep.coords[:, :2]
        solver = FetiSolver(ep, method="af", precond="dirichlet", stream=stream.cuda_stream)
        dU = torch.tensor(U.ravel(), device="cuda")
        Ke = torch.empty((ep.tets.shape[0], 12, 12), dtype=torch.float64, device="cuda")
        fe = torch.empty((ep.tets.shape[0], 12), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            solver.elements(dU, out=(Ke, fe))
        ms = []
        for _ in range(max(3, args.steps // 4)):
            solver.elements(dU, out=(Ke, fe))
            ms.append(solver.element_stats()["elem_ms"])
        st_ = solver.element_stats()
        solver.close()
        kms = statistics.median(ms)
        gbs = st_["elem_bytes"] / (kms / 1e3) / 1e9
        return {"workload": "tube 24x96x48 cells P1, 663,552 tets, two-fibre hyperelastic (Table 1), U = 5 % "
                            "radial expansion", "kernel": "k_elem_hgo", "kernel_ms": kms,
                "elements_per_s": st_["n_elements"] / (kms / 1e3), "achieved_gbs": gbs,
                "hbm_frac": gbs / peaks["hbm_gbs"], "algorithmic_bytes": st_["elem_bytes"],
                "bound": "alu (FP64); ncu FP64-pipe share in profiles/"}

    if args.solve_only:
        def one_solve():
            with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, coarse=args.coarse,
                            stream=stream.cuda_stream, precision=args.solve_only) as s_:
                return s_.solve()[1]
        one_solve()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        rep_ = one_solve()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"solve_only": args.solve_only, "workload": wname,
                              **{k: rep_[k] for k in ("iterations", "outer_iterations", "t_setup_ms", "t_pcg_ms")}}),
                  flush=True)
        return
    if args.elements_only:
        el = measure_elements()
        if rank == 0:
            print(json.dumps({"elements": el}), flush=True)
        return
    def measure_f32factor():
        """FP32 local factorizations with FP64-refined K^+: setup and PCG to 1e-8 (the dual applies
        run the same FP32 operator kernels as the FP32-local form)."""
        solver = FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, coarse=args.coarse,
                            stream=stream.cuda_stream, precision="mixed_f32factor", symmetric=args.symmetric)
        U, rep = solver.solve()
        ref = solver.refinement()
        solver.close()
        return {"U": U, "rep": rep, "refine": ref}

    m64 = measure("fp64")
    m32 = measure("mixed" if args.fp32_form == "mixed" else "mixed_f32factor")
    mf = measure_f32factor() if args.f32factor else None
    # the plain FP64 form: the same kernels with the local applies launched once
    # per subdomain (p launches per apply instead of one batched launch)
    mp = (measure("fp64", batched=False, n_apply=max(1, args.n_apply // 4), steps=max(1, args.steps // 4))
          if args.plain else None)
    # the implicit FP64 form: F_i v by forward and backward sweeps over the local factor
    mi = (measure("fp64", n_apply=max(1, args.n_apply // 4), steps=max(1, args.steps // 4), local_form="implicit")
          if args.implicit else None)
    b64 = measure_block("fp64") if args.block and args.block_fp64 else None
    b32 = measure_block("mixed") if args.block else None
    n64 = np.linalg.norm(m64["U"])
    err = float(np.linalg.norm(m32["U"] - m64["U"]) / n64) if n64 > 0 else None
    ks32, ks64 = m32["ks"], m64["ks"]
    gbs32 = ks32["gemv_bytes"] / (m32["kern_ms"] / 1e3) / 1e9
    tf64 = ks64["gemv_flops"] / (m64["kern_ms"] / 1e3) / 1e12
    gbs64 = ks64["gemv_bytes"] / (m64["kern_ms"] / 1e3) / 1e9

    # end to end through the public API with host buffers: create (H2D of the
    # problem) + solve (mixed form) + D2H of the displacement, per step
    e2e_steps = args.e2e_steps
    u_host = torch.empty(3 * prob.n_nodes, dtype=torch.float64).pin_memory()

    def e2e_rate(precision):
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        its = 0
        for _ in range(e2e_steps):
            with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, coarse=args.coarse,
                            stream=stream.cuda_stream, precision=precision) as s2:
                r2 = s2.solve_host(u_host)
                its += r2["iterations"] + r2["outer_iterations"] + 2
        dt = time.perf_counter() - t0
        if world > 1:
            dist.barrier()
        return its, _max_over_ranks(dt, world, "cuda")

    e2e_forms = {}
    for form in (["mixed_f32factor"] if mf is not None else []) + ["mixed"]:
        its_f, dt_f = e2e_rate(form) if e2e_steps else (0, 1.0)
        e2e_forms[form] = {"value": _job_rate(its_f, world, dt_f) if e2e_steps else None,
                           "s_per_solve": dt_f / max(e2e_steps, 1)}
    e2e_form = max(e2e_forms, key=lambda k: e2e_forms[k]["value"] or 0.0)
    h2d = (prob.coords.nbytes + prob.tets.nbytes + prob.part.nbytes + prob.dir_dof.nbytes + prob.dir_val.nbytes
           + prob.press_tri.nbytes + prob.press_owner.nbytes)
    e2e = {"value": e2e_forms[e2e_form]["value"], "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(u_host.numel() * 8), "form": e2e_form, "forms": e2e_forms,
           "note": "dual applies of complete solves (create + setup + PCG to 1e-8 + recovery) per second of wall "
                   "time through feti_create/feti_solve, problem arrays from host, displacement back to pinned "
                   "host; value = the faster precision form (both listed)"}

    if rank == 0:
        r64, r32 = m64["rep"], m32["rep"]
        line = {
            "metric": METRIC, "value": m32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m32["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_cfg, precision="FP32 local operators, FP64 vectors/projection/coarse/outer "
                                                    "residual", n_apply_per_step=args.n_apply,
                           n_lambda=m32["sizes"]["n_lambda"], coarse_dim=m32["sizes"]["coarse_dim"],
                           coarse=m32["sizes"]["coarse"],
                           local_factor_storage={k: {**v, "workspace_gb": v["workspace"] * v["elem_bytes"] / 1e9,
                                                     "full_workspace_gb": v["full_workspace"] * v["elem_bytes"] / 1e9,
                                                     "compact_gb": v["compact"] * v["elem_bytes"] / 1e9}
                                                 for k, v in (("fp32_local", m32["sizes"]["factor"]),
                                                              ("fp64", m64["sizes"]["factor"]))}),
            "pcg": {"tol": 1e-8,
                    "fp32_local": {"time_to_tol_ms": r32["t_pcg_ms"], "inner_iterations": r32["iterations"],
                                   "outer_iterations": r32["outer_iterations"], "rel_err_vs_fp64": err},
                    "fp64": {"time_to_tol_ms": r64["t_pcg_ms"], "iterations": r64["iterations"],
                             "cond_est": r64["cond_est"]},
                    "setup_ms": r64["t_setup_ms"]},
            "fp32_factor": None if mf is None else {
                "time_to_tol_ms": mf["rep"]["t_pcg_ms"], "setup_ms": mf["rep"]["t_setup_ms"],
                "inner_iterations": mf["rep"]["iterations"], "outer_iterations": mf["rep"]["outer_iterations"],
                "refine_steps": mf["refine"]["steps"], "refine_residual": mf["refine"]["residual"],
                "rel_err_vs_fp64": (float(np.linalg.norm(mf["U"] - m64["U"]) / np.linalg.norm(m64["U"]))
                                    if np.linalg.norm(m64["U"]) > 0 else None),
                "note": "FP32 local factorizations (F_i, S_i from the FP32 elimination) with FP64-refined K^+ "
                        "for d~, the outer residual and the recovery; same FP32 operator kernels per apply"},
            "fp64": {"value": m64["value"], "unit": UNIT, "ms_per_step": m64["ms"] / args.steps,
                     "roofline": {"bound": "alu", "kernel": "k_gemv_loc<double> (F_i apply)", "achieved": tf64,
                                  "peak": fp64_peak, "unit": "TFLOP/s", "frac": tf64 / fp64_peak,
                                  "hbm_gbs": gbs64, "kernel_ms": m64["kern_ms"]},
                     "clocks": m64["clocks"]},
            "fp64_per_subdomain": None if mp is None else {
                "value": mp["value"], "unit": UNIT, "ms_per_step": mp["ms"] / mp["steps"],
                "time_to_tol_ms": mp["rep"]["t_pcg_ms"], "iterations": mp["rep"]["iterations"],
                "local_apply_kernel_ms": mp["kern_ms"],
                "note": "plain form: FP64, one local-apply launch per subdomain instead of one batched launch; "
                        "same kernels, graphs and schedule"},
            "fp64_implicit": None if mi is None else {
                "value": mi["value"], "unit": UNIT, "ms_per_step": mi["ms"] / mi["steps"],
                "time_to_tol_ms": mi["rep"]["t_pcg_ms"], "iterations": mi["rep"]["iterations"],
                "local_apply_ms": mi["kern_ms"],
                "note": "implicit local form: each F_i v is a forward and a backward sweep over the FP64 "
                        "local Cholesky factor on the placed boundary vector (gather, place, sweeps, boundary "
                        "take); local_apply_ms spans those launches per apply"},
            "roofline": {"bound": "hbm",
                         "kernel": ("k_symv2_f32 + k_symv_fix (F_i apply, FP32 lower block-triangle, streamed)"
                                    if m32["sched"]["fp32_F"][0] == -64 else
                                    "k_symv3_f32<%d> (F_i apply, FP32 lower block-triangle, one CTA per subdomain)"
                                    % (-m32["sched"]["fp32_F"][0] - 300)
                                    if m32["sched"]["fp32_F"][0] <= -300 else
                                    "k_symv_f32 + k_symv_fix (F_i apply, FP32 lower block-triangle)"
                                    if m32["sched"]["fp32_F"][0] < 0 else "k_gemv_loc<float> (F_i apply, FP32 copy)"),
                         "achieved": gbs32,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs32 / peaks["hbm_gbs"],
                         "traffic": (TRAFFIC_RATIO["k_symv3_f32<32>"] * ks32["gemv_bytes"]
                                     if m32["sched"]["fp32_F"][0] == -332 else None),
                         "traffic_note": "dram read+write per launch from an ncu capture of the same kernel on "
                                         "128 subdomains of the same size mix, scaled by algorithmic bytes "
                                         "(profiles/k_symv3_f32_traffic_jittered_tube_16x64x32_128sub.md); null "
                                         "for a kernel variant that was not captured",
                         "kernel_ms": m32["kern_ms"], "algorithmic_bytes": ks32["gemv_bytes"],
                         "bytes_note": "n(n+1)/2 distinct FP32 entries per symmetric F_i + 16 B per boundary DOF",
                         "peak_source": src},
            "clocks": m32["clocks"],
            "schedule": {"fp32_F": m32["sched"]["fp32_F"], "fp32_M": m32["sched"]["fp32_M"],
                         "fp64_F": m64["sched"]["fp64_F"], "fp64_M": m64["sched"]["fp64_M"],
                         "meaning": "[rows per warp step, rows per CTA] picked by the setup-time autotuner"},
            "e2e": e2e,
            # per dual apply: gather, local apply, scatter for F and for M; a symmetric
            # local apply is two launches (panel kernel, fixed-order partial sum)
            "gpu_launches": args.steps * args.n_apply * (6 + sum(1 for k in ("fp32_F", "fp32_M")
                                                                 if -300 < m32["sched"][k][0] < 0)),
        }
        if b32 is not None:
            blk = {}
            for name, b in (("fp32_local", b32), ("fp64", b64)):
                if b is None:
                    continue
                # u_k = s_k u for these load cases: check against the single-RHS FP64 solution
                errs = [float(np.linalg.norm(b["U"][k] - b["scales"][k] * m64["U"]) /
                              np.linalg.norm(b["scales"][k] * m64["U"])) for k in range(b["nrhs"])]
                blk[name] = {k: v for k, v in b.items() if k not in ("U", "scales")}
                blk[name]["max_rel_err_vs_single_fp64"] = max(errs)
            blk["fp32_local"]["gemm_hbm_frac"] = blk["fp32_local"]["gemm_gbs"] / peaks["hbm_gbs"]
            blk["note"] = ("16 load cases (pressure x U[8,16], seeded) solved as one block: every dense F_i/S_i "
                           "entry read feeds 16 products; rhs_applies_per_s counts right-hand sides")
            line["block16"] = blk
        if args.elements:
            line["elements"] = measure_elements()
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(prob, n_apply=20)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
