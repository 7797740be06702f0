"""Benchmark of the macro-element HDG hot path on one GB300: time per Newton step of the
DIRK3 integration of the 3D Taylor-Green vortex (periodic [0, 2 pi]^3, 16^3 macro-elements
of 2^3 hexes, p = 2, Re 1600, M0 0.1, dt = 0.05 t_c), FGMRES iterations per step and
batched local LU TFLOP/s.

A "step" is one Newton step of a DIRK stage (Sec. 3.1, eq. C242): assembly of the
residuals and Newton blocks, second-layer condensation and batched LU, FGMRES on the
trace system, local recovery, the state update and the assembly at the new state
(plus, when a step opens a stage, the assembly of the stage's first residual).  Each
step is one mehdg_newton_step call of the library (mehdg_stage_begin / mehdg_stage_end
open and close the stages; three stages make a DIRK step).  The value is the plain FP64
form; the same line reports the mixed-precision form and the learned preconditioner
correction on the same integration, each at the same 1e-8 relative Newton residual.
Inputs (about 150 GB of blocks per step) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                  [--workload tgv|mms|batched] [--impl ours|reference]

--impl reference times the FP64 numpy oracle on the host cores for the same metric on a
bounded sample of the same workload (it prints what it ran and how it was scaled).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "time per Newton/DIRK step & FGMRES iters at 1e-8 residual; batched local LU TFLOP/s"
MIXED_DETAIL = ("f32 blocks, Jacobians and local products; bf16 operator copies in the inner GMRES; "
                "f64 residuals, Krylov vectors and refinement residuals")
UNIT = "s/Newton step"
UNIT_TGV = "s/Newton step"
WORKLOAD_TGV = ("3D Taylor-Green vortex, periodic [0,2pi]^3, Re 1600, M0 0.1, %d^3 macro-elements x 2^3 hexes, "
                "p=2 (%d^3 = %d macros, Nu=625, Nt=750, %d trace DOFs), DIRK3 dt = 0.05 t_c, Newton steps")
WORKLOAD_SPHERE = ("flow past a sphere, Re 100, Mach 0.3: cubed-sphere shell 0.5 <= r <= 10, 6 x %d^2 x %d curved "
                   "macro-elements (layer ratio 1.15) x 2^3 hexes, p=2 (%d macros, Nu=625, Nt=750, %d trace DOFs), "
                   "isothermal wall + characteristic far field, DIRK3 dt = 0.1 (acoustic units) from the blended "
                   "free stream, Newton steps")


NMAC = 8

# DRAM bytes (read + write) per macro-element and launch of the apply kernels, from an ncu
# capture of the 6^3 manufactured-solution cube (216 macros), scaled by the macro count;
# keyed by (phase, precision, apply_mode).  A kernel without
# a capture of its current version has no entry (its traffic is reported as null).
TRAFFIC_PER_MACRO = {("apply", "mixed", 1): (489.032960e6 + 4.069632e6) / 216}


def workload():
    return W.mms(dim=3, nmac=NMAC, m=2, p=2)


def sizes(pr):
    z = W.sizes(pr)
    z["Nu"] = z["ns"] * z["Np"]
    z["Nt"] = z["ns"] * z["Nth"]
    return z


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lrk = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lrk


def rank_barrier(ws):
    """All ranks meet here (no-op on one rank)."""
    if ws > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(x, ws, device=None):
    """The largest x over the ranks (x itself on one rank): a timed region of the
    replicas ends when the slowest rank ends.  device: where the collective's tensor
    lives (the rank's GPU for NCCL, None = CPU for gloo)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws, device=None):
    """The sum of x over the ranks (x itself on one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


def replica_value(seconds_per_step_max, ws):
    """Whole-job time per step of N independent replicas (weak scaling): N steps, one
    per rank, complete in the slowest rank's time per step."""
    return seconds_per_step_max / max(1, ws)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        try:
            sm = [float(r[1]) for r in self.rows if r[1] not in ("", "[N/A]")]
            mx = [float(r[2]) for r in self.rows if r[2] not in ("", "[N/A]")]
            if sm:
                out["sm_mhz"] = float(np.median(sm))
            if mx:
                out["sm_max_mhz"] = max(mx)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for i, n in enumerate(names):
                if any(r[5 + i].lower().startswith("active") for r in self.rows if len(r) > 5 + i):
                    out["reasons"].append(n)
        except (ValueError, IndexError):
            pass
        return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def fp64_peak_tflops(torch):
    """Measured FP64 dense rate on this GPU: cuBLAS DGEMM 4096^3, best of 5 (CUDA events)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 1e9
    for _ in range(5):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        torch.matmul(a, b)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


def phase_work(z, E, precision, apply_mode=0):
    """Algorithmic FLOPs (and bytes for the apply) per launch of the main phases.

    Apply bytes per macro-element: the stored operators read once (Algorithm 2: C, S
    factors, B, D; apply_mode 1: the local operator A^T_i), plus the gathered input
    (8 B), the slot written (8 B) and the gather indices (4 B) per trace entry."""
    Nu, Nt, Np, Nth, d, ns = z["Nu"], z["Nt"], z["Np"], z["Nth"], z["d"], z["ns"]
    w = 8 if precision == "fp64" else 4
    cond = 2.0 * d * ns * (Nu * Np * Np + Nu * Np * Nth + Nt * Np * Np + Nt * Np * Nth) * E
    lu = (2.0 / 3.0) * Nu ** 3 * E
    if apply_mode == 1:
        apply_bytes = (w * Nt * Nt + (8 + 8 + 4) * Nt) * E
        apply_flops = 2.0 * Nt * Nt * E
    else:
        apply_bytes = (w * (2 * Nu * Nt + Nt * Nt + Nu * Nu) + (8 + 8 + 4) * Nt + 4 * Nu) * E
        apply_flops = 2.0 * (2 * Nu * Nt + Nt * Nt + Nu * Nu) * E
    return dict(condense_flops=cond, lu_flops=lu, apply_bytes=apply_bytes, apply_flops=apply_flops)


def newton_solve(ctx, state, tol=1e-8, max_steps=60, record=False):
    """Steady pseudo-transient Newton/SER solve through the C ABI (one call per phase).

    Returns statistics and, when record is set, the input state and pseudo-time step
    of every Newton step (for replay)."""
    import torch
    u, q, uh = (t.clone() for t in state)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    records = []
    tau_init, tau_max = 1.0, 1e8
    its = 0
    status = 0
    e0.record(st)
    norms = ctx.assemble(u, q, uh)
    R0 = norms[3]
    dtau = tau_init
    steps = 0
    while norms[3] > tol * R0 and steps < max_steps:
        if record:
            records.append((u.clone(), q.clone(), uh.clone(), dtau))
        bhat = ctx.condense(shift=1.0 / dtau)
        duh_s, stats = ctx.linear_solve(bhat, allow_not_converged=True)
        its += stats["fgmres_iters"]
        status |= stats["status"]
        dU, dQ = ctx.recover(duh_s)
        u += dU
        q += dQ
        uh += duh_s
        RU_old = norms[1]
        norms = ctx.assemble(u, q, uh)
        dtau = min(max(dtau * RU_old / max(norms[1], 1e-300), tau_init), tau_max)
        steps += 1
    e1.record(st)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    return dict(newton_steps=steps, fgmres_iters=its, converged=bool(norms[3] <= tol * R0), time_s=t,
                s_per_step=t / max(steps, 1), res0=float(R0), res=float(norms[3]), fallback=bool(status & 1),
                records=records, state=(u, q, uh))


def run_ours(args, ws, rank, lrank):
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg

    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    pr = workload()
    z = sizes(pr)
    prec = pkg.PREC_MIXED if args.precision == "mixed" else pkg.PREC_FP64
    base = dict(restart=args.restart, max_iters=3000, lin_rtol=args.lin_rtol, newton_rtol=1e-8, max_newton=60,
                inner_iters=args.inner, tc_mode=args.tc_mode, refine_iters=args.refine)
    opts = dict(base, precision=prec, precond=args.precond, apply_mode=args.apply_mode,
                precond_bf16=args.precond_bf16 if prec == pkg.PREC_MIXED else 0)
    ctx = pkg.Context(pr, opts, device=dev)
    du, duh = W.perturbation(pr, 0)
    du_d = torch.as_tensor(du, device=dev)
    duh_d = torch.as_tensor(duh, device=dev)
    state0 = ctx.init_state(du_d, duh_d, lift=True)
    st = torch.cuda.current_stream(dev)
    learn = args.compare and args.precision == "mixed"
    if learn:
        ctx.mlp_setup(hidden=256, seed=0, max_pairs=512)
        ctx.mlp_set_recording(True)

    # ---- warm-up: the whole steady solve, recording every Newton step's input
    sol = newton_solve(ctx, state0, record=True, max_steps=args.solve_steps)
    records = sol["records"]
    N = len(records)
    assert N > 0
    u, q, uh = sol["state"]
    its_total = sol["fgmres_iters"]
    if learn:
        n_samples = ctx.mlp_set_recording(False)

    def replay(k, host=None):
        u0, q0, uh0, dt_ = records[k % N]
        if host is not None:
            hu, hq, huh = host[k % N]
            u.copy_(hu, non_blocking=True)
            q.copy_(hq, non_blocking=True)
            uh.copy_(huh, non_blocking=True)
        else:
            u.copy_(u0)
            q.copy_(q0)
            uh.copy_(uh0)
        ctx.assemble(u, q, uh)
        bhat = ctx.condense(shift=1.0 / dt_)
        duh_s, stats = ctx.linear_solve(bhat, allow_not_converged=True)
        dU, dQ = ctx.recover(duh_s)
        u.add_(dU)
        q.add_(dQ)
        uh.add_(duh_s)
        return stats["fgmres_iters"]

    for k in range(max(0, args.warmup - N)):
        replay(k)
    torch.cuda.synchronize()
    if args.steps < 0:
        args.steps = N

    # ---- timed region (device-resident inputs)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(lrank)
    clk.start()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phase_acc = {}
    its_timed = 0
    ev0.record(st)
    for k in range(args.steps):
        its_timed += replay(k)
        ph = ctx.phase_times() if args.phases else {}
        for key, v in ph.items():
            phase_acc.setdefault(key, []).append(v)
    ev1.record(st)
    torch.cuda.synchronize()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    launches = ctx.launch_count() - l0
    clocks = clk.stop()
    t_dev = max_over_ranks(t_dev, ws, dev)
    rank_barrier(ws)

    # ---- e2e: host (pinned) buffers in, state out, per step
    host = [(r[0].cpu().pin_memory(), r[1].cpu().pin_memory(), r[2].cpu().pin_memory()) for r in records]
    out_u = torch.empty(u.shape, dtype=torch.float64).pin_memory()
    out_q = torch.empty(q.shape, dtype=torch.float64).pin_memory()
    out_uh = torch.empty(uh.shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    rank_barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(args.steps):
        replay(k, host)
        out_u.copy_(u, non_blocking=True)
        out_q.copy_(q, non_blocking=True)
        out_uh.copy_(uh, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev)
    bytes_io = 8 * (u.numel() + q.numel() + uh.numel())

    # ---- comparison forms on the same workload (same initial state, same tolerance)
    compare = {}
    if args.compare:
        if learn:
            first, last = ctx.mlp_train(epochs=args.mlp_epochs, batch=8192, lr=1e-3)
            ctxl = pkg.Context(pr, dict(opts, precond=2), device=dev)
            ctxl.mlp_setup(hidden=256, seed=0, max_pairs=1)
            ctxl.mlp_params(ctx.mlp_params())
            sl = newton_solve(ctxl, state0)
            du_ = sl["state"][0] - sol["state"][0]
            compare["mixed_learned"] = {k: v for k, v in sl.items() if k not in ("records", "state")}
            compare["mixed_learned"].update(train_samples=n_samples, train_loss_first=first, train_loss_last=last,
                                            rel_diff_u_vs_primary=float(du_.norm() / sol["state"][0].norm()))
            ctxl.close()
        ctxp = pkg.Context(pr, dict(base, precision=pkg.PREC_FP64, precond=1, apply_mode=0), device=dev)
        sp = newton_solve(ctxp, state0)
        dup = sp["state"][0] - sol["state"][0]
        compare["plain_fp64_algorithm2"] = {k: v for k, v in sp.items() if k not in ("records", "state")}
        compare["plain_fp64_algorithm2"]["rel_diff_u_vs_primary"] = float(dup.norm() / sol["state"][0].norm())
        ctxp.close()
        compare["primary_full_solve"] = {k: v for k, v in sol.items() if k not in ("records", "state")}

    # ---- roofline of the dominant kernel: the kernel with the largest device time per step
    # (phase events around single kernels; the BF16 apply is timed inside the inner-GMRES graph)
    work = phase_work(z, z["E"], args.precision, args.apply_mode)
    ph_mean = {k: float(np.mean(v)) for k, v in phase_acc.items() if v and v[0] >= 0}
    peaks = measured_peaks()
    its_step = its_timed / args.steps
    inner = args.inner if args.precond == 1 else 0
    bf = bool(opts.get("precond_bf16")) and args.apply_mode == 1 and args.precond == 1
    per_step = {}
    if "apply" in ph_mean:
        per_step["apply"] = ph_mean["apply"] * (its_step * (1 if bf else 1 + inner) + 1)
    if bf and "apply_bf16" in ph_mean:
        per_step["apply_bf16"] = ph_mean["apply_bf16"] * its_step * inner
    for k in ("cond_gemm", "lu", "vol_contract", "trsm"):
        if k in ph_mean:
            per_step[k] = ph_mean[k]
    roof = None
    if per_step:
        dom = max(per_step, key=per_step.get)
        E, Nu, Nt = z["E"], z["Nu"], z["Nt"]
        if dom in ("apply", "apply_bf16"):
            byts = work["apply_bytes"] if dom == "apply" else (2 * Nt * Nt + 20 * Nt) * E
            ach = byts / (ph_mean[dom] / 1e3) / 1e9
            pk = peaks.get("hbm_gbs", 6800.0)
            tr = TRAFFIC_PER_MACRO.get((dom, args.precision, args.apply_mode))
            name = {"apply": "k_apply_explicit" if args.apply_mode == 1 else "k_apply (Algorithm 2)",
                    "apply_bf16": "k_apply_explicit_bf16 (inner GMRES)"}[dom]
            roof = dict(kernel=name + ", one launch = all %d macro-elements" % E, bound="hbm", achieved=ach, peak=pk,
                        unit="GB/s", frac=ach / pk, traffic=(tr * E / 1e9 if tr else None), traffic_unit="GB/launch",
                        algorithmic=byts / 1e9, peak_source="MEASURED_PEAKS.json hbm_gbs (measured copy)"
                        if "hbm_gbs" in peaks else "fallback 6800 GB/s")
        else:
            # volume contraction: per (macro, input X, test species t, sub-element) a product
            # [NLOC x (d+1) NG] x [(d+1) NG x ns NLOC], NLOC = (p+1)^d, NG = (p+2)^d, m^d sub-elements
            d, p_, m_ = z["d"], 2, 2
            nloc, ngp = (p_ + 1) ** d, (p_ + 2) ** d
            vc = 2.0 * nloc * (z["ns"] * nloc) * ngp * (d + 1) * E * (d + 1) * z["ns"] * m_ ** d
            fl = {"cond_gemm": work["condense_flops"], "lu": work["lu_flops"],
                  "trsm": 2.0 * Nu * Nu * Nt * E, "vol_contract": vc}[dom]
            if args.precision == "fp64":
                pk, src = fp64_peak_tflops(torch), "measured cuBLAS DGEMM 4096^3 in this run (FP64 pipe)"
            else:
                pk = 2 * 128 * 152 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
                src = "FP32 FMA pipe: 128 lanes x 2 flop x 152 SMs x max SM clock (derived)"
            name = {"cond_gemm": "k_cond_gemm (2 launches)", "lu": "k_lu_panel_smem", "trsm": "k_lu_solve_multi",
                    "vol_contract": "k_vol_contract"}[dom]
            ach = fl / (ph_mean[dom] / 1e3) / 1e12
            roof = dict(kernel=name, bound="alu", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                        traffic=None, peak_source=src)
        roof["ms_per_launch"] = ph_mean[dom]
        roof["ms_per_step_all_launches"] = per_step[dom]
    lu_tflops = None
    if "lu" in ph_mean and ph_mean["lu"] > 0:
        lu_tflops = work["lu_flops"] / (ph_mean["lu"] / 1e3) / 1e12
    apply_gbs = work["apply_bytes"] / (ph_mean["apply"] / 1e3) / 1e9 if ph_mean.get("apply") else None

    per_step = t_dev / args.steps
    line = {
        "metric": METRIC,
        "value": replica_value(per_step, ws),
        "unit": UNIT,
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": max(args.warmup, N),
        "ms_per_step": per_step * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "dtype_detail": "f64 throughout" if args.precision == "fp64" else MIXED_DETAIL,
        "data": "synthetic (manufactured solution, seeded 1e-3 perturbation, seed 0)",
        "config": {"workload": "3D steady MMS cube, %d^3 macro-elements x 2^3 hexes, p=2 (%d macros, Nu=%d, Nt=%d, "
                               "%d trace DOFs)" % (NMAC, z["E"], z["Nu"], z["Nt"], z["F"] * z["ns"] * z["Nfn"]),
                   "precision": args.precision, "precond": args.precond, "lin_rtol": args.lin_rtol,
                   "restart": args.restart, "inner_iters": args.inner, "apply_mode": args.apply_mode,
                   "tc_mode": args.tc_mode, "refine_iters": args.refine, "precond_bf16": args.precond_bf16,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "fgmres_iters_per_step": its_timed / args.steps,
        "solve": {"newton_steps": N, "fgmres_iters": its_total, "converged_1e-8": sol["converged"],
                  "time_s": sol["time_s"], "res0": sol["res0"], "res": sol["res"]},
        "batched_lu_tflops": lu_tflops,
        "trace_apply_gbs": apply_gbs,
        "phases_ms": ph_mean,
        "compare": compare,
        "e2e": {"value": replica_value(t_e2e / args.steps, ws), "unit": UNIT, "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
    }
    ctx.close()
    return line


class StepDriver:
    """Newton steps of the DIRK3 integration through the library's step calls: each step()
    is one mehdg_newton_step, with mehdg_stage_begin / mehdg_stage_end opening and closing
    the stages (stage 1, 2, 3, then the next time step)."""

    def __init__(self, ctx, dt, max_newton=60):
        self.ctx, self.dt, self.max_newton = ctx, dt, max_newton
        self.stage, self.open, self.in_stage = 1, False, 0
        self.newton = self.fgmres = self.dirk_steps = self.status = 0

    def step(self, u, q, uh):
        while True:
            if not self.open:
                st = self.ctx.stage_begin(self.stage, self.dt, u, q, uh)
                self.open, self.in_stage = True, 0
                if st["converged"]:
                    self._close(u)
                    continue
            st = self.ctx.newton_step(u, q, uh)
            self.newton += 1
            self.in_stage += 1
            self.fgmres += st["fgmres_iters"]
            self.status |= st["status"]
            if st["converged"]:
                self._close(u)
            elif self.in_stage >= self.max_newton:
                raise RuntimeError("Newton cap reached in DIRK stage %d" % self.stage)
            return st

    def _close(self, u):
        self.ctx.stage_end(u)
        self.open = False
        if self.stage == 3:
            self.dirk_steps += 1
        self.stage = self.stage % 3 + 1

    def finish_dirk_step(self, u, q, uh):
        while self.open or self.stage != 1:
            self.step(u, q, uh)


def dirk_steps_timed(ctx, n, dt, u, q, uh, st):
    """n DIRK steps by mehdg_dirk_stage (three calls per step), timed with CUDA events."""
    import torch
    tot = dict(newton_steps=0, fgmres_iters=0, status=0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        for stage in (1, 2, 3):
            r = ctx.dirk_stage(stage, dt, u, q, uh)
            tot["newton_steps"] += r["newton_steps"]
            tot["fgmres_iters"] += r["fgmres_iters"]
            tot["status"] |= r["status"]
    e1.record(st)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    tot.update(time_s=t, s_per_dirk_step=t / max(n, 1), s_per_newton_step=t / max(tot["newton_steps"], 1),
               fgmres_iters_per_newton_step=tot["fgmres_iters"] / max(tot["newton_steps"], 1),
               fallback=bool(tot["status"] & 1), dirk_steps=n)
    return tot


def gemm_peaks(torch):
    """Measured dense rates of this GPU for the roofline denominators the driver's file does
    not hold: cuBLAS DGEMM 4096^3 (FP64 pipe), SGEMM 8192^3 without and with TF32, best of 5
    (CUDA events).  Returns TFLOP/s."""
    out = {}
    saved = torch.backends.cuda.matmul.allow_tf32
    for name, dt, n, tf32 in (("fp64", torch.float64, 4096, False), ("fp32", torch.float32, 8192, False),
                              ("tf32", torch.float32, 8192, True)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        c = torch.matmul(a, b)
        best = 1e9
        for _ in range(5):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            torch.matmul(a, b, out=c)
            e.record()
            e.synchronize()
            best = min(best, s.elapsed_time(e) / 1e3)
        out[name] = 2.0 * n ** 3 / best / 1e12
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = saved
    torch.cuda.empty_cache()
    return out


def sf_contract_macs(d, p):
    """Multiply-adds of the sum-factorised volume contraction per (input, test species, trial
    species, sub-element): an x pass over the (alpha, beta) pairs grouped by the classes of
    their remaining factors, then a pass per further axis over the merged classes."""
    p1, g1 = p + 1, p + 2

    def cls(a, done):
        return 0 if (a == 0 or a <= done) else a - done
    pairs = [(a, b) for a in range(d + 1) for b in range(d + 1) if not (a == 0 and b != 0)]
    macs = len(pairs) * g1 ** (d - 1) * p1 * p1 * g1                       # x pass
    if d == 3:
        n1c = {}
        for a in range(d + 1):
            n1c.setdefault(cls(a, 2), set()).add(cls(a, 1))
        macs += sum(len(n1c[za]) * len(n1c[zb]) for za in n1c for zb in n1c) * g1 * p1 ** 4 * g1   # y pass
    macs += 4 * g1 * p1 ** (2 * d)                                           # last pass
    return macs


def kernel_work(z, precision, apply_mode, mapped=False):
    """Algorithmic work of one execution of each phase over all E macro-elements:
    (kind, amount, kernel name).  kind "flop" or "byte".  mapped: curved macro-elements, whose
    per-macro liftings are dense (the condensation is the dense product k_cond_gemm)."""
    E, Nu, Nt, Np, Nth, d, ns = z["E"], z["Nu"], z["Nt"], z["Np"], z["Nth"], z["d"], z["ns"]
    n1 = round(Np ** (1.0 / d))
    p_, m_ = (n1 - 1) // 2, 2
    w = 8 if precision == "fp64" else 4
    nloc, ngp = (p_ + 1) ** d, (p_ + 2) ** d
    if precision == "fp64":
        vc = 2.0 * sf_contract_macs(d, p_) * (d + 1) * ns * ns * m_ ** d * E
    else:
        # volume contraction: per (macro, input X, test species, sub-element) the product
        # [nloc x (d+1) ng] [(d+1) ng x ns nloc] plus forming its right factor [(d+1) ng x ns nloc]
        # from the pointwise Jacobian ((d+1) terms per entry)
        vc = (2.0 * nloc * ns * nloc * ngp * (d + 1) + 2.0 * ngp * (d + 1) * ns * nloc * (d + 1)) \
            * (d + 1) * ns * m_ ** d * E
    # Kronecker condensation: n1 terms per direction for each S/B entry, n1 for each C/D entry,
    # plus the rhs product over the row of A_.q
    kron = 2.0 * (Nu + Nt) * (Nu * d * n1 + Nt * n1 + d * Nu) * E
    # dense condensation: [S | C] and [B | D] updated by A_.q [W_k | -Wh_k], per species
    dense = 2.0 * (Nu + Nt) * d * Np * (Np + Nth) * ns * E
    if apply_mode == 1:
        apply = ("byte", (w * Nt * Nt + (8 + 8 + 4) * Nt) * E, "k_apply_explicit")
    else:
        apply = ("byte" if precision != "fp64" else "flop",
                 (w * (2 * Nu * Nt + Nt * Nt + Nu * Nu) + 20 * Nt + 4 * Nu) * E if precision != "fp64"
                 else 2.0 * (2 * Nu * Nt + Nt * Nt + Nu * Nu) * E, "k_apply (Algorithm 2)")
    return {"vol_contract": ("flop", vc, "k_vol_contract"),
            "cond_gemm": ("flop", dense, "k_cond_gemm") if mapped else ("flop", kron, "k_cond_kron"),
            "lu": ("flop", (2.0 / 3.0) * Nu ** 3 * E, "k_lu_panel_smem / k_lu_batched"),
            "trsm": ("flop", 2.0 * Nu * Nu * Nt * E, "k_lu_solve_multi"),
            "apply": apply,
            "apply_bf16": ("byte", (2 * Nt * Nt + 20 * Nt) * E, "k_apply_explicit_bf16 (inner GMRES)")}


def roofline_of(stats, steps, z, precision, apply_mode, peaks, gp, mapped=False):
    """Roofline of the kernel with the largest summed device time over the timed steps."""
    work = kernel_work(z, precision, apply_mode, mapped)
    per_step = {k: v[0] / steps for k, v in stats.items() if v[1] > 0}
    cand = {k: v for k, v in per_step.items() if k in work}
    if not cand:
        return None, per_step
    dom = max(cand, key=cand.get)
    ms_sum, cnt = stats[dom]
    kind, amount, name = work[dom]
    ms_launch = ms_sum / cnt
    if kind == "byte":
        ach = amount / (ms_launch / 1e3) / 1e9
        pk = peaks.get("hbm_gbs")
        roof = dict(bound="hbm", achieved=ach, peak=pk, unit="GB/s", frac=ach / pk if pk else None,
                    peak_source="MEASURED_PEAKS.json hbm_gbs (measured copy)")
    else:
        ach = amount / (ms_launch / 1e3) / 1e12
        if precision == "fp64":
            pk, src = gp["fp64"], "measured cuBLAS DGEMM 4096^3 in this run (FP64 pipe)"
        else:
            pk, src = gp["fp32"], "measured cuBLAS SGEMM 8192^3 without TF32 in this run (FP32 pipe)"
        roof = dict(bound="alu", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk, peak_source=src)
    roof.update(kernel=name + " (one launch = all %d macro-elements)" % z["E"], phase=dom,
                algorithmic=amount / (1e9 if kind == "byte" else 1e12),
                algorithmic_unit="GB/launch" if kind == "byte" else "TFLOP/launch",
                ms_per_launch=ms_launch, launches_per_step=cnt / steps, ms_per_step_all_launches=ms_sum / steps,
                traffic=None, traffic_note="ncu DRAM bytes of this kernel are in profiles/ (captured on a "
                                           "reduced mesh); not re-measured in this run")
    return roof, per_step


def run_tgv(args, ws, rank, lrank):
    """The headline: Newton steps of the DIRK3 integration of the 16^3 Taylor-Green vortex.

    Primary (value): the plain FP64 form.  Warm-up: W Newton steps from the lifted initial
    condition; timed: the next K Newton steps (device-resident state).  e2e: further steps
    with the state copied in from and out to pinned host memory inside the timed region.
    Compare (same integration, same 1e-8 Newton tolerance): the FP64 run is finished to a
    whole number of DIRK steps; the mixed form runs those DIRK steps from the same initial
    state by mehdg_dirk_stage (end-state difference from FP64 reported), recording
    (residual, error) pairs; the learned correction is trained on them and compared with
    the multi-level preconditioner over the next DIRK steps from the same state."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg

    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    # a stream of its own for everything that follows (torch work and library calls alike): the
    # legacy default stream cannot capture the inner-GMRES CUDA graph
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    nmac = args.nmac_tgv
    pr = W.tgv(nmac=nmac)
    z = sizes(pr)
    dt = 0.05 / 0.1          # 0.05 t_c, t_c = L / V0 = 10 acoustic units (L = 1, V0 = M0 = 0.1)
    base = dict(restart=args.restart, max_iters=3000, lin_rtol=args.lin_rtol, newton_rtol=1e-8, newton_atol=1e-14,
                max_newton=60, inner_iters=args.inner, refine_iters=args.refine, tc_mode=args.tc_mode)
    opt64 = dict(base, precision=pkg.PREC_FP64, precond=1, apply_mode=args.fp64_apply_mode)
    optmx = dict(base, precision=pkg.PREC_MIXED, precond=1, apply_mode=1, precond_bf16=args.precond_bf16)
    primary = opt64 if args.precision == "fp64" else optmx
    st = torch.cuda.current_stream(dev)
    peaks = measured_peaks()
    gp = gemm_peaks(torch) if rank == 0 else {}

    ctx = pkg.Context(pr, primary, device=dev)
    u, q, uh = ctx.init_state(None, None, lift=True)
    drv = StepDriver(ctx, dt)
    for _ in range(args.warmup):
        drv.step(u, q, uh)
    torch.cuda.synchronize()
    rank_barrier(ws)
    K = max(1, args.steps)
    ctx.phase_stats(reset=True)
    n0, f0 = drv.newton, drv.fgmres
    clk = ClockSampler(lrank)
    clk.start()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(K):
        drv.step(u, q, uh)
    ev1.record(st)
    torch.cuda.synchronize()
    t_dev = ev0.elapsed_time(ev1) / 1e3
    clocks = clk.stop()
    launches = ctx.launch_count() - l0
    graph_replays = ctx.graph_replays()
    stats = ctx.phase_stats()
    its_timed = drv.fgmres - f0
    t_dev = max_over_ranks(t_dev, ws, dev)
    rank_barrier(ws)

    # ---- e2e: the state in from pinned host memory and out again around every step
    n_e2e = max(1, min(K, args.e2e_steps))
    hu, hq, huh = (x.cpu().pin_memory() for x in (u, q, uh))
    torch.cuda.synchronize()
    rank_barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n_e2e):
        u.copy_(hu, non_blocking=True)
        q.copy_(hq, non_blocking=True)
        uh.copy_(huh, non_blocking=True)
        drv.step(u, q, uh)
        hu.copy_(u, non_blocking=True)
        hq.copy_(q, non_blocking=True)
        huh.copy_(uh, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev)
    bytes_io = 8 * (u.numel() + q.numel() + uh.numel())

    # ---- the primary run to a whole number of DIRK steps (end state for the comparisons)
    drv.finish_dirk_step(u, q, uh)
    n_dirk = drv.dirk_steps
    primary_end = u.clone()
    primary_summary = dict(dirk_steps=n_dirk, newton_steps=drv.newton, fgmres_iters=drv.fgmres,
                           newton_steps_per_dirk_step=drv.newton / max(n_dirk, 1))
    ctx.close()
    del ctx

    compare = {}
    if args.compare:
        other = optmx if args.precision == "fp64" else opt64
        oname = "mixed" if args.precision == "fp64" else "plain_fp64"
        c2 = pkg.Context(pr, other, device=dev)
        uu, qq, hh = c2.init_state(None, None, lift=True)
        learn = oname == "mixed" and args.learn_compare_steps > 0
        if learn:
            c2.mlp_setup(hidden=256, seed=0, max_pairs=args.mlp_pairs, neighbors=args.mlp_neighbors)
            c2.mlp_set_recording(True)
        r = dirk_steps_timed(c2, n_dirk, dt, uu, qq, hh, st)
        r["rel_l2_u_vs_primary_end_state"] = float((uu - primary_end).norm() / primary_end.norm())
        compare[oname] = r
        if learn:
            n_samples = c2.mlp_set_recording(False)
            first, last = c2.mlp_train(epochs=args.mlp_epochs, batch=8192, lr=1e-3)
            state = (uu.clone(), qq.clone(), hh.clone())
            res = {}
            for kind, name in ((1, "multilevel"), (2, "learned"), (0, "block_jacobi")):
                c2.set_precond(kind)
                a, b_, c_ = (x.clone() for x in state)
                res[name] = dirk_steps_timed(c2, args.learn_compare_steps, dt, a, b_, c_, st)
                res[name]["state"] = a
            ref_state = res["multilevel"]["state"]
            for name in ("learned", "block_jacobi"):
                res[name]["rel_l2_u_vs_multilevel"] = float((res[name].pop("state") - ref_state).norm()
                                                            / ref_state.norm())
            res["multilevel"].pop("state")
            res["train"] = dict(pairs_from_dirk_steps=n_dirk, face_samples=n_samples, epochs=args.mlp_epochs,
                                loss_first_epoch=first, loss_last_epoch=last)
            compare["learned_vs_multilevel_mixed"] = res
        c2.close()

    roof, per_step = roofline_of(stats, K, z, args.precision, primary["apply_mode"], peaks, gp)
    lu_tf = None
    if stats.get("lu", (0, 0))[1]:
        lu_tf = kernel_work(z, args.precision, 0)["lu"][1] / (stats["lu"][0] / stats["lu"][1] / 1e3) / 1e12
    per = t_dev / K
    line = {
        "metric": METRIC,
        "value": replica_value(per, ws),
        "unit": UNIT_TGV,
        "n_gpus": ws,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": per * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32",
        "dtype_detail": "f64 throughout" if args.precision == "fp64" else MIXED_DETAIL,
        "data": "synthetic (Taylor-Green initial condition of the paper's Sec. 5.3, closed form; no perturbation)",
        "config": {"workload": WORKLOAD_TGV % (nmac, nmac, z["E"], z["F"] * z["ns"] * z["Nfn"]),
                   "precision": args.precision, "newton_rtol": 1e-8, "precond": 1, "lin_rtol": args.lin_rtol,
                   "restart": args.restart, "inner_iters": args.inner, "apply_mode": primary["apply_mode"],
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "fgmres_iters_per_step": its_timed / K,
        "batched_lu_tflops": lu_tf,
        "batched_lu_note": "sum of (2/3) Nu^3 over the macro-elements / device time of the LU launch",
        "primary_run": primary_summary,
        "phase_ms_per_step": {k: v for k, v in per_step.items()},
        "phase_launches_per_step": {k: stats[k][1] / K for k in stats if stats[k][1]},
        "gemm_peaks_tflops": gp,
        "compare": compare,
        "e2e": {"value": replica_value(t_e2e / n_e2e, ws), "unit": UNIT_TGV, "steps": n_e2e,
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
        "gpu_launches": launches,
        "inner_gmres_graph_replays": graph_replays,
        "roofline": roof,
        "clocks": clocks,
    }
    return line


def run_sphere(args, ws, rank, lrank):
    """Flow past a sphere on curved macro-elements (the cubed-sphere shell): Newton steps of the
    DIRK3 integration from the blended free stream.  Plain FP64 form (default, --precision fp64):
    dense Algorithm-2 apply (the per-macro liftings fill B, C and D), 6 x 8^2 x 12 macros by
    default, because the configuration's 6 x 8^2 x 16 = 6144 macros need about 285 GB of FP64
    blocks and workspace, more than the device holds.  Mixed form (--precision mixed): FP32
    blocks, stored A^T_i."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg

    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    # a stream of its own for everything that follows (torch work and library calls alike): the
    # legacy default stream cannot capture the inner-GMRES CUDA graph
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    fp64 = args.precision == "fp64"
    nr = args.sphere_nr or 12
    pr = W.sphere(nq=args.sphere_nq, nr=nr)
    z = sizes(pr)
    dt = 0.1
    opt = dict(precision=pkg.PREC_FP64, precond=1, apply_mode=args.sphere_apply_mode, restart=args.restart,
               max_iters=3000, lin_rtol=args.lin_rtol, newton_rtol=1e-8, newton_atol=1e-14, max_newton=60,
               inner_iters=args.inner)
    if not fp64:
        opt.update(precision=pkg.PREC_MIXED, apply_mode=1, tc_mode=args.tc_mode, refine_iters=args.refine,
                   precond_bf16=args.precond_bf16)
    st = torch.cuda.current_stream(dev)
    peaks = measured_peaks()
    gp = gemm_peaks(torch) if rank == 0 else {}
    ctx = pkg.Context(pr, opt, device=dev)
    u, q, uh = ctx.init_state(None, None, lift=True)
    drv = StepDriver(ctx, dt)
    for _ in range(args.warmup):
        drv.step(u, q, uh)
    torch.cuda.synchronize()
    rank_barrier(ws)
    K = max(1, args.steps)
    ctx.phase_stats(reset=True)
    f0 = drv.fgmres
    clk = ClockSampler(lrank)
    clk.start()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(K):
        drv.step(u, q, uh)
    ev1.record(st)
    torch.cuda.synchronize()
    t_dev = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    clocks = clk.stop()
    launches = ctx.launch_count() - l0
    stats = ctx.phase_stats()
    its = drv.fgmres - f0
    rank_barrier(ws)
    n_e2e = max(1, min(K, args.e2e_steps))
    hu, hq, huh = (x.cpu().pin_memory() for x in (u, q, uh))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n_e2e):
        u.copy_(hu, non_blocking=True)
        q.copy_(hq, non_blocking=True)
        uh.copy_(huh, non_blocking=True)
        drv.step(u, q, uh)
        hu.copy_(u, non_blocking=True)
        hq.copy_(q, non_blocking=True)
        huh.copy_(uh, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev)
    bytes_io = 8 * (u.numel() + q.numel() + uh.numel())
    bytes_dev = ctx.info["bytes_device"]
    ctx.close()
    roof, per_step = roofline_of(stats, K, z, args.precision, opt["apply_mode"], peaks, gp, mapped=True)
    lu_tf = None
    if stats.get("lu", (0, 0))[1]:
        lu_tf = kernel_work(z, args.precision, 0)["lu"][1] / (stats["lu"][0] / stats["lu"][1] / 1e3) / 1e12
    per = t_dev / K
    return {
        "metric": METRIC, "value": replica_value(per, ws), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if fp64 else "f32",
        "dtype_detail": "f64 throughout" if fp64 else MIXED_DETAIL,
        "data": "synthetic (free stream blended to rest near the sphere; closed form)",
        "config": {"workload": WORKLOAD_SPHERE % (args.sphere_nq, nr, z["E"], z["F"] * z["ns"] * z["Nfn"]),
                   "precision": args.precision, "newton_rtol": 1e-8, "precond": 1, "lin_rtol": args.lin_rtol,
                   "restart": args.restart, "inner_iters": args.inner, "apply_mode": opt["apply_mode"],
                   "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if ws > 1 else "1 GPU",
                   "bytes_device": bytes_dev},
        "fgmres_iters_per_step": its / K,
        "batched_lu_tflops": lu_tf,
        "primary_run": dict(dirk_steps=drv.dirk_steps, newton_steps=drv.newton, fgmres_iters=drv.fgmres),
        "phase_ms_per_step": per_step,
        "phase_launches_per_step": {k: stats[k][1] / K for k in stats if stats[k][1]},
        "gemm_peaks_tflops": gp,
        "e2e": {"value": replica_value(t_e2e / n_e2e, ws), "unit": UNIT, "steps": n_e2e,
                "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
    }


def run_mpsweep(args, ws, rank, lrank):
    """The paper's fixed-local-size study (Sec. 5.1, Tables 3-5) on its 3D Couette case with a
    source: the same number of local unknowns per macro-element with m p fixed and (m, p)
    varied, m p = 6 ((6, 1), (3, 2), (2, 3)) or the paper's m p = 8 ((8, 1), (4, 2); its (2, 4)
    needs p = 4, which these kernels do not provide), each steady-solved from the closed-form
    state plus a seeded 1e-3 perturbation to a 1e-8 residual, plain FP64.  Reported per (m, p): Newton steps, FGMRES
    iterations, seconds per Newton step and its local (assembly, condensation, LU, recovery)
    and global (Krylov) parts."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg

    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    st_ = torch.cuda.current_stream(dev)
    rows = []
    pairs = ((6, 1), (3, 2), (2, 3)) if args.sweep_mp == 6 else ((8, 1), (4, 2))
    for m, p in pairs:
        pr = W.couette3d(nmac=args.nmac_sweep, m=m, p=p)
        z = sizes(pr)
        opt = dict(precision=pkg.PREC_FP64, precond=1, apply_mode=2, restart=args.restart, max_iters=3000,
                   lin_rtol=args.lin_rtol, inner_iters=args.inner, newton_rtol=1e-8, max_newton=60)
        ctx = pkg.Context(pr, opt, device=dev)
        du, duh = W.perturbation(pr, 77)
        u, q, uh = ctx.init_state(torch.as_tensor(du, device=dev), torch.as_tensor(duh, device=dev), lift=True)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(st_)
        st = ctx.dirk_stage(0, 0.0, u, q, uh)
        ev1.record(st_)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        n = max(st["newton_steps"], 1)
        rows.append(dict(m=m, p=p, macros=z["E"], Nu=z["Nu"], trace_dofs=z["F"] * z["ns"] * z["Nfn"],
                         newton_steps=st["newton_steps"], fgmres_iters=st["fgmres_iters"],
                         fgmres_iters_per_newton_step=st["fgmres_iters"] / n, s_per_newton_step=t / n,
                         local_s_per_newton_step=(st["t_assemble"] + st["t_condense"] + st["t_recover"]) / n,
                         krylov_s_per_newton_step=st["t_krylov"] / n, res=st["res"], res0=st["res0"]))
        ctx.close()
    best = min(rows, key=lambda r: r["s_per_newton_step"])
    return {"metric": METRIC, "value": best["s_per_newton_step"], "unit": UNIT, "n_gpus": ws, "steps": 1,
            "warmup": 0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form Couette state with source + seeded 1e-3 perturbation)",
            "config": {"workload": "3D Couette flow with source, %d^3 macro-elements, m p = %d, (m, p) in {%s}, "
                                   "Nu = %d" % (args.nmac_sweep, args.sweep_mp,
                                                ", ".join("(%d,%d)" % mp for mp in pairs), rows[0]["Nu"]),
                       "precision": "fp64", "apply_mode": 2, "lin_rtol": args.lin_rtol, "precond": 1},
            "sweep": rows}


def run_dissipation(args, ws, rank, lrank):
    """The paper's accuracy study of Sec. 5.3 on this GPU: the Taylor-Green vortex at Re = 100
    (M0 = 0.1, (m, p) = (2, 2)) integrated by DIRK3 on two macro meshes, with the kinetic energy
    E_k and the dissipation rate eps of eq. C5321 (mehdg_flow_integrals) after every DIRK step,
    in the scaling rho_0 = L = V0 = 1 over t / t_c.  The ExaDG reference curves are not
    available: reported are the self-convergence between the meshes (largest difference of eps
    over the run, with the value at the coarse mesh's peak) and, per mesh, the gap between eps
    and -dE_k/dt (central differences), which is the compressible and numerical dissipation
    that eq. C5321 leaves out.  Mixed form (FP64 residuals, Newton to 1e-8)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg
    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    st_ = torch.cuda.current_stream(dev)
    V0 = 0.1
    dt_c = args.diss_dt
    n_steps = int(round(args.diss_tend / dt_c))
    opt = dict(precision=pkg.PREC_MIXED, precond=1, apply_mode=1, precond_bf16=args.precond_bf16,
               restart=args.restart, max_iters=3000, lin_rtol=args.lin_rtol, newton_rtol=1e-8, newton_atol=1e-14,
               max_newton=60, inner_iters=args.inner, refine_iters=args.refine, tc_mode=args.tc_mode)
    runs = {}
    t_total = 0.0
    newton_total = 0
    for nm in [int(x) for x in args.diss_nmac.split(",")]:
        pr = W.tgv(nmac=nm, m=2, p=2, Re=args.diss_re, M0=V0)
        ctx = pkg.Context(pr, opt, device=dev)
        u, q, uh = ctx.init_state(None, None, lift=True)
        ek, eps = ctx.tgv_diagnostics(u, q, V0)
        series = [[0.0, ek, eps]]
        newton = fg = status = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(st_)
        for n in range(n_steps):
            for stage in (1, 2, 3):
                r = ctx.dirk_stage(stage, dt_c / V0, u, q, uh)
                newton += r["newton_steps"]
                fg += r["fgmres_iters"]
                status |= r["status"]
            ek, eps = ctx.tgv_diagnostics(u, q, V0)
            series.append([(n + 1) * dt_c, ek, eps])
        ev1.record(st_)
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        t_total += t
        newton_total += newton
        ctx.close()
        ser = np.array(series)
        dek = np.full(len(ser), np.nan)
        dek[1:-1] = -(ser[2:, 1] - ser[:-2, 1]) / (2 * dt_c)
        ipk = int(np.argmax(ser[:, 2]))
        gap = np.nanmax(np.abs(dek - ser[:, 2]))
        runs[nm] = dict(macros=nm ** 3, n_eff=nm * 2 * 2, dirk_steps=n_steps, newton_steps=newton,
                        fgmres_iters=fg, fallback=bool(status & 1), time_s=t,
                        eps_peak=float(ser[ipk, 2]), t_peak=float(ser[ipk, 0]),
                        max_abs_eps_minus_dEk=float(gap),
                        series=[[round(a, 6), float(b), float(c), None if np.isnan(d) else float(d)]
                                for (a, b, c), d in zip(series, dek)])
    keys = sorted(runs)
    conv = None
    if len(keys) >= 2:
        a, b = np.array(runs[keys[0]]["series"], dtype=float), np.array(runs[keys[-1]]["series"], dtype=float)
        conv = dict(max_abs_eps_difference=float(np.max(np.abs(a[:, 2] - b[:, 2]))),
                    max_abs_Ek_difference=float(np.max(np.abs(a[:, 1] - b[:, 1]))),
                    eps_peak_fine=runs[keys[-1]]["eps_peak"])
    return {"metric": "TGV kinetic-energy dissipation rate eps(t) (eq. C5321)", "value": t_total / max(newton_total, 1),
            "unit": "s per Newton step", "n_gpus": ws, "steps": n_steps, "warmup": 0, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 residuals, f32 blocks",
            "data": "synthetic (closed-form TGV initial condition)",
            "config": {"workload": "Taylor-Green vortex Re %g, M0 0.1, (m, p) = (2, 2), macro meshes %s, dt %g t_c, "
                                   "t_end %g t_c" % (args.diss_re, args.diss_nmac, dt_c, args.diss_tend),
                       "precision": "mixed", "newton_rtol": 1e-8},
            "series_columns": ["t/t_c", "E_k/V0^2", "eps L/V0^3", "-dE_k/dt L/V0^3"],
            "runs": {str(k): v for k, v in runs.items()}, "self_convergence": conv}


def run_layers(args, ws, rank, lrank):
    """The paper's Table-4 comparison on this GPU: one-layer (eqs. C46-C47) against second-layer
    (eqs. AP12, ASC2) static condensation, FP64, on a 3D manufactured-solution cube of p = 1
    macro-elements (m = 2; the one-layer local matrix must fit the solver's shared memory).
    Both forms store A^T_i explicitly and apply it the same way, so the FGMRES iterations are
    equal and the local time (condensation, factorisation, b^) is what differs."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg
    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    pr = W.mms(dim=3, nmac=args.nmac_layers, m=2, p=1)
    z = sizes(pr)
    du, duh = W.perturbation(pr, 0)
    st = torch.cuda.current_stream(dev)
    state = None
    res = {}
    for layers in (2, 1):
        ctx = pkg.Context(pr, dict(precision=pkg.PREC_FP64, apply_mode=1, condense_layers=layers, precond=1,
                                   lin_rtol=1e-3, restart=60, max_iters=2000,
                                   inner_iters=10), device=dev)
        if state is None:   # the first Newton system of the steady solve from the lifted initial state
            state = ctx.init_state(torch.as_tensor(du, device=dev), torch.as_tensor(duh, device=dev), lift=True)
        K = max(1, args.steps)
        t_local = 0.0
        for k in range(K + 1):      # the condensation works in place: assemble before each one
            ctx.assemble(*state)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            b = ctx.condense(shift=0.5)
            e1.record(st)
            torch.cuda.synchronize()
            if k > 0:                # the first one is the warm-up
                t_local += e0.elapsed_time(e1) / 1e3 / K
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(st)
        x, stats = ctx.linear_solve(b, allow_not_converged=True)
        g1.record(st)
        torch.cuda.synchronize()
        res["one_layer" if layers == 1 else "second_layer"] = dict(
            local_s=t_local, local_ms_per_macro=t_local / z["E"] * 1e3, global_s=g0.elapsed_time(g1) / 1e3,
            fgmres_iters=stats["fgmres_iters"], fgmres_res=stats["res"], local_matrix_size=(z["d"] + 1) * z["Nu"] if layers == 1 else z["Nu"])
        ctx.close()
    return {"metric": METRIC, "value": res["second_layer"]["local_s"], "unit": "s per condensation (second layer)",
            "n_gpus": ws, "steps": max(1, args.steps), "warmup": 1, "higher_is_better": False, "dtype": "f64",
            "data": "synthetic (lifted manufactured solution + seeded 1e-3 perturbation)", "scaling": "weak",
            "vs_baseline": None,
            "config": {"workload": "3D MMS cube, %d^3 macro-elements x 2^3 hexes, p=1 (Nu=%d, Nt=%d): one-layer vs "
                                   "second-layer condensation" % (args.nmac_layers, z["Nu"], z["Nt"])},
            "layers": res, "speedup_second_over_one_layer": res["one_layer"]["local_s"] / res["second_layer"]["local_s"]}


def run_batched(args, ws, rank, lrank):
    """Batched uneven steady solves: independent manufactured-solution problems of the
    config-2 form with seeded sizes (m_c^3 macro-elements, m_c in 2..6) and degrees
    (p in 1..3), each solved to a 1e-8 residual by the steady Newton-SER iteration.  The
    problems go, largest first, into waves that fit a device-memory budget; each wave is one
    mehdg_batch: lockstep Newton rounds of all its problems, their assembly and condensation
    replayed as CUDA graphs, the local LU of every problem in one persistent work-queue launch
    with autotuned panel widths.  Reports the wall time of the whole set."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as pkg

    dev = torch.device("cuda:%d" % lrank)
    torch.cuda.set_device(dev)
    probs = W.batched_problems(count=args.batch_count, seed0=1000)
    if ws > 1:   # replicas: each rank takes every ws-th problem
        probs = probs[rank::ws]
    szs = [sizes(pr) for pr in probs]

    def mem_bytes(z, amode):
        Nu, Nt, E = z["Nu"], z["Nt"], z["E"]
        w = 8.0 if amode == 0 else 4.0                 # FP64 blocks for p = 3
        blocks = w * (4 * Nu * Nu + 2 * Nu * Nt + 3 * Nt * Nu + Nt * Nt + Nu * Nu)   # + S kept for refinement
        extra = (4.0 * Nu * Nt + 2.0 * Nt * Nt) if amode == 1 else 0.0
        p_ = round(z["Np"] ** (1.0 / 3.0)) // 2        # Np = (2p + 1)^3 for m = 2
        kvol = 4.0 * 4 * z["ns"] * 8 * (p_ + 2) ** 3 * 80                             # pointwise Jacobians
        ntr = z["F"] * z["ns"] * z["Nfn"]
        return 1.25 * E * (blocks + extra + kvol) + 8.0 * ntr * (2 * args.restart + 45) + 256e6

    def opts_for(pr):
        # p <= 2: the mixed path with the stored local operators; p = 3 (Nu = 1715): FP64 blocks
        # and the Algorithm-2 apply (the FP32 factors of these larger S made FGMRES stall)
        base = dict(precond=1, restart=args.restart, max_iters=3000, lin_rtol=args.lin_rtol, inner_iters=args.inner,
                    newton_rtol=1e-8, max_newton=60)
        if pr["p"] <= 2:
            return 1, dict(base, precision=pkg.PREC_MIXED, apply_mode=1, precond_bf16=1, refine_iters=args.refine,
                           tc_mode=args.tc_mode)
        return 0, dict(base, precision=pkg.PREC_FP64, apply_mode=0)

    order = sorted(range(len(probs)), key=lambda i: -szs[i]["E"] * szs[i]["Nu"] ** 2)
    budget = args.batch_mem_gb * 1e9
    waves, cur, used = [], [], 0.0
    for i in order:
        need = mem_bytes(szs[i], opts_for(probs[i])[0])
        if cur and used + need > budget:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(i)
        used += need
    if cur:
        waves.append(cur)

    results = [None] * len(probs)
    wave_info = []
    err = None
    torch.cuda.synchronize()
    rank_barrier(ws)
    clk = ClockSampler(lrank)
    clk.start()
    t0 = time.perf_counter()
    for wv in waves:
        tw = time.perf_counter()
        try:
            batch = pkg.Batch([probs[i] for i in wv], [opts_for(probs[i])[1] for i in wv], device=dev)
            states = []
            for k, i in enumerate(wv):
                du, duh = W.perturbation(probs[i], 1000 + i)
                states.append(batch.contexts[k].init_state(torch.as_tensor(du, device=dev),
                                                           torch.as_tensor(duh, device=dev), lift=True))
            stats, rounds = batch.steady_solve(states, allow_not_converged=True)
            tiles = batch.tiles()
            replays = batch.graph_replays()
            if True:
                for k, i in enumerate(wv):
                    results[i] = dict(E=szs[i]["E"], p=probs[i]["p"], newton=stats[k]["newton_steps"],
                                      fgmres=stats[k]["fgmres_iters"], res=stats[k]["res"], res0=stats[k]["res0"],
                                      retried=bool(stats[k]["status"] & 4), converged=stats[k]["converged"])
            batch.close()
            torch.cuda.synchronize()
            wave_info.append(dict(problems=len(wv), macros=sum(szs[i]["E"] for i in wv), rounds=rounds,
                                  graph_replays=replays, seconds=time.perf_counter() - tw,
                                  tiles=[dict(n=t[0], fp64=t[1], panel_width=t[2], sample_ms=t[3]) for t in tiles]))
        except Exception as exc:   # reported in the JSON line
            err = "wave of %d problems: %s" % (len(wv), exc)
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    wall = max_over_ranks(wall, ws, dev)
    done = [r for r in results if r]
    n_done = int(sum_over_ranks(len(done), ws, dev))
    n_probs = int(sum_over_ranks(len(probs), ws, dev))
    newton = int(sum_over_ranks(sum(r["newton"] for r in done), ws, dev))
    macro_steps = sum_over_ranks(sum(r["newton"] * r["E"] for r in done), ws, dev)
    converged = all(r["converged"] for r in done) and len(done) == len(probs)
    converged = sum_over_ranks(0.0 if converged else 1.0, ws, dev) == 0.0
    by_p = {}
    for r in done:
        b_ = by_p.setdefault(r["p"], dict(problems=0, macros=0, newton_steps=0, fgmres_iters=0, retried=0))
        b_["problems"] += 1
        b_["macros"] += r["E"]
        b_["newton_steps"] += r["newton"]
        b_["fgmres_iters"] += r["fgmres"]
        b_["retried"] += int(r["retried"])
    return {
        "metric": METRIC,
        "value": wall,
        "unit": "s per batch of %d problems" % n_probs,
        "n_gpus": ws,
        "steps": 1,
        "warmup": 0,
        "ms_per_step": wall * 1e3,
        "higher_is_better": False,
        "scaling": "strong",   # one fixed batch, split across the ranks
        "vs_baseline": None,
        "dtype": "f32",
        "dtype_detail": MIXED_DETAIL + " (p = 3 problems in f64)",
        "data": "synthetic (seeded manufactured-solution problems, seeds 1000 + k)",
        "config": {"workload": "batched uneven steady MMS solves: %d problems, m_c in 2..6, p in 1..3, "
                               "2^3 hexes per macro-element" % n_probs,
                   "mem_budget_gb": args.batch_mem_gb,
                   "schedule": "waves under the memory budget, largest first; one mehdg_batch per wave (lockstep "
                               "Newton rounds, graph-replayed assembly and condensation, one work-queue LU launch "
                               "per precision and round, autotuned panel widths)",
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "problems_solved": n_done,
        "all_converged_1e-8": converged,
        "problems_per_s": n_done / wall,
        "newton_steps_total": newton,
        "macro_newton_steps_per_s": macro_steps / wall,
        "by_degree": by_p,
        "by_degree_scope": "rank 0's share of the batch" if ws > 1 else "whole batch",
        "waves": wave_info,
        "not_converged": [dict(problem=i, p=r["p"], macros=r["E"], newton=r["newton"], res=r["res"], res0=r["res0"],
                               retried=r["retried"]) for i, r in enumerate(results) if r and not r["converged"]],
        "error": err,
        "clocks": clocks,
    }


# FGMRES iterations per Newton step of the default line (26.6-26.8 measured on GB300);
# the reference arm runs without a GPU and scales its sampled costs by this count
REF_FGMRES_ITERS = 27


def oracle_sample_time(pr, n_macro=2, fgmres_iters=None, applies_per_iter=1):
    """Oracle (numpy FP64) time of one Newton step on a bounded sample, scaled to the workload:
    assembly, second-layer condensation and LU of every macro, applies_per_iter
    Algorithm-2 applies of every macro per FGMRES iteration (the outer one plus the inner
    GMRES steps of the multi-level preconditioner) and the local recovery of every macro."""
    from oracle import solve as osolve
    from oracle import assemble as oasm
    P = osolve.Problem(pr)
    u, q, uh = W.random_state(pr, 0)
    t0 = time.perf_counter()
    for e in range(n_macro):
        geo = P.geometry(e)
        blk = oasm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), None, P.source(geo),
                                  P.bfaces(e, geo))
        c = osolve.condense_second_layer(geo, blk, 1.0)
    t_local = (time.perf_counter() - t0) / n_macro
    x = np.random.default_rng(1).normal(size=c["C"].shape[1])
    t1 = time.perf_counter()
    for _ in range(3):
        osolve.apply_local(c, x)
    t_apply = (time.perf_counter() - t1) / 3
    t2 = time.perf_counter()
    osolve.recover(geo, blk, c, x)
    t_recover = time.perf_counter() - t2
    its = fgmres_iters if fgmres_iters else REF_FGMRES_ITERS
    per_step = P.E * (t_local + t_recover) + its * applies_per_iter * P.E * t_apply
    return per_step, dict(sample="assembly + second-layer condensation + LU and one recovery of %d macro-element(s), "
                                 "3 Algorithm-2 applies of one macro-element; scaled by %d macros, %d FGMRES "
                                 "iterations per step and %d applies per iteration"
                                 % (n_macro, P.E, its, applies_per_iter), cores=os.cpu_count())


# FGMRES iterations per Newton step of the 16^3 TGV integration (multi-level preconditioner, 10
# inner iterations, rtol 1e-3), measured on GB300; the reference arm runs without a GPU and
# scales its sampled costs by this count
REF_FGMRES_ITERS_TGV = 4
_ORACLE_CACHE = {}


def oracle_tgv_newton_sample(pr, fgmres_iters, applies_per_iter, n_macro=1):
    """Oracle (numpy FP64) cost of one Newton step of the TGV DIRK integration on a bounded
    sample: assembly with a DIRK stage time term, second-layer condensation with LU, one
    recovery and three Algorithm-2 applies of n_macro macro-elements, scaled to every
    macro-element and to fgmres_iters x applies_per_iter applies (outer FGMRES apply plus
    the inner GMRES steps of the multi-level preconditioner).  Returns (seconds, info)."""
    from oracle import solve as osolve
    from oracle import assemble as oasm
    key = (pr["name"], tuple(pr["nmac"]))
    if _ORACLE_CACHE.get("key") != key:     # mesh tables and the sampled state, built once
        P = osolve.Problem(pr)
        _ORACLE_CACHE.update(key=key, P=P, state=W.random_state(pr, 0))
    P = _ORACLE_CACHE["P"]
    u, q, uh = _ORACLE_CACHE["state"]
    t_all = time.perf_counter()
    hist = -2.0 * u[:n_macro]
    t0 = time.perf_counter()
    for e in range(n_macro):
        geo = P.geometry(e)
        tt = dict(coef=2.0, hist=hist[e], supg_time=True)
        blk = oasm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), tt, P.source(geo),
                                  P.bfaces(e, geo))
        c = osolve.condense_second_layer(geo, blk, 0.0)
    t_local = (time.perf_counter() - t0) / n_macro
    x = np.random.default_rng(1).normal(size=c["C"].shape[1])
    t1 = time.perf_counter()
    for _ in range(3):
        osolve.apply_local(c, x)
    t_apply = (time.perf_counter() - t1) / 3
    t2 = time.perf_counter()
    osolve.recover(geo, blk, c, x)
    t_recover = time.perf_counter() - t2
    per_step = P.E * (t_local + t_recover) + fgmres_iters * applies_per_iter * P.E * t_apply
    info = dict(sample="assembly (DIRK time term) + second-layer condensation + LU and one recovery of %d "
                       "macro-element(s) and 3 Algorithm-2 applies of one macro-element, scaled by %d "
                       "macro-elements, %s FGMRES iterations per Newton step and %d applies per iteration"
                       % (n_macro, P.E, fgmres_iters, applies_per_iter),
                cores=os.cpu_count(), sample_wall_s=time.perf_counter() - t_all)
    return per_step, info


def cpu_baseline_tgv(line):
    """cpu_baseline of the headline line: the oracle on the host cores, bounded sample, scaled."""
    import torch
    its = line.get("fgmres_iters_per_step") or REF_FGMRES_ITERS_TGV
    t, info = oracle_tgv_newton_sample(W.tgv(nmac=16), round(its, 2), 1 + 10)
    return {"value": t, "unit": UNIT_TGV, "cores": info["cores"], "kind": "oracle", "sample": info["sample"],
            "extrapolated": True, "sample_wall_s": info["sample_wall_s"],
            "threads_numpy": torch.get_num_threads()}


def run_reference(args):
    """The reference arm: the oracle (this project's FP64 numpy restatement of the paper)
    timed on the host cores for the headline's metric and workload.  Each of the W + K
    steps is one bounded sample scaled to a whole Newton step (extrapolated: true)."""
    pr = W.tgv(nmac=args.nmac_tgv)
    z = sizes(pr)
    applies = 1 + (args.inner if args.precond == 1 else 0)
    times, walls = [], []
    info = None
    t_run = time.perf_counter()
    for k in range(args.warmup + args.steps):
        t, info = oracle_tgv_newton_sample(pr, REF_FGMRES_ITERS_TGV, applies)
        if k >= args.warmup:
            times.append(t)
            walls.append(info["sample_wall_s"])
    val = float(np.mean(times))
    import torch
    threads = torch.get_num_threads() if hasattr(torch, "get_num_threads") else os.cpu_count()
    nmac = args.nmac_tgv
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT_TGV, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TGV % (nmac, nmac, z["E"], z["F"] * z["ns"] * z["Nfn"])},
            "extrapolated": True,
            "timed": "%d bounded samples (%.1f s of host time in all), each scaled to one Newton step"
                     % (len(times), float(np.sum(walls))),
            "run_wall_s": time.perf_counter() - t_run,
            "cpu_baseline": {"value": val, "unit": UNIT_TGV, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"], "threads_numpy": threads, "extrapolated": True},
            "e2e": {"value": val, "unit": UNIT_TGV, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (default: 10 Newton steps for tgv)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv", choices=["tgv", "mms", "batched", "layers", "sphere", "mpsweep",
                                                  "dissipation"],
                    help="tgv: Newton steps of the 16^3 Taylor-Green DIRK integration (default, the headline); "
                         "mms: steady 3D manufactured solution (8^3); batched: independent uneven problems")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="form timed for the value (default: fp64 for tgv, mixed for mms)")
    ap.add_argument("--precond", type=int, default=1)
    ap.add_argument("--lin-rtol", type=float, default=1e-3)
    ap.add_argument("--restart", type=int, default=60)
    ap.add_argument("--inner", type=int, default=10, help="inner GMRES iterations of the multi-level preconditioner")
    ap.add_argument("--apply-mode", type=int, default=1, help="mms workload: 0 Algorithm 2 apply; 1 stored A^T_i")
    ap.add_argument("--fp64-apply-mode", type=int, default=2,
                    help="apply of the plain FP64 form: 2 Algorithm 2 with row-compressed B, C, D (default), "
                         "0 dense Algorithm 2, 1 stored A^T_i")
    ap.add_argument("--tc-mode", type=int, default=4,
                    help="mixed path: 4 forming A^T_i with the swizzled K-major tcgen05 product (default); 0 FP32 "
                         "SIMT; 1 tcgen05 split-TF32 LU updates; 2 also the condensation and A^T_i products (first "
                         "tcgen05 kernel); 3 plain TF32; 5 dense volume contraction")
    ap.add_argument("--refine", type=int, default=1,
                    help="FP64 refinement sweeps of each local S solve (b^ and recovery) on the mixed path")
    ap.add_argument("--precond-bf16", type=int, default=1,
                    help="mixed path: BF16 copy of A^T_i for the inner GMRES of the multi-level preconditioner")
    ap.add_argument("--no-phases", dest="phases", action="store_false")
    ap.add_argument("--nmac", type=int, default=8, help="mms workload: macro-elements per cube edge (8 = the config)")
    ap.add_argument("--no-cpu-baseline", dest="cpu", action="store_false")
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the comparison forms (mixed / learned / FP64)")
    ap.add_argument("--mlp-epochs", type=int, default=200)
    ap.add_argument("--mlp-pairs", type=int, default=64, help="recorded (residual, error) pairs per training run")
    ap.add_argument("--mlp-neighbors", type=int, default=0,
                    help="learned correction: 1 adds the neighbouring faces' block-Jacobi outputs to the input")
    ap.add_argument("--learn-compare-steps", type=int, default=1,
                    help="tgv: DIRK steps on which the learned correction is compared (0 = skip)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="tgv: Newton steps of the host-buffer (e2e) timing")
    ap.add_argument("--solve-steps", type=int, default=60, help="mms: cap on the recorded Newton steps")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-mem-gb", type=float, default=200.0)
    ap.add_argument("--nmac-tgv", type=int, default=16, help="TGV macro-elements per edge (16 = the config)")
    ap.add_argument("--nmac-layers", type=int, default=8, help="layers workload: macro-elements per cube edge")
    ap.add_argument("--nmac-sweep", type=int, default=3, help="mpsweep workload: macro-elements per cube edge")
    ap.add_argument("--sweep-mp", type=int, default=6, choices=[6, 8], help="mpsweep workload: the fixed m p")
    ap.add_argument("--sphere-nq", type=int, default=8, help="sphere workload: cells per cube-panel edge")
    ap.add_argument("--sphere-nr", type=int, default=0, help="sphere workload: radial layers (default 12)")
    ap.add_argument("--diss-nmac", default="4,8", help="dissipation workload: macro-elements per edge, per mesh")
    ap.add_argument("--diss-re", type=float, default=100.0, help="dissipation workload: Reynolds number V0 L / nu")
    ap.add_argument("--diss-dt", type=float, default=0.1, help="dissipation workload: DIRK step in t_c = L / V0")
    ap.add_argument("--diss-tend", type=float, default=10.0, help="dissipation workload: end time in t_c")
    ap.add_argument("--sphere-apply-mode", type=int, default=0,
                    help="sphere workload, FP64 form: 0 dense Algorithm 2 (default)")
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "fp64" if args.workload in ("tgv", "sphere") else "mixed"
    global NMAC
    NMAC = args.nmac
    ws, rank, lrank = dist_env()
    if args.impl == "reference":
        if rank == 0:
            args.steps = args.steps or 1
            print(json.dumps(run_reference(args)))
        return
    if ws > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.workload in ("tgv", "batched", "layers", "sphere", "mpsweep", "dissipation"):
        args.steps = args.steps or 10
        run = {"tgv": run_tgv, "batched": run_batched, "layers": run_layers, "sphere": run_sphere,
               "mpsweep": run_mpsweep, "dissipation": run_dissipation}[args.workload]
        line = run(args, ws, rank, lrank)
        if rank == 0:
            if args.workload == "tgv" and args.cpu and ws == 1:   # the oracle baseline, N = 1 only
                line["cpu_baseline"] = cpu_baseline_tgv(line)
            print(json.dumps(line))
        if ws > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    if args.steps == 0:
        args.steps = -1       # one replay of every recorded Newton step
    line = run_ours(args, ws, rank, lrank)
    if rank == 0:
        if args.cpu and ws == 1:   # the oracle baseline is taken at N = 1 only
            t, info = oracle_sample_time(workload(), n_macro=1,
                                         fgmres_iters=max(1, int(round(line["fgmres_iters_per_step"]))),
                                         applies_per_iter=1 + (args.inner if args.precond == 1 else 0))
            line["cpu_baseline"] = {"value": t, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                                    "sample": info["sample"]}
        print(json.dumps(line))
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
