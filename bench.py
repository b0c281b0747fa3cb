#!/usr/bin/env python3
"""Benchmark: fine cells/s of a full Recursive MRCM solve (build + solve).

Workload (default): the 1024 x 1024 quarter-five-spot problem -- unit square,
log-normal K with sigma^2 = 4 and correlation length 0.05 (seeded FFT
circulant embedding), no-flow boundary with zero-mean pressure, +1 / -1
sources in opposite corner cells, 64 x 64 leaves of 16 x 16 cells, 4-cell
interface segments, alpha = 1, 12 merge levels, FP64 throughout.

One step = mrcm_build_basis + mrcm_solve on inputs resident in HBM; L2 is
flushed (a 256 MiB write) between timed steps, outside the timed events.
`e2e` repeats the step through the same C-ABI calls from pinned host
buffers, host->device copies of K, q and the boundary values and the
device->host copies of p, Fx, Fy inside the timed region.

N > 1 (torchrun): every rank solves its own realisation (independent
replicas, no collective on the data path); value = all ranks' cells / max
time.  --impl reference times the FP64 CPU oracle on a bounded sample.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine cells/s full RecMRCM solve at rel-L2 ≤1e-8 vs FP64 oracle; % roofline"
# FP64 FMA pipe of GB300: 2 DFMA / clock / SM x 152 SMs x 2.07 GHz x 2 flops
FP64_PEAK_TFLOPS = 2 * 152 * 2.07e9 * 2 / 1e12
# rel-L2 bar of the FP64 form against the FP64 oracle (the metric's own
# tolerance, 1e-8, is the mixed form's)
FP64_FORM_TOL = 1e-10
WORKLOAD = ("square1024-qfs: 1024x1024 cells, log-normal K sigma^2=4 corr 0.05 (seed 2000), "
            "quarter-five-spot, no-flow, 64x64 leaves of 16x16, 4-cell segments, alpha=1, 12 levels")
CPU_SAMPLE_N = 256
# DRAM bytes (read + write) per launch of a kernel family at the 1024^2
# workload, from one ncu capture of this bench (dram__bytes_read.sum +
# dram__bytes_write.sum).  A family missing here reports traffic null.
TRAFFIC_PER_LAUNCH = {
    "gj_sweep": dict(bytes=1.216e6, source="ncu capture, mean over the 7 launches of one build"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refine", type=int, default=0,
                    help="iterative-refinement steps per solve in the timed steps (0: the paper's single "
                         "pass; its distance to the refined solution is checked in the same run)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def job_throughput(local_ms, cells_per_rank, steps, world, device="cpu"):
    """Whole-job cells/s of a weakly scaled run: every rank's summed step
    time is reduced to the maximum over ranks (the job ends with its slowest
    rank) and all ranks' cells are counted.  Returns (value, max_ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return cells_per_rank * world * steps / (max_ms / 1e3), max_ms


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm)
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import inputs
from oracle.mrcm import solve_mrcm
prob = inputs.darcy_problem({n}, {n}, sigma2=4.0, corr=0.05, seed=2000, bc="quarter_five_spot")
times = []
for _ in range({reps}):
    t = time.perf_counter()
    solve_mrcm(prob)
    times.append(time.perf_counter() - t)
print(json.dumps(dict(times=times, cells={n} * {n})))
"""


def time_oracle(n, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, n=n, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=1800)
    if out.returncode:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_sample_desc(n):
    return (f"oracle O2 (global MRCM, numpy/scipy FP64, single thread) on the {n}x{n} problem of "
            f"the same recipe (sigma^2=4, corr 0.05, seed 2000, quarter-five-spot, 16x16 leaves)")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = CPU_SAMPLE_N
    res = time_oracle(n, args.warmup + args.steps)
    times = res["times"][args.warmup:]
    value = res["cells"] * len(times) / sum(times)
    line = dict(metric=METRIC, value=value, unit="cells/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sum(times) / len(times),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, sample=f"{n}x{n}"),
                cpu_baseline=dict(value=value, unit="cells/s", cores=1, kind="oracle",
                                  sample=oracle_sample_desc(n)),
                e2e=dict(value=value, unit="cells/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, uuid):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100"]
            if uuid:
                cmd.insert(1, f"--id={uuid}")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in open(self.path):
            parts = [x.strip() for x in row.split(",")]
            if len(parts) < 8:
                continue
            try:
                sms.append(float(parts[0]))
                maxs.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return None
        sms.sort()
        return dict(sm_mhz=sms[len(sms) // 2], sm_max_mhz=max(maxs), reasons=sorted(reasons),
                    samples=len(sms))


def mass_balance(solver, q):
    """max |div F - q| / max |F| per cell, each cell using the one-sided
    fluxes of its own leaf on skeleton faces (MRCM fluxes are continuous only
    per segment, not per fine face)."""
    fa_x, fb_x, fa_y, fb_y = solver.iface_parts()
    div = fa_x[:, 1:] - fb_x[:, :-1] + fa_y[1:, :] - fb_y[:-1, :]
    scale = max(float(fa_x.abs().max()), float(fa_y.abs().max()))
    return float((div - q).abs().max()) / scale


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import inputs
    import paper_2009_07965_gb300 as mr
    from paper_2009_07965_gb300 import build as build_mod

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        build_mod.build()
    if world > 1:
        dist.barrier()
    n = args.size
    prob = inputs.darcy_problem(n, n, sigma2=4.0, corr=0.05, seed=2000 + rank,
                                bc="quarter_five_spot", alpha=1.0)
    stream = torch.cuda.Stream(dev)
    K = torch.from_numpy(prob.K).to(dev)
    q = torch.from_numpy(prob.q).to(dev)
    bcv = torch.from_numpy(prob.bc_val).to(dev)
    with torch.cuda.stream(stream):
        solver = mr.Solver(K, prob.Lx, prob.Ly, prob.sub, prob.seg, prob.alpha, prob.bc_type,
                           stream=stream)
    mr.mrcm_enable_timing(solver.ctx, True)
    mr.mrcm_set_refinement(solver.ctx, args.refine)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        solver.build_basis()
        solver.solve(q, bcv)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    sampler = ClockSampler(uuid)
    phases = {k: 0.0 for k in mr.PHASES}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k, v in mr.mrcm_phase_times(solver.ctx).items():
            phases[k] += v
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    # kernels one timed step launched (read before the accuracy check and
    # the refined step below change the solve's launch sequence)
    launches = (mr.mrcm_query(solver.ctx, "KERNEL_LAUNCHES_BUILD")
                + mr.mrcm_query(solver.ctx, "KERNEL_LAUNCHES_SOLVE"))
    cells = n * n
    value, total_ms = job_throughput(sum(step_ms), cells, args.steps, world, dev)

    # ---- end to end from pinned host buffers ------------------------------
    K_h = torch.from_numpy(prob.K).pin_memory()
    q_h = torch.from_numpy(prob.q).pin_memory()
    bc_h = torch.from_numpy(prob.bc_val).pin_memory()
    p_h = torch.empty(prob.ny, prob.nx, dtype=torch.float64).pin_memory()
    fx_h = torch.empty(prob.ny, prob.nx + 1, dtype=torch.float64).pin_memory()
    fy_h = torch.empty(prob.ny + 1, prob.nx, dtype=torch.float64).pin_memory()
    K_d, q_d, bc_d = torch.empty_like(K), torch.empty_like(q), torch.empty_like(bcv)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        ev0.record(stream)
        with torch.cuda.stream(stream):
            K_d.copy_(K_h, non_blocking=True)
            q_d.copy_(q_h, non_blocking=True)
            bc_d.copy_(bc_h, non_blocking=True)
        solver.set_permeability(K_d)
        solver.build_basis()
        pd, fxd, fyd = solver.solve(q_d, bc_d)
        with torch.cuda.stream(stream):
            p_h.copy_(pd, non_blocking=True)
            fx_h.copy_(fxd, non_blocking=True)
            fy_h.copy_(fyd, non_blocking=True)
        ev1.record(stream)
        ev1.synchronize()
        if it >= args.warmup:
            e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_value, _ = job_throughput(sum(e2e_ms), cells, args.steps, world, dev)
    h2d = (K_h.numel() + q_h.numel() + bc_h.numel()) * 8
    d2h = (p_h.numel() + fx_h.numel() + fy_h.numel()) * 8
    solver.solve(q, bcv, want_iface=True)
    torch.cuda.synchronize(dev)
    balance = mass_balance(solver, q)

    # ---- accuracy of the timed configuration (outside the timed regions):
    # rel-L2 distance to the solve refined to the rounding level, which the
    # parity tests pin to the FP64 oracle
    timed = [x.cpu().numpy().copy() for x in (solver.p, solver.Fx, solver.Fy)]
    mr.mrcm_set_refinement(solver.ctx, 3)
    solver.solve(q, bcv)
    refined = [x.cpu().numpy().copy() for x in (solver.p, solver.Fx, solver.Fy)]
    rel = {name: float(np.linalg.norm(a - b) / np.linalg.norm(b))
           for name, a, b in zip(("p", "Fx", "Fy"), timed, refined)}
    # ---- the same step with one refinement step, for reference ------------
    mr.mrcm_set_refinement(solver.ctx, 1)
    for _ in range(2):
        step()
    ref_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        ref_ms.append(ev0.elapsed_time(ev1))
    mr.mrcm_set_refinement(solver.ctx, args.refine)

    build_flops = mr.mrcm_query(solver.ctx, "BUILD_FLOPS")
    ph = {k: v / args.steps for k, v in phases.items()}          # ms per step
    pf = mr.mrcm_phase_flops(solver.ctx)                          # flops per step
    table = {k: dict(ms=ph[k], gflop=pf[k] / 1e9,
                     tflops=(pf[k] / (ph[k] / 1e3) / 1e12) if ph[k] > 0 else None)
             for k in mr.PHASES}
    # the dominant kernel family: the phase with the largest share of the step
    dom = max(mr.PHASES, key=lambda k: ph[k])
    achieved = pf[dom] / (ph[dom] / 1e3) / 1e12
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            res = time_oracle(CPU_SAMPLE_N, 2)
            cpu = dict(value=res["cells"] * 2 / sum(res["times"]), unit="cells/s", cores=1, kind="oracle",
                       sample=oracle_sample_desc(CPU_SAMPLE_N))
        except Exception as e:  # report, do not hide
            cpu = dict(value=None, unit="cells/s", cores=1, kind="oracle", error=str(e)[-300:])
    line = dict(
        metric=METRIC, value=value, unit="cells/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=total_ms / args.steps, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=WORKLOAD if n == 1024 else f"square{n}-qfs", cells=cells,
                    leaves=mr.mrcm_query(solver.ctx, "LEAVES"),
                    levels=mr.mrcm_query(solver.ctx, "LEVELS"),
                    l2="flushed between timed steps (256 MiB write outside the events)",
                    parallelism=f"replicas x{world}"),
        roofline=dict(bound="alu", achieved=achieved, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                      frac=achieved / FP64_PEAK_TFLOPS,
                      traffic=TRAFFIC_PER_LAUNCH[dom]["bytes"] if n == 1024 and dom in TRAFFIC_PER_LAUNCH else None,
                      traffic_unit="bytes per launch",
                      traffic_source=TRAFFIC_PER_LAUNCH[dom]["source"] if n == 1024 and dom in TRAFFIC_PER_LAUNCH else None,
                      kernel=mr.PHASE_KERNELS[dom],
                      phase=dom, share=ph[dom] / (total_ms / args.steps),
                      peak_source="FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"),
        phases=table,
        model_gflop_per_step=sum(pf.values()) / 1e9,
        e2e=dict(value=e2e_value, unit="cells/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
        gpu_launches=launches * args.steps,
        clocks=clocks,
        check=dict(mass_balance=balance, refine_steps=args.refine, rel_l2_vs_refined=rel,
                   tolerance=FP64_FORM_TOL, within_tolerance=bool(max(rel.values()) <= FP64_FORM_TOL),
                   metric_tolerance=1e-8),
        refined_step=dict(refine_steps=1, ms_per_step=sum(ref_ms) / len(ref_ms),
                          value=cells * world / (sum(ref_ms) / len(ref_ms) / 1e3)),
        cpu_baseline=cpu,
    )
    print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
