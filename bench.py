"""Benchmark of the FMM-BEM hot path on the 5000-bubble cluster (3.21M unknowns).

One step = one pass of the hot path on one synthetic cluster: mesh upload, vertex geometry,
octree, singular diagonals (one 4-RHS product), right-hand side, and the GMRES solve for
q = dphi/dn to relative residual 1e-6 (started from zero). The default precision is the
mixed path (FP32 near field and expansions, FP64 geometry/diagonal assembly/GMRES).

Prints one JSON line (rank 0). `--impl reference` times the CPU FP64 oracle on this host's
cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max clock
P2P_FLOPS_PER_PAIR = 20  # per right-hand side: 3 sub, 5 for r^2, rsqrt, 2 for r^-3, 5 for n.d, 4 accumulate


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bubbles", type=int, default=5000)
    ap.add_argument("--level", type=int, default=3)
    ap.add_argument("--p", type=int, default=14)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--fp64-compare", type=int, default=1, help="also time one FP64 step (0 = skip)")
    ap.add_argument("--mvp-reps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=1, help="run the CPU oracle baseline (rank 0)")
    return ap.parse_args()


def workload(args):
    import synth

    mesh, phi = synth.workload_cluster(bubbles=args.bubbles, level=args.level, seed=3)
    return mesh, phi


def workload_name(args, mesh):
    return "cluster of %d icosphere-L%d bubbles (%d unknowns, %d triangles), lognormal radii, seed 3" % (
        args.bubbles, args.level, mesh.n, mesh.t)


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle baseline


def cpu_oracle_step_time(mesh, n_mvps: int, n_recv: int, seed: int = 0) -> dict:
    """Time the oracle's direct off-diagonal product at n_recv random receivers (all N
    sources) and scale to one step of n_mvps full products (each ~N^2 pairs)."""
    import oracle

    s, n = oracle.vertex_geometry(mesh.xyz, mesh.tri)
    recv = oracle.checkpoint_receivers(mesh.n, n_recv, seed)
    x = np.ones(mesh.n)
    t0 = time.perf_counter()
    oracle.offdiag_apply(mesh.xyz, s, n, 1.0, x, 1.0, x, recv)
    dt = time.perf_counter() - t0
    per_mvp = dt * mesh.n / len(recv)
    return {"sample_s": dt, "receivers": int(len(recv)), "per_mvp_s": per_mvp, "step_s": per_mvp * n_mvps,
            "cores": oracle.num_threads()}


# ------------------------------------------------------------------ distributed helpers


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ reference arm


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    mesh, phi = workload(args)
    # The oracle solve at 3.21M unknowns is ~1e13 pair evaluations per product; each step is
    # a bounded sample: the direct product at 4 sqrt(N) receivers, scaled to the step's
    # products (4 diagonal + 1 right-hand side + GMRES iterations + 2; 12 iterations, the
    # count the GPU path takes from a zero start at this size).
    n_mvps = 4 + 1 + 12 + 2
    n_recv = 4 * int(math.isqrt(mesh.n))
    times = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_oracle_step_time(mesh, n_mvps, n_recv, seed=i)
        if i >= args.warmup:
            times.append(info["step_s"])
    v = statistics.mean(times)
    sample = ("direct FP64 product at %d random receivers x %d sources per step, scaled by N/receivers "
              "to %d full products per step" % (info["receivers"], mesh.n, n_mvps))
    line = {
        "impl": "reference", "metric": "wall-s per time step at 3.2M unknowns (resid 1e-6)", "value": v,
        "unit": "s/step", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, mesh), "operator": "direct O(N^2) oracle"},
        "cpu_baseline": {"value": v, "unit": "s/step", "cores": info["cores"], "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_1905_01341_gb300 import bem, build

    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    mesh, phi = workload(args)
    prec = bem.BEM_PREC_MIXED if args.precision == "mixed" else bem.BEM_PREC_FP64

    xyz_h = mesh.xyz_soa()
    tri_h = mesh.tri_soa()
    voff_h = np.ascontiguousarray(mesh.vert_off, np.int64)
    toff_h = np.ascontiguousarray(mesh.tri_off, np.int64)
    phi_h = np.ascontiguousarray(phi)
    xyz = torch.from_numpy(xyz_h).to(dev)
    tri = torch.from_numpy(tri_h).to(dev)
    voff = torch.from_numpy(voff_h).to(dev)
    toff = torch.from_numpy(toff_h).to(dev)
    phid = torch.from_numpy(phi_h).to(dev)
    q = torch.zeros(mesh.n, dtype=torch.float64, device=dev)

    ctx = bem.BemContext(stream=stream, p_fmm=args.p, precision=prec, leaf_target=args.leaf, gmres_tol=args.tol)

    def step():
        ctx.upload(xyz, tri, voff, toff)
        ctx.build()
        q.zero_()
        return ctx.solve(phid, q)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st0 = ctx.stats()
    bem.bem_profile_enable(ctx.ctx, True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        it, rr = step()
        iters.append((it, rr))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    prof = bem.bem_profile_read(ctx.ctx)
    bem.bem_profile_enable(ctx.ctx, False)
    st1 = ctx.stats()
    ms = max_over_ranks(world, ms)

    # one operator product (single layer), timed on its own
    out = torch.empty(mesh.n, dtype=torch.float64, device=dev)
    for _ in range(2):
        ctx.apply(1.0, q, 0.0, None, out)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.mvp_reps):
        ctx.apply(1.0, q, 0.0, None, out)
    a1.record(stream)
    torch.cuda.synchronize()
    mvp_ms = a0.elapsed_time(a1) / args.mvp_reps

    # e2e through the C ABI with host buffers (copies inside the timed region)
    q_h = np.zeros(mesh.n)
    e2e_times = []
    for i in range(1 + max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bem.bem_mesh_upload(ctx.ctx, mesh.n, xyz_h, mesh.t, tri_h, mesh.m, voff_h, toff_h)
        bem.fmm_build(ctx.ctx)
        q_h[:] = 0.0
        bem.bem_solve(ctx.ctx, phi_h, q_h)
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e_times)
    h2d = xyz_h.nbytes + tri_h.nbytes + voff_h.nbytes + toff_h.nbytes + phi_h.nbytes + q_h.nbytes
    d2h = q_h.nbytes

    st = ctx.stats()
    nmv_step = (st1["n_apply"] - st0["n_apply"]) / args.steps
    it_mean = statistics.mean(i for i, _ in iters)

    # roofline of the dominant kernel (device time inside the timed region)
    per_step = {k: v[0] / args.steps for k, v in prof.items()}
    work = {}
    R1_applies = nmv_step - 1  # products with one right-hand side per step (the diagonal is 4-RHS)
    rhs_per_step = R1_applies + 4
    work["p2p"] = ("alu", P2P_FLOPS_PER_PAIR * st["p2p_pairs"] * rhs_per_step, FP32_ALU_PEAK_TFLOPS,
                   prof["p2p"][1] / args.steps)
    P = args.p * args.p
    work["m2l"] = ("alu", 2.0 * P * P * st["m2l_pairs"] * rhs_per_step, FP32_ALU_PEAK_TFLOPS,
                   prof["m2l"][1] / args.steps)
    cand = [k for k in ("p2p", "m2l") if per_step.get(k, 0) > 0]
    dom = max(cand, key=lambda k: per_step[k]) if cand else None
    roof = None
    if dom:
        bound, flops, peak, launches = work[dom]
        launches = max(1, launches)
        t_launch = per_step[dom] / 1e3 / launches
        achieved = flops / launches / t_launch / 1e12
        if args.precision == "fp64":
            peak = None
        roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if peak else None, "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                "launch_ms": t_launch * 1e3, "launches_per_step": launches}

    line = {
        "metric": "wall-s per time step & FMM matvec Gpairs/s at 3.2M unknowns, resid 1e-6, vs FP64",
        "value": ms / 1e3, "unit": "s/step", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == bem.BEM_PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, mesh), "p_fmm": args.p, "precision": args.precision,
                   "leaf_target": args.leaf, "gmres_tol": args.tol, "x0": "zero",
                   "levels": st["levels"], "leaves": st["leaves"], "l2": "inputs and working set > L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "solve": {"iters": it_mean, "relres": iters[-1][1], "mvps_per_step": nmv_step},
        "mvp": {"ms": mvp_ms, "gpairs_per_s_dense_equiv": mesh.n ** 2 / (mvp_ms / 1e3) / 1e9,
                "p2p_pairs": st["p2p_pairs"], "m2l_pairs": st["m2l_pairs"]},
        "phases_ms_per_step": {k: round(v, 3) for k, v in per_step.items() if v > 0},
        "roofline": roof,
        "e2e": {"value": e2e_s, "unit": "s/step", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int((st1["n_launches"] - st0["n_launches"]) / args.steps),
        "clocks": clk,
    }

    if args.fp64_compare and prec == bem.BEM_PREC_MIXED:
        ctx64 = bem.BemContext(stream=stream, p_fmm=args.p, precision=bem.BEM_PREC_FP64, leaf_target=args.leaf,
                               gmres_tol=args.tol)

        def step64():
            ctx64.upload(xyz, tri, voff, toff)
            ctx64.build()
            q.zero_()
            return ctx64.solve(phid, q)

        step64()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        it64, rr64 = step64()
        f1.record(stream)
        torch.cuda.synchronize()
        line["fp64_compare"] = {"s_per_step": f0.elapsed_time(f1) / 1e3, "iters": it64, "relres": rr64,
                                "timed_steps": 1, "warmup": 1}
        ctx64.close()

    if rank == 0 and args.cpu_sample:
        n_recv = 4 * int(math.isqrt(mesh.n))
        info = cpu_oracle_step_time(mesh, int(round(nmv_step)) + 1, n_recv)
        line["cpu_baseline"] = {
            "value": info["step_s"], "unit": "s/step", "cores": info["cores"], "kind": "oracle",
            "sample": "direct FP64 product at %d random receivers x %d sources (%.1f s), scaled by N/receivers to "
                      "%d full products per step" % (info["receivers"], mesh.n, info["sample_s"],
                                                     int(round(nmv_step)) + 1)}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
