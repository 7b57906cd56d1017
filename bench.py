"""Benchmark of the FMM-BEM hot path on the 5000-bubble cluster (3.21M unknowns).

One step = one time step of the bubble-dynamics method (bem_step): shape filter, vertex
geometry, octree, singular diagonals (one 4-RHS product), right-hand side, GMRES solve for
q = dphi/dn to relative residual 1e-6 warm-started from the previous q, tangential velocity,
curvature, volumes and gas pressure, and the 6th-order Adams-Bashforth update. The warm-up
steps are the 4th-order Runge-Kutta start (the first solve starts from zero). The default
precision is the mixed path (FP32 near field and expansions; FP64 geometry, diagonal
assembly, GMRES and time integration).

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

METRIC = "wall-s per time step & FMM matvec Gpairs/s at 3.2M unknowns, resid 1e-6, vs FP64"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 flops x max clock
# Algorithmic FP32 flops per near-field pair, per kernel variant (rsqrt counted as one):
#   single layer: 3 (r_i - r_j) + 5 (r^2) + 1 (rsqrt) + 2 (q / r accumulated)          = 11
#   double layer: 3 + 5 + 1 + 2 (r^-3) + 5 (n . d) + 1 (scale) + 2 (w n.d / r^3 acc.)  = 19
#   both layers, 4 RHS (diagonal product): 3 + 5 + 1 + 2 + 5 + 1 + 4 x (2 + 2)         = 33
P2P_FLOPS_SL, P2P_FLOPS_DL, P2P_FLOPS_4RHS = 11, 19, 33


def progress(msg: str) -> None:
    """One line of progress on stderr (the JSON result goes to stdout)."""
    print("[bench] " + msg, file=sys.stderr, flush=True)


def _load_peaks() -> dict:
    """Measured HBM / BF16 peaks of this GPU pool, when present beside this file."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PEAKS = _load_peaks()
# Tensor-core M2L: six BF16 products per translation (three-piece split of both operands).
M2L_TC_PRODUCTS = 6
# DRAM traffic per unit from the ncu capture of the 2000-bubble cluster at depth 5 (profiles/;
# 1,284,000 points, 2,231,186 translations: large enough that the near field's shares and the
# M2L's partial expansions leave L2), scaled to a full launch by the units it processes. Near
# field (symmetric kernel + gather of the shares): 25.2 + 22.5 MB and 89.5 + 0.3 MB; target-major
# M2L: 228.7 MB read (gathered multipoles, operator blocks) + 269.4 MB written (partials).
P2P_DRAM_BYTES_PER_POINT = (25.21e6 + 22.49e6 + 89.54e6 + 0.34e6) / 1284000
M2L_DRAM_BYTES_PER_TRANSLATION = (228.67e6 + 269.36e6) / 2231186


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cluster", choices=["cluster", "batched", "learned"],
                    help="cluster: the 5000-bubble headline; batched: 64 uneven independent clusters in "
                         "one launch per phase; learned: record/train/use the learned GMRES guess")
    ap.add_argument("--learn-bubbles", type=int, default=1000)
    ap.add_argument("--learn-summary", type=int, default=100,
                    help="bubbles of the reduced learned-guess run reported in the default line (0 = skip)")
    ap.add_argument("--learn-steps", type=int, default=100, help="recorded steps, then as many compared")
    ap.add_argument("--bubbles", type=int, default=5000)
    ap.add_argument("--level", type=int, default=3)
    ap.add_argument("--p", type=int, default=14)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--leaf", type=int, default=0, help="mean points per leaf; 0 = autotune the octree depth")
    ap.add_argument("--tree-level", type=int, default=0, help="fixed octree depth (0 = from --leaf)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--maxit", type=int, default=400)
    ap.add_argument("--restart", type=int, default=100)
    ap.add_argument("--precond", type=int, default=2,
                    help="GMRES right preconditioning: 0 none (the paper), 1 Jacobi, 2 bubble blocks")
    ap.add_argument("--m2l-tc", type=int, default=3,
                    help="M2L on the tensor cores: 1 single-RHS products, 2 also the 4-RHS diagonal product, "
                         "3 (default) as 2 for bubbles of at most 2562 vertices, 0 none")
    ap.add_argument("--overlap", type=int, default=-1,
                    help="near field on its own stream: 1 from the far field's start, 2 from the M2L's, 0 off, "
                         "-1 autotuned")
    ap.add_argument("--guess", type=int, default=2,
                    help="AB6 GMRES start: 0 previous q (the paper), 1/2/3 extrapolation in t of that degree")
    ap.add_argument("--pa", type=float, default=0.5, help="acoustic amplitude Pa/p0")
    ap.add_argument("--pf", type=int, default=6, help="shape-filter bandwidth")
    ap.add_argument("--fp64-compare", type=int, default=1,
                    help="also time the plain FP64 FMM-BEM step from the same checkpoint (0 = skip)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="FP64 steps timed (at most --steps)")
    ap.add_argument("--mvp-reps", type=int, default=5)
    ap.add_argument("--eps-bubbles", type=int, default=300, help="cluster size of the dynamics-error run (0 = skip)")
    ap.add_argument("--eps-steps", type=int, default=20, help="steps of the dynamics-error run")
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


def oracle_solve_residual(case, tri, n_recv: int, seed: int) -> dict:
    """True relative residual of a GPU solution q of L q = b, b = -phi/2 + M phi, against the
    oracle's dense discrete operator (FP64 direct sums, identity diagonals), estimated at
    n_recv random receivers (the paper's checkpoint method): |(b - L q)_recv| / |b_recv|."""
    import oracle

    xyz, phi, q = case["xyz"], case["phi"], case["q"]
    s, nrm = oracle.vertex_geometry(xyz, tri)
    recv = oracle.checkpoint_receivers(xyz.shape[0], n_recv, seed)
    t0 = time.perf_counter()
    ld, md = oracle.diagonals(xyz, s, nrm, recv)
    b = -0.5 * phi[recv] + oracle.offdiag_apply(xyz, s, nrm, 0.0, None, 1.0, phi, recv) + md * phi[recv]
    lq = oracle.offdiag_apply(xyz, s, nrm, 1.0, q, 0.0, None, recv) + ld * q[recv]
    rr = float(np.linalg.norm(b - lq) / np.linalg.norm(b))
    return {"oracle_relres_at_receivers": rr, "receivers": int(len(recv)), "gpu_relres": case["gpu_relres"],
            "gmres_iters": case["gmres_iters"], "oracle_s": time.perf_counter() - t0,
            "what": "GPU solve (mixed, tolerance as configured) of the current state; true residual against the "
                    "CPU FP64 oracle's operator at sampled receivers"}


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
    # products as the GPU path counts them for an AB6 step at this size with the default solver
    # settings (4 for the diagonals, 1 for the right-hand side, 11 GMRES iterations from the
    # extrapolated guess and 3 initial/true-residual products).
    n_mvps = 4 + 1 + 11 + 3
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
        "impl": "reference", "metric": METRIC, "value": v,
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
    N = mesh.n

    xyz = torch.from_numpy(mesh.xyz_soa()).to(dev)
    tri = torch.from_numpy(mesh.tri_soa()).to(dev)
    voff = torch.from_numpy(np.ascontiguousarray(mesh.vert_off, np.int64)).to(dev)
    toff = torch.from_numpy(np.ascontiguousarray(mesh.tri_off, np.int64)).to(dev)
    phid = torch.from_numpy(np.ascontiguousarray(phi)).to(dev)

    def make_ctx(precision, overlap=None, fixed_level=None):
        overlap = args.overlap if overlap is None else overlap
        c = bem.BemContext(stream=stream, p_fmm=args.p, precision=precision, leaf_target=args.leaf,
                           fixed_level=args.tree_level if fixed_level is None else fixed_level, gmres_tol=args.tol,
                           gmres_maxit=args.maxit, gmres_restart=args.restart, gmres_precond=args.precond,
                           m2l_tensor_cores=args.m2l_tc, overlap=overlap)
        return c

    progress("workload ready: %d unknowns, %d bubbles" % (N, mesh.m))
    ctx = make_ctx(prec)
    ctx.upload(xyz, tri, voff, toff)
    sp = bem.bem_step_params_default(pa=args.pa, pf=args.pf, guess=args.guess)
    bem.bem_step_init(ctx.ctx, phid, sp)

    warm = []
    for _ in range(args.warmup):
        t0 = time.perf_counter()
        warm.append(bem.bem_step(ctx.ctx))
        progress("warm-up step %d: %.2f s, %d GMRES iterations, %d not converged, levels %d" % (
            len(warm), time.perf_counter() - t0, warm[-1]["gmres_iters"], warm[-1]["nonconverged"],
            ctx.stats()["levels"]))
    torch.cuda.synchronize()
    # checkpoint of the state after the warm-up: the FP64 comparison below replays the timed
    # steps from it
    ck = torch.empty(bem.bem_step_save(ctx.ctx), dtype=torch.uint8, device=dev)
    bem.bem_step_save(ctx.ctx, ck)
    st0 = ctx.stats()
    bem.bem_profile_enable(ctx.ctx, True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        infos.append(bem.bem_step(ctx.ctx))
        ev[k + 1].record(stream)
        progress("timed step %d: %d GMRES iterations" % (len(infos), infos[-1]["gmres_iters"]))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / args.steps
    for k in range(args.steps):
        infos[k]["dev_s"] = ev[k].elapsed_time(ev[k + 1]) / 1e3
    clk = clocks.stop()
    prof = bem.bem_profile_read(ctx.ctx)
    bem.bem_profile_enable(ctx.ctx, False)
    st1 = ctx.stats()
    ms = max_over_ranks(world, ms)

    # one single-layer product on the current geometry, timed on its own
    q = torch.zeros(N, dtype=torch.float64, device=dev)
    bem.bem_step_get_state(ctx.ctx, None, None, q)
    out = torch.empty(N, dtype=torch.float64, device=dev)
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
    st = ctx.stats()

    # per-kernel timings for the rooflines: in the step the near field overlaps the far field on
    # two streams, so each kernel's own duration is taken from single-layer products of the same
    # geometry and depth on a context that runs the phases one after another
    xs_now = torch.empty(3 * N, dtype=torch.float64, device=dev)
    bem.bem_step_get_state(ctx.ctx, xs_now, None, None)
    ctx_iso = make_ctx(prec, overlap=0, fixed_level=st["levels"])
    ctx_iso.upload(xs_now.view(3, N), tri, voff, toff)
    ctx_iso.build()
    for _ in range(2):
        ctx_iso.apply(1.0, q, 0.0, None, out)
    torch.cuda.synchronize()
    bem.bem_profile_enable(ctx_iso.ctx, True)
    for _ in range(args.mvp_reps):
        ctx_iso.apply(1.0, q, 0.0, None, out)
    iso = bem.bem_profile_read(ctx_iso.ctx)
    st_iso = ctx_iso.stats()
    # one Dirichlet solve on the current geometry and potential with the step's solver settings,
    # for the full-size solve parity (its true residual against the oracle's operator is
    # evaluated at sampled receivers in the CPU oracle leg below)
    ph_now = torch.empty(N, dtype=torch.float64, device=dev)
    bem.bem_step_get_state(ctx.ctx, None, ph_now, None)
    q_sol = q.clone()
    sol_it, sol_rr = ctx_iso.solve(ph_now, q_sol, raise_on_noconv=False)
    solve_case = {"xyz": xs_now.cpu().numpy().reshape(3, N).T.copy(), "phi": ph_now.cpu().numpy(),
                  "q": q_sol.cpu().numpy(), "gpu_relres": sol_rr, "gmres_iters": sol_it}
    ctx_iso.close()
    del xs_now, q_sol

    # end to end through the C ABI, with the state held in pinned host memory: every step copies
    # the state (r, phi, q) from the host into the context, advances, and reads the new state
    # back to the host
    xyz_h = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    phi_h = torch.empty(N, dtype=torch.float64).pin_memory()
    q_h = torch.empty(N, dtype=torch.float64).pin_memory()
    bem.bem_step_get_state(ctx.ctx, xyz_h, phi_h, q_h)
    # (these are the steps after the timed ones: their GMRES iteration counts and device times
    # are reported beside the host-clock value)
    e2e_t, e2e_dev, e2e_it = [], [], []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        d0.record(stream)
        bem.bem_step_set_state(ctx.ctx, xyz_h, phi_h, q_h)
        info = bem.bem_step(ctx.ctx)
        bem.bem_step_get_state(ctx.ctx, xyz_h, phi_h, q_h)
        d1.record(stream)
        e2e_t.append(time.perf_counter() - t0)
        torch.cuda.synchronize()
        e2e_dev.append(d0.elapsed_time(d1) / 1e3)
        e2e_it.append(info["gmres_iters"])
    e2e_s = statistics.mean(e2e_t)
    d2h = (xyz_h.numel() + phi_h.numel() + q_h.numel()) * 8
    h2d = d2h

    rhs = sum(i["rhs_calls"] for i in infos)
    mvps = sum(i["mvps"] for i in infos)
    iters = sum(i["gmres_iters"] for i in infos)
    n_r4 = rhs                  # one 4-RHS diagonal product per right-hand side
    n_r1 = mvps - rhs           # single-RHS products (right-hand side b and GMRES)
    per_step = {k: v[0] / args.steps for k, v in prof.items()}
    P = args.p * args.p
    n_dl = rhs                  # b = -phi/2 + M phi: double layer only, once per right-hand side
    n_sl = n_r1 - n_dl          # GMRES products (and restart residuals): single layer only
    pairs = st["p2p_pairs"]
    work = {
        "p2p": (P2P_FLOPS_SL * n_sl + P2P_FLOPS_DL * n_dl + P2P_FLOPS_4RHS * n_r4) * pairs / args.steps,
        "m2l": 2.0 * st["m2l_macs"] * (n_r1 + 4 * n_r4) / args.steps,
    }
    launches = {k: prof[k][1] / args.steps for k in ("p2p", "m2l")}

    def p2p_roofline():
        ms_i, n_i = iso.get("p2p", (0.0, 0))
        if n_i <= 0 or ms_i <= 0:
            return None
        t_launch = ms_i / 1e3 / n_i
        achieved = P2P_FLOPS_SL * st_iso["p2p_pairs"] / t_launch / 1e12
        peak = FP32_ALU_PEAK_TFLOPS if prec == bem.BEM_PREC_MIXED else None
        kname = ("k_p2p_units_x2 + k_p2p_back_gather (near field, single layer, symmetric)"
                 if prec == bem.BEM_PREC_MIXED else "k_p2p_units (near field, single layer)")
        return {"kernel": kname, "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if peak else None,
                "traffic": P2P_DRAM_BYTES_PER_POINT * N if prec == bem.BEM_PREC_MIXED else None,
                "traffic_source": "ncu capture of the 2000-bubble cluster, bytes per point x N (both kernels)",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (max SM clock)",
                "launch_ms": t_launch * 1e3, "launches_timed": n_i,
                "launch_ms_in_step": per_step.get("p2p", 0) / max(1.0, launches["p2p"]),
                "work_per_launch": "11 flops x %d near-field pairs (algorithmic; the symmetric kernel evaluates "
                                   "each pair of distinct leaves once for both directions)" % st_iso["p2p_pairs"],
                "timing": "single-layer products on the step's geometry, phases run one after another"}

    def m2l_roofline():
        # tensor-core translations (with the split of the multipoles into BF16 pieces) against
        # the measured sustained BF16 peak
        ms_i, n_i = iso.get("m2l", (0.0, 0))
        if not (prec == bem.BEM_PREC_MIXED and args.m2l_tc and n_i > 0 and ms_i > 0):
            return None
        t_launch = ms_i / 1e3 / n_i
        achieved = M2L_TC_PRODUCTS * 2.0 * st_iso["m2l_macs"] / t_launch / 1e12
        pk = PEAKS.get("bf16_tflops_sustained")
        return {"kernel": "k_m2l_tm (M2L, target-major)", "bound": "tensor", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk if pk else None,
                "traffic": M2L_DRAM_BYTES_PER_TRANSLATION * st_iso["m2l_pairs"],
                "traffic_source": "ncu capture of the 2000-bubble cluster, bytes per translation x translations",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS, long loop)",
                "launch_ms": t_launch * 1e3, "launches_timed": n_i,
                "launch_ms_in_step": per_step.get("m2l", 0) / max(1.0, launches["m2l"]),
                "work_per_launch": "6 BF16 products x 2 flops x %d multiply-adds (%d M2L translations, each "
                                   "truncated to its class's order, sizes padded to 16; the target-major tiles "
                                   "also multiply zero rows, not counted)" % (st_iso["m2l_macs"], st_iso["m2l_pairs"]),
                "timing": "single-layer products on the step's geometry, phases run one after another"}

    roof_p2p, roof_m2l = p2p_roofline(), m2l_roofline()
    dom = "m2l" if roof_m2l and iso.get("m2l", (0, 0))[0] > iso.get("p2p", (0, 0))[0] else "p2p"
    roof = roof_m2l if dom == "m2l" else roof_p2p

    line = {
        "metric": METRIC,
        "value": ms / 1e3, "unit": "s/step", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == bem.BEM_PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": workload_name(args, mesh), "p_fmm": args.p, "precision": args.precision,
                   "leaf_target": args.leaf, "gmres_tol": args.tol, "gmres_precond": args.precond,
                   "m2l_tensor_cores": args.m2l_tc, "overlap": args.overlap, "guess": args.guess,
                   "scheme": ("AB6 (steps after the 5 RK4 start steps)" if rhs / args.steps < 2 else
                              "RK4 start steps (the paper's AB6 begins after 5)"),
                   "pa": args.pa, "pf": args.pf, "dt": infos[-1]["dt"], "levels": st["levels"],
                   "leaves": st["leaves"], "l2": "inputs and working set > L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "step": {"rhs_calls": rhs / args.steps, "gmres_iters": iters / args.steps, "mvps": mvps / args.steps,
                 "max_relres": max(i["max_relres"] for i in infos),
                 "nonconverged": sum(i["nonconverged"] for i in infos),
                 "warmup_gmres_iters": [w["gmres_iters"] for w in warm]},
        "mvp": {"ms": mvp_ms, "gpairs_per_s_dense_equiv": N ** 2 / (mvp_ms / 1e3) / 1e9,
                "p2p_pairs": st["p2p_pairs"], "m2l_pairs": st["m2l_pairs"]},
        "phases_ms_per_step": {k: round(v, 3) for k, v in per_step.items() if v > 0},
        "phases_note": "per-stream device time; the near field (p2p) overlaps the far field",
        "kernel_ms_per_product": {k: round(v[0] / max(1, v[1]), 4) for k, v in iso.items() if v[1] > 0},
        "roofline": roof,
        "roofline_p2p": roof_p2p,
        "roofline_m2l": roof_m2l,
        "e2e": {"value": e2e_s, "unit": "s/step", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "device_s_per_step": statistics.mean(e2e_dev), "gmres_iters_per_step": statistics.mean(e2e_it),
                "what": "host clock per step: bem_step_set_state from pinned host buffers (r, phi, q), bem_step, "
                        "bem_step_get_state back into them"},
        "gpu_launches": int((st1["n_launches"] - st0["n_launches"]) / args.steps),
        "clocks": clk,
    }

    if args.fp64_compare and prec == bem.BEM_PREC_MIXED:
        # the plain FP64 FMM-BEM on the same GPU, like for like: the same checkpoint (state,
        # Adams-Bashforth history, extrapolation history), the same octree depth, preconditioner,
        # initial guess and tolerance; its operators, buffers and preconditioner are built by one
        # untimed step from the checkpoint, then the checkpoint is loaded again and the same
        # steps as the mixed path's timed ones are timed with CUDA events
        n64 = max(1, min(args.steps, args.fp64_steps))
        progress("FP64 comparison: %d AB6 steps from the warm-up checkpoint" % n64)
        ctx64 = make_ctx(bem.BEM_PREC_FP64, fixed_level=st["levels"])
        ctx64.upload(xyz, tri, voff, toff)
        bem.bem_step_load(ctx64.ctx, ck)
        bem.bem_step(ctx64.ctx)
        bem.bem_step_load(ctx64.ctx, ck)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        infos64 = [bem.bem_step(ctx64.ctx) for _ in range(n64)]
        f1.record(stream)
        torch.cuda.synchronize()
        s64 = f0.elapsed_time(f1) / 1e3 / n64
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        ctx64.apply(1.0, q, 0.0, None, out)
        g1.record(stream)
        torch.cuda.synchronize()
        mixed_same = sum(e["dev_s"] for e in infos[:n64]) / n64
        line["fp64_compare"] = {
            "s_per_step": s64, "steps": n64, "gmres_iters_per_step": sum(i["gmres_iters"] for i in infos64) / n64,
            "max_relres": max(i["max_relres"] for i in infos64), "mvp_ms": g0.elapsed_time(g1),
            "mixed_s_per_step_same_steps": mixed_same,
            "mixed_gmres_iters_same_steps": sum(i["gmres_iters"] for i in infos[:n64]) / n64,
            "speedup_mixed_vs_fp64": s64 / mixed_same,
            "what": "AB6 steps from the same checkpoint as the mixed path's first timed steps: same depth, "
                    "preconditioner, guess and GMRES tolerance; FP64 throughout"}
        ctx64.close()
    del ck

    if args.eps_steps > 0 and args.eps_bubbles > 0 and prec == bem.BEM_PREC_MIXED:
        line["dynamics_error"] = dynamics_error(args, bem, stream)
    if args.learn_summary > 0:
        progress("learned guess: %d bubbles, %d + %d steps" % (args.learn_summary, 40, 20))
        line["learned_guess"] = learned_guess_run(args, bem, stream, args.learn_summary, 40, 20)

    if rank == 0 and args.cpu_sample:
        n_recv = 4 * int(math.isqrt(N))
        n_mv = int(round(mvps / args.steps)) + 3 * int(round(rhs / args.steps))  # 4-RHS products count 4
        info = cpu_oracle_step_time(mesh, n_mv, n_recv)
        line["cpu_baseline"] = {
            "value": info["step_s"], "unit": "s/step", "cores": info["cores"], "kind": "oracle",
            "sample": "direct FP64 product at %d random receivers x %d sources (%.1f s), scaled by N/receivers to "
                      "%d full single-RHS products per step (the GPU step's product count)" % (
                          info["receivers"], N, info["sample_s"], n_mv)}
        line["solve_parity"] = oracle_solve_residual(solve_case, mesh.tri, 400, seed=41)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def dynamics_error(args, bem, stream) -> dict:
    """Eq. (eqErr): eps(t) = |x(t) - x_ref(t)|_2 / max_{tau <= t} |x_ref(tau) - x_ref(0)|_2 over the
    surface-point coordinates, of this benchmark's mixed-precision step against the FP64 path at
    p + 2 with GMRES to 1e-10 (the reference run), on a smaller cluster of the same recipe."""
    import synth
    import torch

    mesh, phi = synth.workload_cluster(bubbles=args.eps_bubbles, level=args.level, seed=3)
    sp = bem.bem_step_params_default(pa=args.pa, pf=args.pf, guess=args.guess)
    runs, secs = {}, {}
    for key, prm in (("mixed", dict(precision=bem.BEM_PREC_MIXED, p_fmm=args.p, gmres_tol=args.tol)),
                     ("ref", dict(precision=bem.BEM_PREC_FP64, p_fmm=min(args.p + 2, 20), gmres_tol=1e-10))):
        progress("dynamics error: %s run, %d steps of %d bubbles" % (key, args.eps_steps, args.eps_bubbles))
        c = bem.BemContext(stream=stream, leaf_target=args.leaf, gmres_maxit=args.maxit, gmres_restart=args.restart,
                           gmres_precond=args.precond, m2l_tensor_cores=args.m2l_tc, **prm)
        c.upload_mesh(mesh)
        bem.bem_step_init(c.ctx, phi, sp)
        xs, nc = [], 0
        t0 = time.perf_counter()
        for _ in range(args.eps_steps):
            nc += bem.bem_step(c.ctx)["nonconverged"]
            x = np.zeros(3 * mesh.n)
            bem.bem_step_get_state(c.ctx, x)
            xs.append(x)
        torch.cuda.synchronize()
        secs[key] = time.perf_counter() - t0
        runs[key] = (xs, nc)
        c.close()
    x0 = mesh.xyz_soa().reshape(-1)
    span, eps = 0.0, []
    for x, xr in zip(runs["mixed"][0], runs["ref"][0]):
        span = max(span, float(np.linalg.norm(xr - x0)))
        eps.append(float(np.linalg.norm(x - xr)) / span)
    return {"eps_final": eps[-1], "eps_max": max(eps), "eps_by_step": [float("%.3e" % e) for e in eps],
            "steps": args.eps_steps, "nonconverged": {k: v[1] for k, v in runs.items()},
            "wall_s": secs,
            "config": "%d icosphere-L%d bubbles (%d unknowns), seed 3; test: this benchmark's configuration; reference: "
                      "FP64, p = %d, GMRES 1e-10" % (args.eps_bubbles, args.level, mesh.n, min(args.p + 2, 20))}


def run_batched(args):
    """64 independent clusters of uneven size stepped together: one octree per cluster (cluster
    id in the key), one launch per phase for all of them, one GMRES over the block-diagonal
    system. Every cluster's step completes with the batch, so its latency is the batch step
    time; a sample of clusters is also stepped alone for the unbatched latency."""
    import torch
    import synth
    from paper_1905_01341_gb300 import bem, build

    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    cl = synth.workload_uneven_clusters(64, seed=5)
    mesh, phi, boff = synth.concat_meshes([c[0] for c in cl], [c[1] for c in cl])
    prec = bem.BEM_PREC_MIXED if args.precision == "mixed" else bem.BEM_PREC_FP64

    def stepper(m, ph, clusters=None):
        c = bem.BemContext(stream=stream, p_fmm=args.p, precision=prec, leaf_target=args.leaf, gmres_tol=args.tol,
                           gmres_maxit=args.maxit, gmres_restart=args.restart, gmres_precond=args.precond)
        c.upload_mesh(m)
        if clusters is not None:
            bem.bem_mesh_set_clusters(c.ctx, len(clusters) - 1, clusters)
        bem.bem_step_init(c.ctx, ph, bem.bem_step_params_default(pa=args.pa, pf=args.pf, guess=args.guess))
        return c

    ctx = stepper(mesh, phi, boff)
    for _ in range(args.warmup):
        bem.bem_step(ctx.ctx)
    torch.cuda.synchronize()
    st0 = ctx.stats()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    C = len(boff) - 1
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    infos, cstats = [], []
    e0.record(stream)
    ev[0].record(stream)
    for k in range(args.steps):
        infos.append(bem.bem_step(ctx.ctx))
        ev[k + 1].record(stream)
        cstats.append(bem.bem_get_cluster_stats(ctx.ctx, C))  # the step's (last) solve
    e1.record(stream)
    torch.cuda.synchronize()
    st1 = ctx.stats()
    batch_s = e0.elapsed_time(e1) / 1e3 / args.steps
    # per-cluster step latency: the step's work before and after its solve (shared by all
    # clusters) plus the time from the solve's start until the cluster's own solution was final
    lat = []
    for k in range(args.steps):
        step_ms = ev[k].elapsed_time(ev[k + 1])
        lat.extend(step_ms - cstats[k]["solve_ms"] + cstats[k]["done_ms"])
    lat = np.sort(np.asarray(lat)) / 1e3
    iters_c = np.concatenate([x["iters"] for x in cstats])
    ctx.close()
    # unbatched latency of a few clusters (smallest, median, largest)
    order = np.argsort([c[0].n for c in cl])
    alone = {}
    for k in (order[0], order[len(order) // 2], order[-1]):
        m, ph = cl[k]
        c = stepper(m, ph)
        for _ in range(args.warmup):
            bem.bem_step(c.ctx)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            bem.bem_step(c.ctx)
        f1.record(stream)
        torch.cuda.synchronize()
        alone[int(m.n)] = f0.elapsed_time(f1) / 1e3 / args.steps
        c.close()
    seq_estimate = None
    line = {
        "metric": "batched step of 64 independent uneven clusters", "workload": "batched",
        "value": batch_s, "unit": "s/step", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "dtype": "f32+f64" if prec == bem.BEM_PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "64 clusters, 1-200 bubbles each, icosphere levels 2-4, seed 5 (%d unknowns, %d bubbles)"
                               % (mesh.n, mesh.m), "p_fmm": args.p, "gmres_tol": args.tol},
        "aggregate_unknown_steps_per_s": mesh.n / batch_s,
        "per_cluster_latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                  "min": float(lat[0]), "max": float(lat[-1]), "samples": int(len(lat)),
                                  "what": "per timed step and cluster: the step's shared work before and after "
                                          "its solve plus the device time until the cluster's own GMRES met "
                                          "the tolerance and took its solution (one GMRES per cluster, in "
                                          "lockstep)"},
        "per_cluster_gmres_iters": {"p50": float(np.percentile(iters_c, 50)), "max": int(iters_c.max())},
        "alone_latency_s_by_size": alone,
        "step": {"gmres_iters": sum(i["gmres_iters"] for i in infos) / args.steps,
                 "max_relres": max(i["max_relres"] for i in infos)},
        "gpu_launches": int((st1["n_launches"] - st0["n_launches"]) / args.steps),
    }
    del seq_estimate
    print(json.dumps(line), flush=True)


def learned_guess_run(args, bem, stream, nb, rec_steps, cmp_steps, epochs=30, seed=4) -> dict:
    """Learned GMRES initial guess on a cluster of the learned-guess recipe (nb bubbles of icosphere
    level 3 or 4, lognormal radii, seed-fixed): record the Adams-Bashforth solves of rec_steps steps,
    train the network on the device, then step on cmp_steps steps starting every solve from the
    learned guess while also solving from the base start (compare mode). A second run of the same
    cluster with the paper's start (the previous step's q, guess = 0) gives the third count over the
    same steps."""
    import torch
    import synth

    rng = np.random.Generator(np.random.PCG64(seed))
    radii = np.exp(0.3 * rng.standard_normal(nb))
    centres = synth._place_centres(radii, 4.0 * nb ** (1 / 3), 0.5, rng)
    levels = rng.choice(np.array([3, 4]), size=nb)
    mesh = synth.cluster(levels, radii, centres)
    phi = synth.cluster_potential(mesh, 6, 0.01, rng, radius_scaled=True)
    prec = bem.BEM_PREC_MIXED if args.precision == "mixed" else bem.BEM_PREC_FP64

    def stepper(guess):
        c = bem.BemContext(stream=stream, p_fmm=args.p, precision=prec, leaf_target=args.leaf, gmres_tol=args.tol,
                           gmres_maxit=args.maxit, gmres_restart=args.restart, gmres_precond=args.precond)
        c.upload_mesh(mesh)
        bem.bem_step_init(c.ctx, phi, bem.bem_step_params_default(pa=args.pa, pf=args.pf, guess=guess))
        return c

    ctx = stepper(args.guess)
    bem.bem_mlp_init(ctx.ctx, hidden=256, lmax=10, seed=1)
    bem.bem_mlp_set_mode(ctx.ctx, record=True)
    t0 = time.perf_counter()
    for _ in range(rec_steps):
        bem.bem_step(ctx.ctx)
    t_rec = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    l0 = bem.bem_mlp_train(ctx.ctx, epochs=1, batch=1024, lr=1e-3)
    l1 = bem.bem_mlp_train(ctx.ctx, epochs=epochs, batch=1024, lr=1e-3)
    t_train = time.perf_counter() - t0
    bem.bem_mlp_set_mode(ctx.ctx, record=False, use_guess=True, compare=True)
    for _ in range(cmp_steps):
        bem.bem_step(ctx.ctx)
    info = bem.bem_mlp_info(ctx.ctx)
    ctx.close()
    c0 = stepper(0)
    it0 = []
    for k in range(rec_steps + cmp_steps):
        st = bem.bem_step(c0.ctx)
        if k >= rec_steps:
            it0.append(st["gmres_iters"])
    c0.close()
    n = max(1, info["compared_solves"])
    return {
        "gmres_iters_per_solve": {"learned": info["iters_guess"] / n,
                                  ("extrapolated" if args.guess else "previous_step"): info["iters_fallback"] / n,
                                  "previous_step_q": sum(it0) / max(1, len(it0))},
        "initial_relres": {"learned": info["res0_guess"] / n,
                           ("extrapolated" if args.guess else "previous_step"): info["res0_fallback"] / n},
        "train": {"samples": info["samples"], "loss_first_epoch": l0, "loss_last_epoch": l1, "epochs": epochs,
                  "seconds": t_train, "params": info["num_params"], "dims": info["dims"]},
        "record_seconds": t_rec, "compared_solves": info["compared_solves"],
        "config": "%d bubbles, icosphere level 3 or 4, seed %d (%d unknowns); %d recorded + %d compared "
                  "Adams-Bashforth steps (after the RK4 start); the learned guess corrects the %s start"
                  % (nb, seed, mesh.n, rec_steps, cmp_steps, "extrapolated" if args.guess else "previous-step"),
    }


def run_learned(args):
    """The learned-guess workload at the size of its configuration (1000 bubbles, 100 recorded
    and 100 compared steps by default)."""
    import torch
    from paper_1905_01341_gb300 import bem, build

    build.build()
    stream = torch.cuda.current_stream(torch.device("cuda", 0))
    r = learned_guess_run(args, bem, stream, args.learn_bubbles, args.learn_steps, args.learn_steps)
    it = r["gmres_iters_per_solve"]
    line = {"metric": "GMRES iterations per solve, learned guess vs its base start and the previous-step q",
            "workload": "learned", "value": it["learned"], "unit": "iterations/solve", "higher_is_better": False,
            "data": "synthetic", **r}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "ours" and args.workload == "batched":
        run_batched(args)
        return
    if args.impl == "ours" and args.workload == "learned":
        run_learned(args)
        return
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
