#!/usr/bin/env python
"""Benchmark of the spherical tree-code velocity evaluation on synthetic spherical inputs.

One step = the whole hot path of one BVE velocity evaluation from particle positions:
the icosahedral tree build (faces, refinement, radix sort), interaction lists, sorted source
copies, the upward pass (SBB moments, proxy weights) and the far + near evaluation, all on
the GPU through the C ABI (``paper_2401_07361_gb300.sts``).  The default workload is the
single-instance precision study: N = 655362 uniform random points on the unit sphere
(seed 0), spherical-Voronoi area weights, zero-mean vorticity = random real spherical-
harmonic series to degree 16 (coefficients N(0, 1) / l, seed 0), theta = 0.7, degree 8,
N_T = 128, mixed precision.  The line also reports the FP64 GPU tree code, the error of the
mixed result against the FP64 oracle tree code, the roofline of the evaluation kernel, and
the FP64 CPU oracle timed on this host's cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BVE velocity targets/s, mixed vs FP64 tree code at ≤1e-6 rel L2; % FP32 peak"
SMS = 152
FP32_LANES = 128
L2_BYTES = 129 * 2**20
FP64_STEPS = 5  # timed steps of the FP64 GPU tree code (about 155 ms each at 655k)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="rand655k_sh16")
    ap.add_argument("--theta", type=float, default=0.7)
    ap.add_argument("--degree", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=None)
    ap.add_argument("--tau-c", type=float, default=0.01,
                    help="near FP64 threshold tau = c * 4 pi / N (half squared chord)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rk4", type=int, default=0,
                    help="time this many RK4 steps of the workload instead of single evaluations "
                         "(Omega = 2 pi per day, dt = 1/288 day) and report the invariants' drift")
    ap.add_argument("--forcing", type=int, default=0,
                    help="with --rk4: the forced system of Sec. 4.4 with this zonal wavenumber (0: none)")
    ap.add_argument("--t0", type=float, default=0.0, help="with --forcing: start time of the run (days)")
    ap.add_argument("--potential", action="store_true",
                    help="time the mixed-precision tree-code stream function (build + potential) instead, "
                         "the FP64 tree code beside")
    ap.add_argument("--dual", action="store_true",
                    help="the tree code by the dual traversal of Sec. 3.4 (PP, PC, CP, CC) instead of the "
                         "target-leaf lists (PC, PP)")
    ap.add_argument("--amr", type=int, default=0,
                    help="time this many RK4 steps of the Gaussian vortex with an AMR pass after each "
                         "(Appendix A; level-5 icosahedral mesh, eps1 0.0025, eps2 0.2, dt 0.01 day)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel from the host instead of replaying the recorded step")
    ap.add_argument("--shard", action="store_true",
                    help="one instance spread over the ranks (strong scaling): every rank builds the tree, "
                         "evaluates a range of target leaves balanced by interaction counts, and the ranks "
                         "all-gather the velocities (NCCL)")
    ap.add_argument("--profile", action="store_true",
                    help="timed device steps only (no e2e, FP64 or CPU legs): the command profiled by ncu")
    return ap.parse_args(argv)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest value of x over the ranks of the job (x itself on one rank): every timed
    quantity is taken from the slowest rank."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_workload(name):
    from paper_2401_07361_gb300 import workloads as W

    return W.workload(name)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        return out


def profile_traffic(kernel_file, workload, dual=False):
    """DRAM bytes per launch of the evaluation kernel from the committed ncu summary of this
    workload and traversal, or None when there is none or it was taken on a different kernel
    source."""
    import hashlib

    name = f"k_eval_mixed_{workload}{'_dual_leaves' if dual else ''}.md"
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    with open(kernel_file, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    src_hash, traffic = None, None
    with open(prof) as f:
        for line in f:
            if line.startswith("source_sha256_16:"):
                src_hash = line.split(":", 1)[1].strip()
            if line.startswith("dram_bytes_per_launch:"):
                traffic = float(line.split(":", 1)[1].strip())
    return traffic if src_hash == h else None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    from oracle import oracle as O

    wl = load_workload(args.workload)
    pos, zeta, area = wl["pos"], wl["zeta"], wl["area"]
    leaf = args.leaf or wl["leaf_size"]
    n = len(pos)
    cores = os.cpu_count() or 1

    offs = wl.get("offsets", np.array([0, n], dtype=np.int64))

    def step():
        for b in range(len(offs) - 1):
            lo, hi = int(offs[b]), int(offs[b + 1])
            tr = O.Tree(pos[lo:hi], leaf, 16)
            tr.velocity(zeta[lo:hi], area[lo:hi], args.theta, args.degree, nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    val = n / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "targets/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "N": n, "theta": args.theta, "degree": args.degree,
                   "leaf_size": leaf, "precision": "fp64", "l2": "inputs on host"},
        "cpu_baseline": {"value": val, "unit": "targets/s", "cores": cores, "kind": "oracle",
                         "sample": f"full workload: oracle tree build + FP64 tree-code velocity of all {n} "
                                   f"targets per step, OpenMP over target leaves"},
        "e2e": {"value": val, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_rk4(args):
    """RK4 time stepping (the Sec. 4 integrator) of the workload, each step recorded once as a
    CUDA graph and replayed: steps/s, particle-stages/s, and the drift of the energy
    E = 1/2 sum |u|^2 A (and its second quadrature 1/2 sum psi zeta A from the FP64 tree-code
    stream function), the enstrophy Z = 1/2 sum zeta^2 A, the circulation sum zeta A and
    the per-particle absolute vorticity zeta + 2 Omega z (carried exactly by the
    unprojected scheme)."""
    import numpy as np
    import torch

    from paper_2401_07361_gb300 import sts

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = load_workload(args.workload)
    n = len(wl["pos"])
    leaf = args.leaf or wl["leaf_size"]
    offsets = wl.get("offsets")
    n_tau = n if offsets is None else int(np.min(np.diff(offsets)[np.diff(offsets) > 0]))
    tau = args.tau_c * 4.0 * math.pi / n_tau
    pm = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16,
                    precision=sts.STS_MIXED, near_fp64_tau=tau)
    Omega, dt = 2.0 * math.pi, 1.0 / 288.0
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    pos = torch.from_numpy(wl["pos"]).to(dev)
    zeta = torch.from_numpy(wl["zeta"]).to(dev)
    area = torch.from_numpy(wl["area"]).to(dev)
    vel = torch.empty((n, 3), dtype=torch.float64, device=dev)
    ctx = sts.Context()
    h = ctx.h
    sts.sts_set_traversal(h, args.dual)

    p64 = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16, precision=sts.STS_FP64)
    psi = torch.empty(n, dtype=torch.float64, device=dev)

    def invariants():
        sts.sts_set_graph(h, False)
        sts.sts_tree_velocity(h, pos, zeta, area, pm, vel, offsets=offsets)
        sts.sts_potential(h, zeta, area, p64, psi)  # on the tree just built (a forest for offsets)
        torch.cuda.synchronize()
        u, z, a, x = vel.cpu().numpy(), zeta.cpu().numpy(), area.cpu().numpy(), pos.cpu().numpy()
        return dict(E=0.5 * float(np.sum(np.sum(u * u, 1) * a)), Epsi=0.5 * float(np.sum(psi.cpu().numpy() * z * a)),
                    Z=0.5 * float(np.sum(z * z * a)), C=float(np.sum(z * a)), q=z + 2 * Omega * x[:, 2],
                    r=np.linalg.norm(x, axis=1))

    forcing = sts.forcing(args.forcing, 0.6 * Omega) if args.forcing > 0 else None
    clock = [args.t0]

    def step():
        if forcing is not None:
            sts.bve_rk4_step_forced(h, pos, zeta, area, clock[0], dt, Omega, forcing, pm)
            clock[0] += dt
        elif offsets is None:
            sts.bve_rk4_step(h, pos, zeta, area, dt, Omega, pm)
        else:
            sts.bve_rk4_step_batched(h, pos, zeta, area, offsets, dt, Omega, pm)

    inv0 = invariants()
    sts.sts_set_graph(h, not args.no_graph)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = sts.sts_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.rk4):
        step()
    e1.record()
    e1.synchronize()
    clocks = sampler.stop()
    launches = sts.sts_launch_count() - l0
    ms = e0.elapsed_time(e1)
    inv1 = invariants()
    nsteps = args.rk4 + max(3, args.warmup)
    line = {
        "metric": "BVE RK4 particle-steps/s (4 tree-code velocity evaluations per step)", "value": n * args.rk4 / (ms / 1e3),
        "unit": "particle-steps/s", "n_gpus": ws, "steps": args.rk4, "warmup": max(3, args.warmup),
        "ms_per_step": ms / args.rk4, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "N": n, "theta": args.theta, "degree": args.degree, "leaf_size": leaf,
                   "dt_day": dt, "Omega_per_day": Omega, "near_fp64_tau": tau,
                   "traversal": "dual (PP, PC, CP, CC)" if args.dual else "target-leaf lists (PC, PP)",
                   "forcing": ({"k": args.forcing, "amplitude": "3/5 Omega", "Tp": 4.0, "Tf": 15.0,
                                "theta1": "pi/3", "t0": args.t0} if forcing is not None else None),
                   "launch": ("host launches (forced steps are not recorded)" if forcing is not None or args.no_graph
                              else "recorded CUDA graph per step")},
        "gpu_launches": int(launches), "clocks": clocks,
        "drift_after_steps": nsteps,
        "drift": {"energy_rel": (inv1["E"] - inv0["E"]) / inv0["E"],
                  "energy_psi_rel": (inv1["Epsi"] - inv0["Epsi"]) / inv0["Epsi"],
                  "enstrophy_rel": (inv1["Z"] - inv0["Z"]) / inv0["Z"],
                  "circulation_abs": inv1["C"] - inv0["C"],
                  "abs_vorticity_max_change": float(np.max(np.abs(inv1["q"] - inv0["q"]))),
                  "max_radius_error": float(np.max(np.abs(inv1["r"] - 1.0)))},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_amr(args):
    """RK4 steps of the Gaussian vortex (Sec. 4.3) with the adaptive mesh refinement of
    Appendix A after every step: per step, the particles are gathered from the mesh, advanced by
    one RK4 step of the tree code (eager: the particle count changes between steps), written
    back, and one AMR pass splits and merges triangles.  Reports particle-steps/s and the AMR
    pass time; the CPU baseline is the oracle's AMR pass on the same mesh (its cost depends on
    the number of possible triangles, not on the state)."""
    import numpy as np
    import torch

    from paper_2401_07361_gb300 import sts
    from paper_2401_07361_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    level, levels, eps1, eps2, dt, Omega = 5, 3, 0.0025, 0.2, 0.01, 2.0 * math.pi
    pos0, faces = W.icosahedral_mesh(level)
    n0 = len(pos0)
    zeta0 = W.gaussian_vortex_vorticity(pos0, W.equal_areas(n0))
    leaf = args.leaf or 64
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    mesh, tree = sts.Context(), sts.Context()
    sts.sts_amr_init(mesh.h, faces, torch.from_numpy(pos0).to(dev), torch.from_numpy(zeta0).to(dev), levels)

    def params(n):
        return sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16,
                          precision=sts.STS_MIXED, near_fp64_tau=args.tau_c * 4.0 * math.pi / n)

    t_rk = [0.0]
    t_amr = [0.0]
    particle_steps = [0]

    def step():
        x, z, a, _ = sts.sts_amr_gather(mesh.h)
        n = x.shape[0]
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        sts.bve_rk4_step(tree.h, x, z, a, dt, Omega, params(n))
        sts.sts_amr_scatter(mesh.h, x, z)
        e1.record()
        counts = sts.sts_amr_step(mesh.h, eps1, eps2)
        e2.record()
        e2.synchronize()
        t_rk[0] += e0.elapsed_time(e1)
        t_amr[0] += e1.elapsed_time(e2)
        particle_steps[0] += n
        return counts

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    t_rk[0] = t_amr[0] = 0.0
    particle_steps[0] = 0
    sampler = ClockSampler(local)
    sampler.start()
    l0 = sts.sts_launch_count()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record()
    last = None
    for _ in range(args.amr):
        last = step()
    c1.record()
    c1.synchronize()
    clocks = sampler.stop()
    launches = sts.sts_launch_count() - l0
    ms = c0.elapsed_time(c1)
    nfinal = sts.sts_amr_info(mesh.h)["particles"]
    line = {
        "metric": "BVE RK4 + AMR particle-steps/s (Gaussian vortex, one AMR pass per step)",
        "value": particle_steps[0] / (ms / 1e3), "unit": "particle-steps/s", "n_gpus": ws, "steps": args.amr,
        "warmup": max(3, args.warmup), "ms_per_step": ms / args.amr, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "gaussian_vortex_ico5_amr", "N_start": n0, "levels": levels, "eps1": eps1,
                   "eps2": eps2, "dt_day": dt, "theta": args.theta, "degree": args.degree, "leaf_size": leaf,
                   "precision": "mixed", "launch": "host launches (the particle count changes every step)"},
        "phases_ms_per_step": {"rk4": t_rk[0] / args.amr, "amr_pass": t_amr[0] / args.amr},
        "particles_end": nfinal, "last_pass": {"splits": last[0], "merges": last[1], "particles": last[2],
                                               "leaf_triangles": last[3]},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O

        # a pass visits every possible triangle on both sides, so its cost hardly depends on
        # the state: the oracle's passes from the initial vortex on the same mesh are timed
        m = O.Amr(faces, n0, levels)
        m.set(pos0, zeta0)
        t0 = time.perf_counter()
        reps = 0
        while reps < 3 or time.perf_counter() - t0 < 2.0:
            m.step(eps1, eps2)
            reps += 1
        cpu_ms = (time.perf_counter() - t0) * 1e3 / reps
        line["cpu_baseline"] = {"value": n0 / (cpu_ms / 1e3), "unit": "vertices/s (AMR pass)", "cores": 1,
                                "kind": "oracle", "sample": f"{reps} oracle AMR passes from the initial vortex "
                                                            f"on the base mesh ({n0} particles, "
                                                            f"{m.nt} possible triangles), single thread"}
        line["amr_pass_gpu_ms"] = t_amr[0] / args.amr
        line["amr_pass_cpu_ms"] = cpu_ms
    if rank == 0:
        print(json.dumps(line), flush=True)
    mesh.close()
    tree.close()
    return 0


def run_potential(args):
    """The stream function psi_i = -(1/4pi) sum_{j != i} log(1 - x_i.x_j) zeta_j A_j by the
    mixed-precision tree code (tree build + potential per step, same lists and proxies as the
    velocity), timed like the velocity bench; roofline against the derived FP32 peak with 12
    flop per interaction (3 FSUB, |d|^2 = 5, 1/2, log2 counted as 1, the weight, the sum; the
    TwoSum compensation is not counted), the FP64 tree code (median of 3 steps) and the oracle
    tree code beside."""
    import numpy as np
    import torch

    from paper_2401_07361_gb300 import sts

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = load_workload(args.workload)
    n = len(wl["pos"])
    leaf = args.leaf or wl["leaf_size"]
    offsets = wl.get("offsets")
    p64 = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16, precision=sts.STS_FP64)
    pm = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16, precision=sts.STS_MIXED,
                    near_fp64_tau=args.tau_c * 4 * math.pi / n)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    pos = torch.from_numpy(wl["pos"]).to(dev)
    zeta = torch.from_numpy(wl["zeta"]).to(dev)
    area = torch.from_numpy(wl["area"]).to(dev)
    psi = torch.empty(n, dtype=torch.float64, device=dev)
    psi64 = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = sts.Context()
    h = ctx.h

    def step(p=pm, out=psi):
        if offsets is None:
            sts.sts_tree_build(h, pos, p)
        else:
            sts.sts_tree_build_batched(h, pos, offsets, p)
        sts.sts_potential(h, zeta, area, p, out)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stats = sts.sts_stats(h)
    sampler = ClockSampler(local)
    sampler.start()
    sts.sts_set_timing(h, True)
    l0 = sts.sts_launch_count()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    launches = sts.sts_launch_count() - l0
    phases = sts.sts_phase_times(h)
    sts.sts_set_timing(h, False)
    total_ms = max_over_ranks(sum(times), ws, dev)
    ms = total_ms / max(1, args.steps)
    eval_ms = phases["eval"][0] / max(1, phases["eval"][1])
    inter = stats["pc"] + stats["pp"]
    peaks = measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0)) if isinstance(peaks, dict) else 2070.0
    peak_fp32 = 152 * 128 * 2 * mhz * 1e6 / 1e12  # TFLOP/s
    achieved = 12.0 * inter / (eval_ms / 1e3) / 1e12
    # the FP64 tree code on the same workload: median of 3 timed steps after one warm-up
    step(p64, psi64)
    t64 = []
    for _ in range(3):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(p64, psi64)
        e1.record()
        e1.synchronize()
        t64.append(e0.elapsed_time(e1))
    ms64 = float(np.median(t64))
    step()  # psi back from the mixed path (the tree is rebuilt identically)
    torch.cuda.synchronize()
    got, got64 = psi.cpu().numpy(), psi64.cpu().numpy()
    a = wl["area"]
    line = {
        "metric": "stream function targets/s, mixed tree code (FP64 tree code beside)", "value": ws * n / (ms / 1e3),
        "unit": "targets/s", "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "N": n, "theta": args.theta, "degree": args.degree, "leaf_size": leaf,
                   "precision": "mixed (f32 log2 terms, compensated sums, f64 close pairs below tau)",
                   "near_fp64_tau": pm.near_fp64_tau, "l2": "flushed between timed steps (256 MiB write)",
                   "launch": "host launches (build + potential)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                     "frac": achieved / peak_fp32, "traffic": None, "kernel": "k_eval_mixed<true>",
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x sm_max_mhz; 12 flop per interaction",
                     "kernel_ms": eval_ms},
        "gpu_launches": int(launches), "clocks": clocks,
        "phases_ms_per_step": {k: v[0] / max(1, v[1]) for k, v in phases.items() if v[1]},
        "interactions_per_step": stats,
        "fp64_tree": {"value": n / (ms64 / 1e3), "unit": "targets/s", "ms": ms64, "ms_samples": t64},
        "error": {"mixed_vs_fp64_gpu_tree_rel_l2": float(np.sqrt(np.sum((got - got64) ** 2 * a) / np.sum(got64**2 * a)))},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and n <= 3_000_000:
        from oracle import oracle as O

        t0 = time.perf_counter()
        if offsets is None:
            ref = O.Tree(wl["pos"], leaf).potential(wl["zeta"], wl["area"], args.theta, args.degree)
        else:
            ref = np.concatenate([O.Tree(wl["pos"][a:b], leaf).potential(wl["zeta"][a:b], wl["area"][a:b], args.theta,
                                                                         args.degree)
                                  for a, b in zip(offsets[:-1], offsets[1:]) if b > a])
        cpu_s = time.perf_counter() - t0
        line["error"]["vs_fp64_oracle_tree_rel_l2"] = float(np.sqrt(np.sum((got - ref) ** 2 * a) / np.sum(ref**2 * a)))
        line["error"]["fp64_gpu_vs_fp64_oracle_tree_rel_l2"] = float(
            np.sqrt(np.sum((got64 - ref) ** 2 * a) / np.sum(ref**2 * a)))
        line["cpu_baseline"] = {"value": n / cpu_s, "unit": "targets/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"full workload: oracle tree build + FP64 tree-code stream function of all "
                                          f"{n} targets, OpenMP over target leaves"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_shard(args):
    """One tree-code velocity of the workload spread over the job's ranks: a step is the tree
    build (every rank), the rank's leaf range and the all-gather of the velocities, so the
    work per step is fixed as ranks are added (strong scaling)."""
    import numpy as np
    import torch

    from paper_2401_07361_gb300 import shard, sts

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = load_workload(args.workload)
    if "offsets" in wl:
        raise SystemExit("--shard takes a single-instance workload")
    n = len(wl["pos"])
    leaf = args.leaf or wl["leaf_size"]
    p = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16, precision=sts.STS_MIXED,
                   near_fp64_tau=args.tau_c * 4.0 * math.pi / n)
    pos, zeta, area = (torch.from_numpy(wl[k]).to(dev) for k in ("pos", "zeta", "area"))
    vel = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = sts.Context()

    def step():
        sts.sts_tree_build(ctx.h, pos, p)
        shard.sharded_velocity(ctx.h, zeta, area, p, rank, ws, vel=vel)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    l0 = sts.sts_launch_count()
    barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = sts.sts_launch_count() - l0
    total_ms = max_over_ranks(sum(times), ws, dev)
    got = vel.cpu().numpy()
    full = sts.sts_velocity(ctx.h, zeta, area, p).cpu().numpy()
    a = wl["area"]
    err = float(np.sqrt(np.sum(np.sum((got - full) ** 2, 1) * a) / np.sum(np.sum(full**2, 1) * a)))
    parts = shard.partition(sts.sts_leaf_work(ctx.h, args.degree), ws)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * args.steps / (total_ms / 1e3), "unit": "targets/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / max(1, args.steps),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N": n, "theta": args.theta, "degree": args.degree,
                       "leaf_size": leaf, "precision": "mixed", "parallelism": f"leaf-range shards x{ws}",
                       "launch": "host launches", "l2": "flushed between timed steps (256 MiB write)"},
            "gpu_launches": int(launches), "clocks": clocks,
            "shards": [{"leaves": [lo, hi]} for lo, hi in parts],
            "error": {"sharded_vs_one_gpu_rel_l2": err},
        }), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.shard:
        return run_shard(args)
    if args.amr > 0:
        return run_amr(args)
    if args.rk4 > 0:
        return run_rk4(args)
    if args.potential:
        return run_potential(args)
    import numpy as np
    import torch

    from paper_2401_07361_gb300 import sts

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = load_workload(args.workload)
    pos_h, zeta_h, area_h = wl["pos"], wl["zeta"], wl["area"]
    n = len(pos_h)
    leaf = args.leaf or wl["leaf_size"]
    # one tau for the whole forest: that of the smallest instance (widest particle spacing)
    n_tau = n if "offsets" not in wl else int(np.min(np.diff(wl["offsets"])[np.diff(wl["offsets"]) > 0]))
    tau = args.tau_c * 4.0 * math.pi / n_tau
    pm = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16,
                    precision=sts.STS_MIXED, near_fp64_tau=tau)
    p64 = sts.params(theta=args.theta, degree=args.degree, leaf_size=leaf, max_level=16, precision=sts.STS_FP64)
    pos = torch.from_numpy(pos_h).to(dev)
    zeta = torch.from_numpy(zeta_h).to(dev)
    area = torch.from_numpy(area_h).to(dev)
    vel = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ctx = sts.Context()
    h = ctx.h
    # the step is recorded once as a CUDA graph and replayed (recording needs its own stream)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sts.sts_set_graph(h, not args.no_graph)
    sts.sts_set_traversal(h, args.dual)
    sts.sts_set_timing(h, True)

    offsets = wl.get("offsets")

    def step(p=pm):
        sts.sts_tree_velocity(h, pos, zeta, area, p, vel, offsets=offsets)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stats = sts.sts_dual_stats(h, args.degree) if args.dual else sts.sts_stats(h)
    info = sts.sts_tree_info(h)

    # ---- device-resident timed steps ------------------------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    sts.sts_set_timing(h, True)  # resets the totals; events recorded in the graph stay
    l0 = sts.sts_launch_count()
    barrier()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    launches = sts.sts_launch_count() - l0
    phases = sts.sts_phase_times(h)
    sts.sts_set_timing(h, False)
    total_ms = max_over_ranks(sum(times), ws, dev)
    ms_step = total_ms / max(1, args.steps)
    value = ws * n * args.steps / (total_ms / 1e3)
    v_mixed = vel.cpu().numpy().copy()
    if args.profile:
        clocks = sampler.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "targets/s", "ms_per_step": ms_step,
                              "profile": True, "gpu_launches": int(launches), "clocks": clocks,
                              "phases_ms_per_step": {k: v[0] / max(1, v[1]) for k, v in phases.items() if v[1]},
                              "interactions_per_step": stats, "tree": info}), flush=True)
        ctx.close()
        return 0

    # ---- end to end through host buffers ----------------------------------------------
    pos_p = torch.from_numpy(pos_h).pin_memory()
    zeta_p = torch.from_numpy(zeta_h).pin_memory()
    area_p = torch.from_numpy(area_h).pin_memory()
    vel_p = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pos2 = torch.empty_like(pos)
    zeta2 = torch.empty_like(zeta)
    area2 = torch.empty_like(area)
    vel2 = torch.empty_like(vel)
    e2e_times = []
    e2e_steps = max(3, min(args.steps, 10))
    barrier()
    for it in range(e2e_steps + 1):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pos2.copy_(pos_p, non_blocking=True)
        zeta2.copy_(zeta_p, non_blocking=True)
        area2.copy_(area_p, non_blocking=True)
        sts.sts_tree_velocity(h, pos2, zeta2, area2, pm, vel2, offsets=offsets)
        vel_p.copy_(vel2, non_blocking=True)
        e1.record()
        e1.synchronize()
        if it > 0:
            e2e_times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    e2e_ms = max_over_ranks(sum(e2e_times) / len(e2e_times), ws, dev)
    assert np.array_equal(vel_p.numpy(), v_mixed), "end-to-end result differs from the device-resident one"

    # ---- FP64 GPU tree code (same tree), error of the mixed result ------------------
    # timed like the mixed step (warm-up, L2 flushed, CUDA events per step); the median of
    # FP64_STEPS steps is reported, with every sample
    step(p64)
    torch.cuda.synchronize()
    fp64_times = []
    for _ in range(FP64_STEPS):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step(p64)
        e1.record()
        e1.synchronize()
        fp64_times.append(e0.elapsed_time(e1))
    fp64_ms = float(np.median(fp64_times))
    v64 = vel.cpu().numpy()

    def rel_l2(a, b, w):
        num = np.sum(np.sum((a - b) ** 2, axis=1) * w)
        den = np.sum(np.sum(b ** 2, axis=1) * w)
        return float(math.sqrt(num / den))

    def rel_max(a, b):
        return float(np.max(np.linalg.norm(a - b, axis=1)) / np.max(np.linalg.norm(b, axis=1)))

    err_vs_gpu64 = rel_l2(v_mixed, v64, area_h)

    # ---- roofline of the evaluation kernel ----------------------------------------------
    # (the launch over the leaf lists: PC + PP, which the dual traversal's PP and PC pairs fill)
    eval_ms, eval_cnt = phases["eval"]
    eval_avg_ms = eval_ms / max(1, eval_cnt)
    inter = stats["pc"] + stats["pp"]
    flops = 16.0 * inter
    sm_max = measured_peaks().get("sm_max_mhz", 2070.0)
    peak_tflops = SMS * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (eval_avg_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": profile_traffic(os.path.join(ROOT, "paper_2401_07361_gb300", "csrc", "sts_eval.cu"),
                                           args.workload, args.dual),
                "kernel": "k_eval_mixed (leaf lists)" if args.dual else "k_eval_mixed", "flops_per_launch": flops,
                "peak_source": f"derived: {SMS} SMs x {FP32_LANES} FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                               f"(MEASURED_PEAKS sm_max_mhz); 16 flop per interaction",
                "kernel_ms": eval_avg_ms}

    # ---- CPU oracle baseline (rank 0 only) -----------------------------------------------
    cpu = None
    err_vs_oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O

        cores = os.cpu_count() or 1
        offs = offsets if offsets is not None else np.array([0, n], dtype=np.int64)
        t0 = time.perf_counter()
        ref = np.zeros((n, 3))
        for b in range(len(offs) - 1):
            lo, hi = int(offs[b]), int(offs[b + 1])
            tr = O.Tree(pos_h[lo:hi], leaf, 16)
            vfun = tr.velocity_dual if args.dual else tr.velocity
            ref[lo:hi] = vfun(zeta_h[lo:hi], area_h[lo:hi], args.theta, args.degree, nthreads=cores)
        dt = time.perf_counter() - t0
        how = ("dual traversal (PP, PC, CP, CC), OpenMP over target clusters and leaves" if args.dual
               else "OpenMP over target leaves")
        cpu = {"value": n / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
               "sample": f"one full evaluation: oracle tree build + FP64 tree-code velocity of all {n} targets "
                         f"(theta {args.theta}, degree {args.degree}, N_T {leaf}), {how}"}
        err_vs_oracle = {"rel_l2": rel_l2(v_mixed, ref, area_h), "rel_max": rel_max(v_mixed, ref),
                         "fp64_gpu_rel_l2": rel_l2(v64, ref, area_h)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "N": n, "theta": args.theta, "degree": args.degree,
                       "leaf_size": leaf, "max_level": 16, "precision": "mixed (f32 pairs, f64 positions/"
                       "contraction/near pairs below tau)", "near_fp64_tau": tau,
                       "traversal": "dual (PP, PC, CP, CC)" if args.dual else "target-leaf lists (PC, PP)",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                       "launch": "host launches" if args.no_graph else "recorded CUDA graph, replayed per step"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": ws * n / (e2e_ms / 1e3), "unit": "targets/s",
                    "h2d_bytes_per_step": int(pos_h.nbytes + zeta_h.nbytes + area_h.nbytes),
                    "d2h_bytes_per_step": int(n * 3 * 8)},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "error": {"mixed_vs_fp64_gpu_tree_rel_l2": err_vs_gpu64, "vs_fp64_oracle_tree": err_vs_oracle},
            "fp64_tree": {"value": n / (fp64_ms / 1e3), "unit": "targets/s", "ms": fp64_ms,
                          "ms_samples": fp64_times, "stat": f"median of {FP64_STEPS} timed steps after 1 warm-up"},
            "phases_ms_per_step": {k: v[0] / max(1, v[1]) for k, v in phases.items() if v[1]},
            "interactions_per_step": stats,
            "tree": info,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
