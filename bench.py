#!/usr/bin/env python3
"""Soft-step benchmark of the P3T integrator with individual cut-off radii.

One "step" is one full soft step of the paper's procedure (steps 3-9): kick,
hard part (Hermite clusters with perfect-accretion collisions + Kepler
drift), tree build, soft force walk, neighbour lists + clusters, kick, and
when bodies collided the merge with new cut-off radii, force and neighbours
-- all in libp3t's kernels.  Workload: the N = 10^6 wide disk on 1-10 au
(power-law planetesimals on [1e-12, 1e-8] plus 20 protoplanets of 1e-7; e/i
rms 2h and h; density 2 g/cm^3, radius factor f = 1), theta = 0.5, leaf 16,
target groups of up to 64, dt = 1/64, mixed precision.  Synthetic, seeded
(seed 1003).

Reported value: pair interactions (p-p + p-node terms of the soft force) per
second of whole-step wall time.  Also reported: the soft-step time, Hermite
particle-steps per second, per-phase times, a roofline entry for the tree walk
(FP32-bound, algorithmic FLOPs), an end-to-end number through the C ABI with
host buffers, and the CPU oracle timed on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): independent replicas, one per rank (the soft step of one
disk does not shard across GPUs here); value = sum over ranks / max time.
"""
from __future__ import annotations

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

METRIC = "soft-step wall time & pair-interactions/s at N=1e6; hard-part Hermite steps/s"
UNIT = "pair-interactions/s"
# algorithmic work per unit (counted from the method): changeover pair term
# ~30 flops + rsqrt, monopole + quadrupole node term ~70 flops + rsqrt
FLOP_PP, FLOP_PN = 30.0, 70.0
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 (FMA)
# x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 peak likewise: 152 SMs x 2 FP64 FMA lanes x 2 x 2.07 GHz (a dependent-
# free DFMA stream was measured at 1.25 TFLOP/s on this part)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) of one k_walk launch on the N = 10^6 wide disk,
# group size 64, from a single-pass ncu capture of this kernel
# (dram__bytes_read.sum 78.90 MB + dram__bytes_write.sum 16.13 MB)
WALK_TRAFFIC_1E6 = 95.03e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--group-size", type=int, default=64,
                    help="target group size of the tree walk (0: one group per leaf)")
    ap.add_argument("--f-radius", type=float, default=1.0,
                    help="collision radius factor f (0: no collisions)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=8,
                    help="most whole oracle soft steps timed for the CPU baseline "
                         "(stops after ~20 s of stepping)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time one gradient of the 32-step soft KDK rollout at N=1e4")
    ap.add_argument("--adjoint-n", type=int, default=10_000)
    ap.add_argument("--adjoint-form", default="direct", choices=["direct", "p3t"],
                    help="direct: all-pairs soft force (FP32 pairs) and Kepler drift of every "
                         "particle; p3t: tree soft force and the paper's hard part (Hermite "
                         "clusters, Kepler singles), FP64")
    ap.add_argument("--ensemble", action="store_true",
                    help="the ensemble of 256 independent disks: batched in one context "
                         "(one launch sequence per step) vs per-disk contexts in one CUDA "
                         "graph vs per-disk contexts one after another")
    ap.add_argument("--precision-study", action="store_true",
                    help="FP64 vs mixed path over 64 soft steps of the N=1e5 ring, with the "
                         "per-particle force error against the oracle (max, p99)")
    ap.add_argument("--cutoff-sweep", action="store_true",
                    help="compare the cut-off schemes (shared / individual / individual with "
                         "random velocity) over R~cut,0 on the mass-spectrum ring; one JSON "
                         "line per configuration")
    return ap.parse_args()


def workload(n, seed=1003):
    from paper_2007_15432_gb300 import disks
    return disks.wide_power_law(n=n, seed=seed)


def workload_name(n):
    return (f"wide power-law disk N={n} (1-10 au, m in [1e-12,1e-8] dN/dm~m^-2.5 + 20 "
            "protoplanets 1e-7, e/i rms 2h/h), theta=0.5, leaf 16, dt=1/64")


# ---------------------------------------------------------------- clocks -----
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return dict(sm_mhz=float(np.median(sm)) if sm else None,
                    sm_max_mhz=float(max(smax)) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ------------------------------------------------------------ distributed ----
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return rank, local, world, dist
    return rank, local, world, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def allmax(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------- CPU oracle ----
def oracle_steps(s, k_steps, warmup=0, group_size=64, f_radius=1.0, budget_s=None):
    """The CPU oracle stepping the same workload: after the initial force
    (untimed), whole soft steps (kick, Hermite clusters + Kepler drift with
    collisions, cut-offs held, tree build, tree walk, neighbour filter,
    clusters, kick, and the merge with new radii, tree, walk and neighbours
    when bodies collided); `warmup` steps untimed, then up to k_steps timed
    ones, stopping early once budget_s seconds of timed stepping have passed
    (at least one step).  Returns (pair interactions, seconds, timed steps,
    info)."""
    from oracle import oracle as O
    from paper_2007_15432_gb300 import disks
    s = disks.copy_state(s)
    rp = disks.physical_radius(s["m"])
    p = O.Params(theta=0.5, eta=0.01, eta0=0.001, group_size=group_size, f_radius=f_radius)
    ro, rs, _, _ = O.cutoffs(s, p)
    acc, cl, _ = O.initial_force(s, ro, rs, p)
    inter, secs, done = 0, 0.0, 0
    for k in range(warmup + k_steps):
        t0 = time.perf_counter()
        acc, cl, info = O.soft_step(s, ro, rs, p, acc, cl, r_phys=rp)
        dt = time.perf_counter() - t0
        if info["merged"]:
            rp, ro, rs = info["r_phys"], info["r_out"], info["r_search"]
        if k < warmup:
            continue
        secs += dt
        inter += info["n_pp"] + info["n_pnode"]
        done += 1
        if budget_s is not None and secs >= budget_s:
            break
    return inter, secs, done, dict(threads=O.num_threads())


def _oracle_sample_text(n, done):
    return (f"{done} whole oracle soft steps of the N={n} workload (kick, Hermite clusters "
            "and Kepler drift with collisions, tree build, tree walk, neighbour filter, "
            "clusters, kick, merges with new radii/force/neighbours), each timed; "
            "initial force untimed")


def run_reference(args):
    rank, local, world, dist = dist_setup(args)
    if rank != 0:
        return 0
    s = workload(args.n)
    from oracle import oracle as O
    O.build()
    t_wall = time.perf_counter()
    # warm-up steps are stepped but not timed; then args.steps timed steps
    inter_t, secs_t, done_t, info = oracle_steps(s, args.steps, warmup=args.warmup,
                                                 group_size=args.group_size,
                                                 f_radius=args.f_radius)
    value = inter_t / secs_t
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=done_t,
                warmup=args.warmup, ms_per_step=1e3 * secs_t / done_t, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=workload_name(args.n), n=args.n, group_size=args.group_size,
                            precision="fp64 (CPU oracle)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=info["threads"], kind="oracle",
                                  sample=_oracle_sample_text(args.n, done_t)),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                wall_s=time.perf_counter() - t_wall)
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours -----
def run_ours(args):
    rank, local, world, dist = dist_setup(args)
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2007_15432_gb300 import build
    build.build()
    from paper_2007_15432_gb300 import p3t as P

    s = workload(args.n, seed=1003 + 1000 * rank)
    n = len(s["m"])
    prec = P.P3T_MIXED if args.precision == "mixed" else P.P3T_FP64
    prm = P.Params(theta=0.5, precision=prec, eta=0.01, eta0=0.001, group_size=args.group_size,
                   f_radius=args.f_radius)
    from paper_2007_15432_gb300 import disks
    # one (10, n) device tensor holds the state (the end-to-end leg moves it
    # in one copy each way)
    st, stbuf = P.State.from_numpy_packed(s, device=dev, r_phys=disks.physical_radius(s["m"]))
    ss = P.SoftStep(prm, st, device=local)
    stream = torch.cuda.current_stream(dev)
    ss.init(update_cutoffs=True)            # cut-off radii at init, then after merges
    torch.cuda.synchronize(dev)
    ss.status()

    K, W = args.steps, args.warmup
    counts_all = torch.zeros(K, 2, 2, dtype=torch.int64, device=dev)
    hsteps_all = torch.zeros(K, dtype=torch.int64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(K)]
    h = 0.5 * prm.dt_soft
    scratch_counts = torch.zeros(2, 2, dtype=torch.int64, device=dev)
    e_disp = [0.0, 0.0]
    merged = [0]

    def step(k=None, counts=None, out=None):
        e = ev[k] if k is not None else None
        cnt = counts if counts is not None else (counts_all[k] if k is not None else scratch_counts)
        if e: e[0].record(stream)
        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)
        P.p3t_hard_step(ss.ctx, st, ss.cl, prm.dt_soft,
                        hsteps_all[k:k + 1] if k is not None else ss.hsteps, stream)
        if out is not None:
            out.after_hard(st, stream)   # rows the rest of the step leaves alone
        if e: e[1].record(stream)
        # composites formed by this hard step: the merge after the second
        # kick rebuilds the neighbour lists, so the force before it builds
        # none.  The count is copied after the hard step and read while the
        # tree and the force run.
        if ss.collisions:
            P.p3t_collisions_pending_async(ss.ctx, stream)
        P.p3t_build_tree(ss.ctx, st, False, stream)
        if e: e[2].record(stream)
        P.p3t_soft_force(ss.ctx, st, ss.acc, cnt[0], stream)
        if e: e[3].record(stream)
        pending = ss.collisions and P.p3t_collisions_pending_wait(ss.ctx) > 0
        if not pending:
            ss.cl = P.p3t_neighbours(ss.ctx, st, ss.nb_off, ss.nb_idx, stream)
        if e: e[4].record(stream)
        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)
        if e: e[5].record(stream)
        if pending:
            # procedure step 9: merge (synchronises), then new radii and force
            if out is not None:
                out.fence(stream)
            nm, eh, es = P.p3t_merge(ss.ctx, st, None, stream)
            e_disp[0] += eh
            e_disp[1] += es
            if nm:
                merged[0] += nm
                ss.n = len(st.m)
                ss.acc = ss.acc[:, :ss.n]
                P.p3t_cutoffs(ss.ctx, st, stream)
                P.p3t_build_tree(ss.ctx, st, False, stream)
                P.p3t_soft_force(ss.ctx, st, ss.acc, cnt[1], stream)
                ss.cl = P.p3t_neighbours(ss.ctx, st, ss.nb_off, ss.nb_idx, stream)
            else:
                raise RuntimeError("composites pending but nothing merged")
        if out is not None:
            out.finish(st, stream, pending)
        if e: e[6].record(stream)

    for _ in range(W):
        step()
    torch.cuda.synchronize(dev)
    ss.status()
    n_start = len(st.m)
    m_start = float(st.m.sum().item())

    energy = torch.zeros(2, 4, dtype=torch.float64, device=dev)
    P.p3t_energy(ss.ctx, st, energy[0], stream)   # energy, outside the timed region
    e_disp[0] = e_disp[1] = 0.0
    merged[0] = 0
    counts_all.zero_()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(dist)
    torch.cuda.synchronize(dev)
    launches0 = P.p3t_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(K):
        step(k)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    launches = P.p3t_launch_count() - launches0
    barrier(dist)
    P.p3t_energy(ss.ctx, st, energy[1], stream)
    clk = clocks.stop()
    ss.status()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    phase = np.zeros(6)
    for k in range(K):
        e = ev[k]
        phase += [e[q].elapsed_time(e[q + 1]) for q in range(6)]
    phase /= K
    c = counts_all.cpu().numpy()               # [step, first / after-merge force, pp / pnode]
    inter = float(c.sum())
    hsteps = float(hsteps_all.sum().item())
    walk_s = phase[2] / 1e3
    E0, E1 = (float(v) for v in energy[:, 0].cpu())
    flops_per_launch = (FLOP_PP * c[:, 0, 0] + FLOP_PN * c[:, 0, 1]).mean()

    # ---- end to end through the C ABI with host buffers --------------------
    # the state's (10, n) block: x, y, z, vx, vy, vz, m, r_out, r_search,
    # r_phys (rows shortened by merges keep their storage; the block moves in
    # whole).  The result comes back row by row (StateCopyOut): the rows the
    # second kick leaves alone cross the link while the tree and the force
    # run, the velocities after the kick (every row again after a merge).
    host = stbuf.cpu().pin_memory()
    host_out = torch.empty_like(host).pin_memory()
    out = P.StateCopyOut(host_out)
    E = max(1, args.e2e_steps)
    e2e_counts = torch.zeros(E, 2, 2, dtype=torch.int64, device=dev)
    h2d = 0
    torch.cuda.synchronize(dev)
    barrier(dist)
    t0 = time.perf_counter()
    for k in range(E):
        stbuf.copy_(host, non_blocking=True)
        h2d += host.numel() * host.element_size()
        out.host = host_out
        step(None, counts=e2e_counts[k], out=out)
        torch.cuda.synchronize(dev)
        host, host_out = host_out, host   # the result is the next step's input
    t_e2e = time.perf_counter() - t0
    e2e_inter = float(e2e_counts.sum().item())
    h2d //= E
    d2h = out.d2h_bytes // E
    ss.status()

    tot_elapsed = allmax(dist, elapsed)
    tot_inter = allsum(dist, inter)
    tot_e2e_t = allmax(dist, t_e2e)
    tot_e2e_inter = allsum(dist, e2e_inter)
    if rank != 0:
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        i_cpu, t_cpu, done, info = oracle_steps(workload(args.n), args.cpu_steps,
                                                group_size=args.group_size,
                                                f_radius=args.f_radius, budget_s=20.0)
        cpu = dict(value=i_cpu / t_cpu, unit=UNIT, cores=info["threads"], kind="oracle",
                   sample=_oracle_sample_text(args.n, done) + f"; {t_cpu / done:.2f} s per step")
    achieved = flops_per_launch / walk_s / 1e12
    peak = FP32_PEAK_TFLOPS if prec == P.P3T_MIXED else FP64_PEAK_TFLOPS
    line = dict(
        metric=METRIC, value=tot_inter / tot_elapsed, unit=UNIT, n_gpus=world, steps=K,
        warmup=W, ms_per_step=1e3 * tot_elapsed / K, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f32/f64" if prec == P.P3T_MIXED else "f64",
        data="synthetic (seeded disk)",
        config=dict(workload=workload_name(args.n), n=args.n, group_size=args.group_size,
                    f_radius=args.f_radius, density_g_cm3=2.0,
                    precision=args.precision, l2="per-step working set > L2 (inputs ~0.5 GB)",
                    parallelism="replicas only" if world > 1 else "single GPU"),
        soft_step_ms=1e3 * elapsed / K,
        hermite_steps_per_s=hsteps / (phase[0] * K / 1e3),   # over the kick + hard phase
        hermite_steps_per_step=hsteps / K,
        energy_error=abs((E1 + e_disp[0] + e_disp[1]) / E0 - 1.0),
        energy_dissipated=e_disp[0] + e_disp[1],
        collisions=dict(merged=merged[0], n_start=n_start, n_end=len(st.m),
                        mass_error=abs(float(st.m.sum().item()) / m_start - 1.0)),
        interactions_per_step=inter / K,
        phases_ms=dict(kick_and_hard=phase[0], tree=phase[1], soft_force=phase[2],
                       neighbours_clusters=phase[3], kick=phase[4],
                       merge_and_recompute=phase[5]),
        roofline=dict(kernel=("k_walk (mixed) + float-float refinement" if prec == P.P3T_MIXED
                              else "k_walk (fp64)"),
                      bound="alu", pipe="fp32" if prec == P.P3T_MIXED else "fp64",
                      achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                      traffic=WALK_TRAFFIC_1E6 if (args.n == 1_000_000 and args.group_size == 64
                                                   and prec == P.P3T_MIXED) else None,
                      traffic_kernel="k_walk"),
        e2e=dict(value=tot_e2e_inter / tot_e2e_t, unit=UNIT, h2d_bytes_per_step=h2d,
                 d2h_bytes_per_step=d2h),
        gpu_launches=int(launches),
        clocks=clk,
        cpu_baseline=cpu,
    )
    print(json.dumps(line), flush=True)
    ss.close()
    return 0


# ------------------------------------------------------- cut-off schemes -----
def run_cutoff_sweep(args):
    """Shared vs individual vs individual + random-velocity cut-off (Sec.
    2.1.1-2.1.3, Eqs. rout1, routi, routi2): mean neighbour count, largest
    neighbour cluster and soft-step time (with its phases and interaction
    count) against R~cut,0, on seeded stand-ins for the paper's mass-spectrum
    snapshot (N = 377,740 on 0.9-1.1 au, power-law masses on [1e-12,
    4.25e-9]): "cold" (e/i rms 2h/h per particle) and "warm" (e/i rms
    1e-3 / 5e-4, where the random-velocity term sets most radii).  Perfect
    accretion as in the paper's runs (f = 1, 2 g/cm^3).  Steps are timed only
    while the largest cluster has at most 600 members: a cluster's block step
    costs its size squared on one block."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    from paper_2007_15432_gb300 import build, disks
    build.build()
    from paper_2007_15432_gb300 import p3t as P
    n = 377_740
    rings = {"cold": disks.mass_spectrum_ring(n), "warm": disks.mass_spectrum_ring(n, e_rms=1e-3,
                                                                                 i_rms=5e-4)}
    names = {P.P3T_CUT_SHARED: "shared", P.P3T_CUT_HILL: "individual",
             P.P3T_CUT_HILL_VRAN: "individual+random-velocity"}
    # untimed warm-up through every stage, merges included, so that the
    # first timed configuration does not pay for first launches
    w0 = disks.planted_impacts(disks.mass_spectrum_ring(20_000, seed=7),
                               [(10, 11), (20, 21), (30, 31)])
    for mode in (P.P3T_CUT_SHARED, P.P3T_CUT_HILL):
        prm = P.Params(theta=0.5, precision=P.P3T_MIXED, eta=0.01, eta0=0.001, group_size=64,
                       cutoff_mode=mode, f_radius=1.0)
        st = P.State.from_numpy(w0, device=dev, r_phys=disks.physical_radius(w0["m"]))
        ss = P.SoftStep(prm, st, device=0, nb_cap=64 * len(w0["m"]))
        ss.init(update_cutoffs=True)
        for _ in range(3):
            ss.step()
        ss.status()
        ss.close()
    torch.cuda.synchronize(dev)
    for ring, s0 in rings.items():
        for mode in (P.P3T_CUT_SHARED, P.P3T_CUT_HILL, P.P3T_CUT_HILL_VRAN):
            for rc in (0.5, 1.0, 2.0, 3.0):
                prm = P.Params(theta=0.5, precision=P.P3T_MIXED, eta=0.01, eta0=0.001,
                               group_size=64, rcut0=rc, cutoff_mode=mode, f_radius=1.0)
                st = P.State.from_numpy(s0, device=dev, r_phys=disks.physical_radius(s0["m"]))
                ss = P.SoftStep(prm, st, device=0, nb_cap=64 * n)
                ok = False
                for _ in range(3):   # grow the candidate buffer when it overflowed
                    ss.init(update_cutoffs=True)
                    code, _ = P.p3t_status(ss.ctx)
                    if code == 0:
                        ok = True
                        break
                line = dict(study="cutoff schemes", ring=ring, scheme=names[mode], rcut0=rc, n=n)
                if not ok:
                    line["error"] = P.p3t_strerror(code)
                    print(json.dumps(line), flush=True)
                    ss.close()
                    continue
                cl = P.clusters_to_host(ss.ctx, ss.cl, n)
                line.update(mean_neighbours=int(ss.nb_off[n].item()) / n,
                            largest_cluster=int(cl["max_size"]), clusters=int(len(cl["cl_off"]) - 1),
                            mean_r_out=float(st.r_out.mean().item()))
                if cl["max_size"] <= 600:
                    K, h = 4, 0.5 * prm.dt_soft
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                    ph = np.zeros(5)
                    merged = 0
                    counts = torch.zeros(2, dtype=torch.int64, device=dev)
                    inter = 0
                    for k in range(K + 2):
                        timed = k >= 2
                        ev[0].record(stream)
                        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)
                        P.p3t_hard_step(ss.ctx, st, ss.cl, prm.dt_soft, ss.hsteps, stream)
                        ev[1].record(stream)
                        P.p3t_build_tree(ss.ctx, st, False, stream)
                        ev[2].record(stream)
                        P.p3t_soft_force(ss.ctx, st, ss.acc, counts, stream)
                        ev[3].record(stream)
                        ss.cl = P.p3t_neighbours(ss.ctx, st, ss.nb_off, ss.nb_idx, stream)
                        P.p3t_kick(ss.ctx, st, ss.acc, h, stream)
                        ev[4].record(stream)
                        nm = ss.merge(stream)      # procedure step 9 (synchronises)
                        ev[5].record(stream)
                        torch.cuda.synchronize(dev)
                        # read after the last event: the first reduction in a
                        # process loads its module, which no phase should pay
                        if timed:
                            inter += int(counts.sum().item())
                            ph += [ev[q].elapsed_time(ev[q + 1]) for q in range(5)]
                            merged += nm
                    ss.status()
                    ph /= K
                    line.update(ms_per_step=float(ph.sum()), interactions_per_step=inter / K,
                                merged=merged,
                                phases_ms=dict(kick_and_hard=ph[0], tree=ph[1], soft_force=ph[2],
                                               neighbours_and_kick=ph[3], merge_and_recompute=ph[4]))
                else:
                    line["ms_per_step"] = None
                    line["note"] = "steps not timed: largest cluster above 600 members"
                print(json.dumps(line), flush=True)
                ss.close()
    return 0


# -------------------------------------------------------- FP64 vs mixed ------
def run_precision_study(args):
    """The N = 1e5 equal-mass ring (0.9-1.1 au, m = 1e-11, e/i rms
    0.01/0.005, seed 1002), theta = 0.5, monopole + quadrupole, leaf 16,
    target groups of up to 64, dt = 1/64: 64 soft steps in the plain FP64
    path and in the mixed path, each from the same initial state.  Reported
    per path: time per soft step and pair interactions per second, and the
    per-particle relative error of the soft force against the FP64 oracle
    (same tree rules) on the initial state and on the state after the 64
    steps: max, p99, median and max(|a - a_ref|) / rms|a_ref|."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    from paper_2007_15432_gb300 import build, disks
    build.build()
    from paper_2007_15432_gb300 import p3t as P
    from oracle import oracle as O
    n, K = args.n if args.n != 1_000_000 else 100_000, 64
    s0 = disks.equal_mass_ring(n=n, seed=1002)

    def force_err(st, ctx, op):
        acc = torch.zeros(3, len(st.m), dtype=torch.float64, device=dev)
        P.p3t_build_tree(ctx, st, False, stream)
        P.p3t_soft_force(ctx, st, acc, None, stream)
        torch.cuda.synchronize(dev)
        g = st.numpy()
        ref = O.tree_soft(g, g["r_out"], g["r_search"], op).acc
        a = acc.cpu().numpy().T
        e = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
        rms = float(np.sqrt((ref * ref).sum(1).mean()))
        return dict(max=float(e.max()), p99=float(np.percentile(e, 99)),
                    median=float(np.median(e)),
                    max_over_rms=float(np.linalg.norm(a - ref, axis=1).max() / rms))

    out = {}
    for name, prec in (("fp64", P.P3T_FP64), ("mixed", P.P3T_MIXED)):
        prm = P.Params(theta=0.5, precision=prec, eta=0.01, eta0=0.001, group_size=64)
        op = O.Params(theta=0.5, eta=0.01, eta0=0.001, group_size=64)
        st = P.State.from_numpy(s0, device=dev)
        ss = P.SoftStep(prm, st, device=0)
        ss.init(update_cutoffs=True)
        ss.status()
        err0 = force_err(st, ss.ctx, op)
        ss.force(stream)                       # the step's force again (tree of this state)
        counts = torch.zeros(K, 2, dtype=torch.int64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        E = torch.zeros(2, 4, dtype=torch.float64, device=dev)
        P.p3t_energy(ss.ctx, st, E[0], stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for k in range(K):
            ss.counts = counts[k]
            ss.step(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ss.status()
        P.p3t_energy(ss.ctx, st, E[1], stream)
        t = e0.elapsed_time(e1) / 1e3
        errK = force_err(st, ss.ctx, op)
        Ev = E.cpu().numpy()
        out[name] = dict(ms_per_step=1e3 * t / K, value=float(counts.sum().item()) / t,
                         force_error_initial=err0, force_error_after_64=errK,
                         energy_error=abs(Ev[1, 0] / Ev[0, 0] - 1.0))
        ss.close()
    line = dict(study="precision", metric="soft step: FP64 vs mixed path, force error vs the "
                "FP64 oracle", unit=UNIT, n=n, steps=K,
                config=dict(workload=f"equal-mass ring N={n}, 0.9-1.1 au, m=1e-11, e/i rms "
                            "0.01/0.005, theta=0.5, leaf 16, groups of <= 64, dt=1/64, eta=0.01"),
                data="synthetic (seeded ring)", **out)
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- ensemble ------
def run_ensemble(args):
    """256 independent disks (sizes round(exp U(ln 512, ln 16384)), seeds
    4000 + d; even disks equal-mass rings, odd disks power-law wide disks), no
    collisions.  Three ways to step them, each timed over the same K steps:
    batched (one context, every disk a segment of one particle set, so one
    launch sequence per step for all disks; group size from the batched
    autotuner; replayed as a captured CUDA graph), per-disk contexts in a
    captured graph (disks forked over 16 streams; group sizes per disk-size
    class from the per-disk autotuner) and the per-disk kernels issued disk
    after disk on one stream.  Value: pair interactions of all disks per
    second of the batched step."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2007_15432_gb300 import build, disks
    build.build()
    from paper_2007_15432_gb300 import ensemble as EN
    from paper_2007_15432_gb300 import p3t as P
    ds = disks.ensemble_disks()
    base = P.Params(theta=0.5, precision=P.P3T_MIXED, eta=0.01, eta0=0.001)
    K, W = args.steps, args.warmup

    def timed(run, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            run()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    # batched
    ens = EN.Ensemble(ds, [base] * len(ds), batched=True)
    ens.init()
    t0 = time.perf_counter()
    tune_b = ens.autotune_batched()
    t_tune_b = time.perf_counter() - t0
    l0 = P.p3t_launch_count()
    ens.step_sequential()
    launches_b = P.p3t_launch_count() - l0
    ens.capture()
    for _ in range(W):
        ens.step_graph()
    torch.cuda.synchronize(dev)
    t_b = timed(ens.step_graph, K)
    ens.status()
    inter_b = ens.interactions()
    ens.close()

    # per-disk contexts
    t0 = time.perf_counter()
    tune = EN.autotune(ds, base)
    t_tune = time.perf_counter() - t0
    params = []
    for d in ds:
        p = P.Params(**{f[0]: getattr(base, f[0]) for f in P.Params._fields_})
        p.group_size = tune[EN.size_class(len(d["m"]))]
        params.append(p)
    ens = EN.Ensemble(ds, params)
    ens.init()
    l0 = P.p3t_launch_count()
    ens.step_sequential()
    launches_d = P.p3t_launch_count() - l0
    ens.capture()
    for _ in range(W):
        ens.step_graph()
    torch.cuda.synchronize(dev)
    t_graph = timed(ens.step_graph, K)
    ens.status()
    inter = ens.interactions()
    for _ in range(W):
        ens.step_sequential()
    torch.cuda.synchronize(dev)
    t_seq = timed(ens.step_sequential, K)
    ens.status()
    inter_seq = ens.interactions()
    ens.close()
    line = dict(metric="ensemble soft step: pair-interactions/s of all disks", study="ensemble",
                value=inter_b / (t_b / K), unit=UNIT, n_gpus=1, steps=K, warmup=W,
                ms_per_step=1e3 * t_b / K, higher_is_better=True,
                gpu_launches=launches_b * K,
                batched=dict(tuned=tune_b, autotune_s=t_tune_b, launches_per_step=launches_b),
                per_disk_graph=dict(value=inter / (t_graph / K), ms_per_step=1e3 * t_graph / K,
                                    launches_per_step=launches_d, streams=16,
                                    group_size_by_log2_n={str(k): v
                                                          for k, v in sorted(tune.items())},
                                    autotune_s=t_tune),
                sequential=dict(value=inter_seq / (t_seq / K), ms_per_step=1e3 * t_seq / K),
                speedup_vs_per_disk_graph=t_graph / t_b, speedup_vs_sequential=t_seq / t_b,
                dtype="f32/f64", data="synthetic (seeded disks)",
                config=dict(workload="ensemble of 256 disks, sizes round(exp U(ln 512, ln 16384))",
                            n_total=int(sum(len(d["m"]) for d in ds))))
    print(json.dumps(line), flush=True)
    return 0


def run_adjoint(args):
    """The differentiation workload: N = 1e4 equal-mass ring on 0.95-1.05 au
    (m = 1e-10, seed 1006), 32 soft kick-drift-kick steps (every particle on
    its Kepler orbit, direct changeover soft force, cut-off radii frozen at
    the initial state), checkpoint every 8 steps, FP32 pair arithmetic with
    FP64 state.  One step = one gradient of L = sum |x_N - x_target|^2 with
    respect to x_0, v_0 and m (forward sweep + checkpointed reverse sweep);
    x_target = x_N + seeded offsets of rms 1e-4 au.  Value: pair terms of
    the forward forces, the recomputed forces and the VJPs per second."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2007_15432_gb300 import build, disks
    build.build()
    from paper_2007_15432_gb300 import adjoint as AD
    from paper_2007_15432_gb300 import p3t as P
    n, steps, ck = args.adjoint_n, 32, 8
    s = disks.adjoint_disk(n)
    X0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]]), device=dev)
    V0 = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]]), device=dev)
    M = torch.tensor(s["m"], device=dev)
    p3t = args.adjoint_form == "p3t"
    if p3t:
        prm = P.Params(theta=0.5, precision=P.P3T_FP64, group_size=64)
        RO, RS = AD.cutoffs(prm, X0, V0, M, with_search=True)
        run = AD.SoftKDK(prm, n, steps, ck, force="tree", hard="p3t")
    else:
        RO, RS = AD.cutoffs(P.Params(), X0, V0, M), None
        run = AD.SoftKDK(P.Params(precision=P.P3T_MIXED), n, steps, ck)
    TGT = run.forward(X0, V0, M, RO, RS)[0] + torch.tensor(disks.target_offsets(n), device=dev)

    def grad():
        x0, v0, m = X0.clone().requires_grad_(True), V0.clone().requires_grad_(True), \
            M.clone().requires_grad_(True)
        xN, _ = AD.soft_kdk(x0, v0, m, RO, run, RS)
        ((xN - TGT) ** 2).sum().backward()
        return x0.grad, v0.grad, m.grad

    K, W = args.steps, args.warmup
    for _ in range(W):
        grad()
    torch.cuda.synchronize(dev)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(K):
        grad()
    e[1].record()
    torch.cuda.synchronize(dev)
    t = e[0].elapsed_time(e[1]) / 1e3 / K
    # phases of one gradient
    e[0].record()
    xN, vN, tape = run.forward(X0, V0, M, RO, RS)
    e[1].record()
    run.backward(tape, 2.0 * (xN - TGT), torch.zeros_like(vN))
    e[2].record()
    torch.cuda.synchronize(dev)
    t_fwd, t_bwd = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    if p3t:
        run.status()
        line = dict(metric="adjoint of 32 soft KDK steps at N=1e4 (tree force, Hermite clusters):"
                    " gradient time", study="adjoint", form="p3t", value=1e3 * t,
                    unit="ms per gradient", n_gpus=1, steps=K, warmup=W, ms_per_step=1e3 * t,
                    higher_is_better=False,
                    phases_ms=dict(forward=1e3 * t_fwd, backward=1e3 * t_bwd),
                    dtype="f64", data="synthetic (seeded ring)",
                    config=dict(workload=f"equal-mass ring N={n}, 0.95-1.05 au, m=1e-10, 32 KDK "
                                "steps, checkpoint 8, theta=0.5, groups of <= 64", n=n,
                                steps_per_gradient=steps, checkpoint=ck))
        run.close()
        print(json.dumps(line), flush=True)
        return 0
    lp = torch.zeros(3, n, dtype=torch.float64, device=dev)
    lxx = torch.zeros(3, n, dtype=torch.float64, device=dev)
    gm = torch.zeros(n, dtype=torch.float64, device=dev)
    st = run._state(X0.contiguous(), V0.contiguous(), M, RO)
    e[3].record()
    for _ in range(10):
        P.p3t_soft_force_vjp(run.ctx, st, 1.0, lp, lxx, gm)
    e4 = torch.cuda.Event(enable_timing=True)
    e4.record()
    torch.cuda.synchronize(dev)
    run.status()
    t_vjp = e[3].elapsed_time(e4) / 1e3 / 10
    segs = (steps + ck - 1) // ck
    forces = (steps + 1) + (steps + segs)  # forward sweep + recomputation
    vjps = steps + 1
    pairs = float(n) * (n - 1)
    # FP32 work of one VJP pair term (float-float difference 9, r2 5, rsqrt,
    # y and the changeover polynomial ~14, phi/psi 7, w 6, the four sums 14)
    flop_vjp = 55.0
    line = dict(metric="adjoint of 32 soft KDK steps at N=1e4: gradient time and pair terms/s",
                study="adjoint", value=(forces + vjps) * pairs / t, unit=UNIT, n_gpus=1, steps=K,
                warmup=W, ms_per_step=1e3 * t, higher_is_better=True,
                phases_ms=dict(forward=1e3 * t_fwd, backward=1e3 * t_bwd, soft_vjp=1e3 * t_vjp),
                roofline=dict(kernel="k_soft_vjp<FP32>", bound="alu",
                              achieved=flop_vjp * pairs / t_vjp / 1e12, peak=FP32_PEAK_TFLOPS,
                              unit="TFLOP/s", frac=flop_vjp * pairs / t_vjp / 1e12 / FP32_PEAK_TFLOPS,
                              traffic=None),
                dtype="f32 pair terms / f64 state", data="synthetic (seeded ring)",
                config=dict(workload=f"equal-mass ring N={n}, 0.95-1.05 au, m=1e-10, 32 KDK steps, "
                            "checkpoint 8", n=n, steps_per_gradient=steps, checkpoint=ck,
                            forces_per_gradient=forces, vjps_per_gradient=vjps))
    run.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.adjoint:
        return run_adjoint(args)
    if args.ensemble:
        return run_ensemble(args)
    if args.cutoff_sweep:
        return run_cutoff_sweep(args)
    if args.precision_study:
        return run_precision_study(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
