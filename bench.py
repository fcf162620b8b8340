"""Benchmark of the hot path: particle-steps/s of the binary Lennard-Jones mixture on one
GB300, default workload = the 16,384,000-particle supercooling quench (FCC 4*160^3, 80:20,
rho = 1.2, Nose-Hoover ramp 2.0 -> 0.4 over 1e5 steps, dt = 0.005, mixed precision,
Verlet list with skin 0.4 by default, --skin).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Besides the 16M-particle line it measures, in the same run, the 1,024,191,500-particle
cell-mode step (mixed and FP64 forms: "large") and a batch of 64 replicas of uneven size
("replicas"); --large-steps 0 / --replicas 0 skip them.

Prints one JSON line (rank 0).  `value` is device-timed (CUDA events on the handle's
stream, state resident in HBM); `e2e` is the same metric through the C ABI with host
buffers (upload of the state, the steps, energy read-back and download of the state).
Under torchrun each rank runs its own independent replica (weak scaling; the single
system is not decomposed across GPUs).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RAMP_STEPS = 100_000
T_HIGH, T_LOW, TAU, DT = 2.0, 0.4, 0.5, 0.005
NCELL_FCC = 160                      # N = 4 * 160^3 = 16,384,000
FLOP_PER_HALF_PAIR = 25.0            # r^2, reciprocal, LJ force scalar and vector update
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_PER_SM_CLK = 128                # FP32 lanes per SM (nominal, for the derived peak)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def workload_config(args, ws):
    """The "config" object of both arms: the supercooling-quench workload."""
    from inputs import generate as gen

    n = 4 * args.ncell ** 3
    return {"workload": f"supercooling quench, N={n} (4*{args.ncell}^3 FCC, 80:20), rho=1.2, "
                        "equilibrated at T=2.0, Nose-Hoover ramp 2.0->0.4 over 1e5 steps, "
                        f"dt=0.005, mixed, Verlet skin {args.skin}",
            "equilibration_steps": args.equil, "n_particles": n, "box": gen.box_for(n, 1.2),
            "parallelism": f"replicas x{ws}",
            "l2": "state and per-step traffic (>6 GB) far larger than the 129 MB L2"}


def max_over_ranks(x, device="cpu"):
    """Largest value of x over the ranks of the default process group (x itself alone)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world_size, ms_max):
    """Whole-job throughput: the units every rank processed over the slowest rank's time
    (every rank runs the same independent workload: weak scaling)."""
    return world_size * units_per_rank / (ms_max / 1e3)


def ramp_T(step):
    return T_HIGH + (T_LOW - T_HIGH) * min(step, RAMP_STEPS) / RAMP_STEPS


def half_pairs_per_particle(rho=1.2, xb=0.2, rc_factor=2.5):
    """Expected interacting pairs per particle inside r_c,ab (uniform-density estimate):
    1/2 sum_ab x_a x_b rho (4 pi / 3) rc_ab^3."""
    sig = ((1.0, 0.8), (0.8, 0.88))
    x = (1.0 - xb, xb)
    s = 0.0
    for a in range(2):
        for b in range(2):
            rc = rc_factor * sig[a][b]
            s += x[a] * x[b] * rho * 4.0 * math.pi / 3.0 * rc ** 3
    return 0.5 * s


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms into a temporary file
    (copied to `keep` when given, e.g. as evidence beside a profile)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, keep=None, gpu=None, tmpdir=None):
        import tempfile

        fd, self.path = tempfile.mkstemp(prefix="bbmd_clocks_", suffix=".csv", dir=tmpdir)
        os.close(fd)
        self.keep = keep
        self.gpu = gpu  # nvidia-smi index of this rank's GPU (None: every GPU)
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            sel = [] if self.gpu is None else ["-i", str(self.gpu)]
            self.proc = subprocess.Popen(
                ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
        if self.keep:
            try:
                shutil.copyfile(self.path, self.keep)
            except OSError:
                pass

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r]
            os.unlink(self.path)
        except Exception:
            rows = []
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_stream():
    import torch

    return torch.cuda.Stream()


def run_ours(args):
    import torch

    from inputs import generate as gen
    from paper_1105_5613_gb300 import bbmd
    from paper_1105_5613_gb300 import build as b

    ws, rank = _dist()
    if ws > 1:
        import torch.distributed as dist

        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if rank == 0:
        b.build()  # one rank compiles (a no-op when the library is up to date)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    bbmd.load()
    n = 4 * args.ncell ** 3
    L = gen.box_for(n, 1.2)
    sp = gen.assign_species(n, n // 5, 0)
    stream = make_stream()
    p = bbmd.ka_params(nbr_mode=bbmd.NBR_CELL if args.profile_cell else bbmd.NBR_VERLET,
                       block_z=args.block_z, skin=args.skin)
    sim = bbmd.Sim(p, n, L, sp, None, None, T0=T_HIGH, seed=rank, stream=stream.cuda_stream,
                   use_torch_allocator=True)
    step = 0

    def therm(k):
        return (bbmd.THERMO_NH, ramp_T(step), ramp_T(step + k), TAU)

    # the workload starts from an equilibrated liquid at T=2.0 (untimed; not part of the
    # ramp), then untimed warm-up steps of the ramp (the first also captures the graph)
    if args.equil > 0:
        sim.step(args.equil, DT, (bbmd.THERMO_NH, T_HIGH, T_HIGH, TAU))
        sim.tune()  # block shape re-timed on the liquid (creation timed it on the lattice)
    if args.profile_phases > 0:
        # profiling case: one forced rebuild, then K steps with every phase launched on
        # its own (the kernel launches that ncu captures), per-phase times printed
        sim.rebuild()
        k = args.profile_phases
        ph, nr = sim.step_profiled(k, DT, (bbmd.THERMO_NH, T_HIGH, T_HIGH, TAU))
        stream.synchronize()
        sim_block_z = sim.info()["block_z"]
        sim.close()
        if rank == 0:
            print(json.dumps({"profile_case": {"n_particles": n, "equil": args.equil,
                                               "block_z": sim_block_z,
                                               "steps": k, "rebuilds": nr,
                                               "phases_ms_per_step":
                                                   {a: v / k for a, v in ph.items()}}}))
        return None
    sim.step(args.warmup, DT, therm(args.warmup))
    step += args.warmup
    stream.synchronize()
    rebuilds_before = sim.observe(0)["n_rebuilds"]  # (synchronising; outside the timed region)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- device-timed region ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    local_gpu = torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else None
    keep = os.environ.get("BBMD_CLOCKS_CSV")  # optional copy of the raw samples
    clk = ClockSampler(f"{keep}.rank{rank}" if keep else None, gpu=local_gpu)
    barrier()
    torch.cuda.synchronize()
    with clk:
        e0.record(stream)
        sim.step(args.steps, DT, therm(args.steps))
        e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    step += args.steps
    ms = e0.elapsed_time(e1)
    if ws > 1:
        import torch.distributed as dist

        ms = max_over_ranks(ms, "cuda")
    obs = sim.observe(bbmd.OBS_ENERGY)
    timed_rebuilds = obs["n_rebuilds"] - rebuilds_before
    info = sim.info()
    block_z = info["block_z"]
    # the re-tuning's per-shape times on the equilibrated liquid (0: shape not timed)
    shape_times = {"block_z": [1, 2, 4, 8], "force_ms": info["shape_force_ms"],
                   "list_ms": info["shape_list_ms"]}
    clocks = clk.summary()

    # ---- measured FP32 / FP64 FMA peaks of this GPU (the ALU roofline denominators) ----
    probe = optional_leg(fma_probe, bbmd, local_gpu)

    # ---- per-phase attribution (same steps, phases launched one by one) ----
    nprof = max(2, min(args.steps, 10))
    phases, nreb = sim.step_profiled(nprof, DT, therm(nprof))
    step += nprof
    force_ms = phases["force"] / nprof

    # ---- end-to-end through the C ABI with host buffers ----
    pos, vel, img = sim.get_state()
    pin = [torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.int32,
                       pin_memory=True) for a in (pos, vel, img)]
    for t, a in zip(pin, (pos, vel, img)):
        t.numpy()[...] = a
    hp, hv, hi = (t.numpy() for t in pin)
    outp = [torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.int32,
                        pin_memory=True) for a in (pos, vel, img)]
    gp, gv, gi = (t.numpy() for t in outp)
    ke2 = max(1, args.e2e_steps)
    obs_bytes = ctypes_sizeof_obs(bbmd)
    barrier()
    t0 = time.perf_counter()
    # upload of the state from pinned host memory, then every step: one step and the read
    # back of its result (kinetic energy, temperature, momentum, step count), then the
    # download of the final state into pinned host memory
    sim.set_state(hp, hv, hi)
    for k in range(ke2):
        sim.step(1, DT, (bbmd.THERMO_NH, ramp_T(step + k), ramp_T(step + k + 1), TAU))
        sim.observe(0)
    sim.get_state(out=(gp, gv, gi))
    t1 = time.perf_counter()
    barrier()
    step += ke2
    e2e_s = t1 - t0
    h2d = hp.nbytes + hv.nbytes + hi.nbytes
    d2h = gp.nbytes + gv.nbytes + gi.nbytes + ke2 * obs_bytes
    sim.close()

    # ---- FP64 form on the same workload (a few steps) ----
    def leg_fp64():
        p64 = bbmd.ka_params(precision=bbmd.PREC_FP64, skin=args.skin)
        sim64 = bbmd.Sim(p64, n, L, sp, None, None, T0=T_HIGH, seed=rank,
                         stream=stream.cuda_stream, use_torch_allocator=True)
        sim64.step(1, DT, therm(1))
        stream.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k64 = args.fp64_steps
        a0.record(stream)
        sim64.step(k64, DT, therm(k64))
        a1.record(stream)
        a1.synchronize()
        ms64 = a0.elapsed_time(a1)
        ph64, _ = sim64.step_profiled(1, DT, therm(1))
        sim64.close()
        return {"value": n * k64 / (ms64 / 1e3), "unit": "particle-steps/s", "steps": k64,
                "ms_per_step": ms64 / k64, "force_ms": ph64["force"]}

    fp64 = None if args.no_fp64 else optional_leg(leg_fp64)

    # ---- soft-sphere mixture with the shifted-force truncation (Eqs. sc0, mod0), the paper's
    # own benchmark potential, on the same N: melted at T=2.0, then timed at T=0.5 ----
    def leg_soft():
        ps = bbmd.ka_params(potential=bbmd.POT_SOFT, shift=bbmd.SHIFT_FORCE, skin=args.skin)
        sims = bbmd.Sim(ps, n, L, sp, None, None, T0=T_HIGH, seed=rank,
                        stream=stream.cuda_stream, use_torch_allocator=True)
        sims.step(200, DT, (bbmd.THERMO_NH, T_HIGH, 0.5, TAU))
        sims.tune()
        sims.step(args.warmup, DT, (bbmd.THERMO_NH, 0.5, 0.5, TAU))
        stream.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sims.step(args.soft_steps, DT, (bbmd.THERMO_NH, 0.5, 0.5, TAU))
        s1.record(stream)
        s1.synchronize()
        mss = s0.elapsed_time(s1)
        out = {"workload": f"soft-sphere mixture (Eq. sc0) with shifted-force truncation "
                           f"(Eq. mod0), rc = 2.5 sigma_ab, N={n}, rho=1.2, Nose-Hoover T=0.5 "
                           "after melting at T=2.0",
               "value": n * args.soft_steps / (mss / 1e3), "unit": "particle-steps/s",
               "steps": args.soft_steps, "ms_per_step": mss / args.soft_steps,
               "block_z": sims.info()["block_z"],
               "T": sims.observe(bbmd.OBS_ENERGY)["temperature"]}
        sims.close()
        return out

    soft = optional_leg(leg_soft) if args.soft_steps > 0 else None
    replicas = optional_leg(run_replicas, args, stream) if args.replicas > 0 else None
    peak_for_large = probe.get("fp32_tflops") if isinstance(probe, dict) else None
    large = (optional_leg(run_large, args, stream, peak_for_large)
             if args.large_steps > 0 or args.large_fp64_steps > 0 else None)
    if rank != 0:
        return None
    value = whole_job_rate(n * args.steps, ws, ms)
    pk = peaks()
    clock_mhz = pk.get("sm_max_mhz", 2070.0)
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    derived = nsm * FP32_PER_SM_CLK * 2 * clock_mhz * 1e6 / 1e12  # TFLOP/s
    measured = probe.get("fp32_tflops") if isinstance(probe, dict) else None
    fp32_peak = measured or derived
    hp_per = half_pairs_per_particle()
    flops_launch = n * hp_per * FLOP_PER_HALF_PAIR
    achieved = flops_launch / (force_ms / 1e3) / 1e12
    traffic = force_traffic(n, args.skin)
    out = {
        "metric": "particle-steps/s (binary LJ, 16M & 1.02B N) mixed vs FP64 GPU; % of roofline",
        "value": value,
        "unit": "particle-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 pair forces, i64 fixed-point state, f64 reductions",
        "data": f"synthetic: FCC 4*{args.ncell}^3 lattice, seeded 80:20 species, "
                "Maxwell-Boltzmann T=2.0",
        "config": workload_config(args, ws),
        "e2e": {"value": ws * n * ke2 / e2e_s, "unit": "particle-steps/s",
                "h2d_bytes_per_step": h2d / ke2, "d2h_bytes_per_step": d2h / ke2,
                "steps": ke2},
        "roofline": {"bound": "alu", "kernel": "k_force (Verlet list, NH kinetic partials)",
                     "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic,
                     "peak_source": ("measured: FP32 FMA-chain probe (bbmd_fma_peak), this run"
                                     if measured else
                                     f"derived: {nsm} SMs x {FP32_PER_SM_CLK} FP32 lanes x 2 "
                                     f"flop x {clock_mhz:.0f} MHz"),
                     "peak_derived": derived,
                     "algorithmic": f"{hp_per:.2f} half pairs/particle x {FLOP_PER_HALF_PAIR:.0f} "
                                    f"flop x {n} particles per launch",
                     "force_ms": force_ms,
                     "issue": force_issue(n, force_ms, block_z, clock_mhz, nsm, args.skin)},
        "fma_probe": probe,
        "phases_ms_per_step": {k: v / nprof for k, v in phases.items()},
        "block_z": block_z,
        "shape_times": shape_times,
        "rebuilds_per_step": timed_rebuilds / args.steps,  # over the timed steps
        "phases_rebuilds_per_step": nreb / nprof,
        # per step: integrate, 2 trigger kernels, 9 gated sort kernels, gated list build,
        # list force and the stencil force that stands in for cut lists (one of the two
        # returns at once), finalize (one graph); plus begin and finish of the call
        "gpu_launches": args.steps * 16 + 2,
        "clocks": clocks,
        "fp64": fp64,
        "large": large,
        "soft_sphere": soft,
        "replicas": replicas,
        "observables": {"T": obs["temperature"], "pe_per_particle": obs["pe"] / n},
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = optional_leg(cpu_baseline, args.cpu_seconds)
    return out


def optional_leg(fn, *a):
    """Run one secondary leg of the bench; a failure is reported in its place (an "error"
    entry) instead of ending the run, so the headline line is printed either way."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - any failure of a secondary leg
        try:
            import torch

            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        except Exception:  # noqa: BLE001
            pass
        return {"error": f"{type(e).__name__}: {str(e)[:300]}"}


def run_large(args, stream, fp32_peak=None):
    """The 1,024,191,500-particle step: FCC 4*635^3 (80:20) at rho = 1.2, displaced by the
    generator's seeded jitter (0.05 per coordinate), T = 0.6 NVE, dt = 0.005, forces from
    the cell stencil on the fly (no stored Verlet list), positions and velocities
    generated on the device.  Mixed precision: args.large_untimed untimed steps, then
    args.large_steps timed steps, then 2 steps phase by phase (per-phase split and the
    roofline of the cell-mode force kernel); then the FP64 form over
    args.large_fp64_steps steps (one handle at a time)."""
    import torch

    from inputs import generate as gen
    from paper_1105_5613_gb300 import bbmd

    torch.cuda.empty_cache()  # the 16M handles' memory back to the driver
    ncell = args.large_ncell
    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    t0 = time.perf_counter()
    sp = gen.assign_species(n, n // 5, 0)
    t_species = time.perf_counter() - t0
    out = {"workload": f"large step, N={n} (4*{ncell}^3 FCC jittered by 0.05, 80:20), "
                       "rho=1.2, T=0.6 NVE, dt=0.005, cell stencil on the fly (no stored list)",
           "n_particles": n, "box": L, "species_host_s": t_species}
    for prec, steps, key in ((bbmd.PREC_MIXED, args.large_steps, "mixed"),
                             (bbmd.PREC_FP64, args.large_fp64_steps, "fp64")):
        if steps <= 0:
            continue
        p = bbmd.ka_params(precision=prec, nbr_mode=bbmd.NBR_CELL, init_jitter=0.05)
        t0 = time.perf_counter()
        sim = bbmd.Sim(p, n, L, sp, None, None, T0=0.6, seed=0, stream=stream.cuda_stream)
        t_create = time.perf_counter() - t0
        untimed = args.large_untimed if prec == bbmd.PREC_MIXED else 1
        sim.step(untimed, DT)
        stream.synchronize()
        r0 = sim.observe(0)["n_rebuilds"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps, DT)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        info = sim.info()
        obs = sim.observe(0)  # kinetic only: the FP64 energy pass of 1e9 particles takes ~20 s
        out[key] = {"value": n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps,
                    "untimed_steps_before": untimed,
                    "ms_per_step": ms / steps, "create_s": t_create, "block_z": info["block_z"],
                    "rebuilds_per_step": (obs["n_rebuilds"] - r0) / steps,
                    "device_gb": info["device_bytes"] / 1e9, "T": obs["temperature"]}
        if prec == bbmd.PREC_MIXED:
            nprof = 2
            ph, nreb = sim.step_profiled(nprof, DT)
            force_ms = ph["force"] / nprof
            out[key]["phases_ms_per_step"] = {k: v / nprof for k, v in ph.items()}
            out[key]["phase_rebuilds"] = nreb
            if fp32_peak:
                hp_per = half_pairs_per_particle()
                ach = n * hp_per * FLOP_PER_HALF_PAIR / (force_ms / 1e3) / 1e12
                out[key]["roofline"] = {
                    "bound": "alu", "kernel": "k_force (cell stencil on the fly, NVE)",
                    "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak, "force_ms": force_ms,
                    "algorithmic": f"{hp_per:.2f} half pairs/particle x "
                                   f"{FLOP_PER_HALF_PAIR:.0f} flop x {n} particles per launch"}
        sim.close()
        del sim
    return out


def run_replicas(args, stream):
    """Batched replicas: args.replicas mixtures of uneven size N_r in [2048, 32768] (multiples
    of 5), random sequential addition (d_min = 0.7) relaxed by 200 steepest-descent steps,
    temperatures evenly spaced in [0.4, 2.0], Nose-Hoover (tau = 0.5), dt = 0.005; all
    replicas advanced by the persistent kernel, one launch for the timed steps
    (bbmd_step_batch)."""
    import torch

    from inputs import generate as gen
    from paper_1105_5613_gb300 import bbmd

    R = args.replicas
    t0 = time.perf_counter()
    ns, boxes, pos, sp = gen.replica_batch(R, 2048, 32768, 0)
    t_gen = time.perf_counter() - t0
    temps = [0.4 + 1.6 * r / max(R - 1, 1) for r in range(R)]
    t0 = time.perf_counter()
    b = bbmd.Batch(bbmd.ka_params(skin=args.replica_skin), ns, boxes, sp, pos, None, T0=temps,
                   seed=0, stream=stream.cuda_stream)
    for r in range(R):
        b.replica(r).minimize(200)
    stream.synchronize()
    t_setup = time.perf_counter() - t0
    th = [(bbmd.THERMO_NH, T, T, TAU) for T in temps]
    b.step(args.warmup, DT, th)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.replica_steps, DT, th)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    shapes = sorted({b.replica(r).info()["block_z"] for r in range(R)})
    path = "persistent" if b.uses_persistent() else "graph"
    Ts = [b.replica(r).observe(bbmd.OBS_ENERGY)["temperature"] for r in (0, R - 1)]
    b.close()
    ntot = sum(ns)
    return {"workload": f"{R} replicas, N_r in [2048, 32768] (sum {ntot}), RSA + 200 SD steps, "
                        f"T_r = 0.4 .. 2.0, Nose-Hoover, dt=0.005, skin {args.replica_skin}, "
                        + ("one persistent kernel launch per call (up to 1024 steps)"
                           if path == "persistent" else "one graph launch per step"),
            "path": path,
            "value": ntot * args.replica_steps / (ms / 1e3), "unit": "particle-steps/s",
            "steps": args.replica_steps, "ms_per_step": ms / args.replica_steps,
            "n_total": ntot, "block_z_used": shapes, "generate_s": t_gen, "setup_s": t_setup,
            "T_first_last": Ts}


def fma_probe(bbmd, gpu=None):
    """Measured FP32 and FP64 fused multiply-add peaks of this GPU (bbmd_fma_peak: FMA
    chains with no memory traffic, CUDA events, best of 3), with the SM clocks sampled
    while it ran."""
    clk = ClockSampler(gpu=gpu)
    with clk:
        f32, nsm = bbmd.fma_peak(bbmd.PREC_MIXED)
        f64, _ = bbmd.fma_peak(bbmd.PREC_FP64)
        # shared-memory scatter-adds (the reaction update of a half-list kernel)
        scatter = {name: bbmd.smem_scatter_rate(kind)
                   for kind, name in ((0, "fixed64_from_f32"), (1, "u32"), (2, "f32"))}
    return {"fp32_tflops": f32, "fp64_tflops": f64, "sm_count": nsm,
            "smem_scatter_adds_per_s": scatter, "clocks": clk.summary()}


def ctypes_sizeof_obs(bbmd):
    import ctypes

    return ctypes.sizeof(bbmd.bbmd_obs)


def force_counters(skin=None):
    """The committed ncu record of one list-mode k_force launch (DRAM bytes and warp
    instructions per particle, block shape, skin), or None when the kernel source changed
    since those counters were taken, or the record is of another skin (the list length
    follows the skin)."""
    import hashlib

    tf = os.path.join(ROOT, "profiles", "force_traffic.json")
    src = os.path.join(ROOT, "paper_1105_5613_gb300", "csrc", "k_force.cu")
    try:
        rec = json.load(open(tf))
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
        if skin is not None and abs(rec.get("skin", 0.3) - skin) > 1e-9:
            return None
        return rec if rec.get("k_force_cu_sha1") == sha else None
    except Exception:
        return None


def force_traffic(n, skin=None):
    """DRAM bytes (read + write) per k_force launch, scaled to n particles (every array the
    kernel touches is per particle), or None."""
    rec = force_counters(skin)
    return rec["bytes_per_particle"] * n if rec else None


def force_issue(n, force_ms, block_z, clock_mhz, nsm, skin=None):
    """Issue-slot view of the same launch: warp instructions (from the ncu record, same
    block shape) per second against 4 warp instructions per SM per cycle."""
    rec = force_counters(skin)
    if not rec or rec.get("block_z") != block_z or "warp_inst_per_particle" not in rec:
        return None
    peak = nsm * 4 * clock_mhz * 1e6
    rate = rec["warp_inst_per_particle"] * n / (force_ms / 1e3)
    return {"warp_inst_per_s": rate, "peak": peak, "frac": rate / peak,
            "warp_inst_per_particle": rec["warp_inst_per_particle"]}


def cpu_sample_state(ncell=40, seed=0):
    from inputs import generate as gen

    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    pos = gen.fcc_lattice(ncell, L)
    sp = gen.assign_species(n, n // 5, seed)
    vel = gen.maxwell_boltzmann(n, T_HIGH, seed, np.ones(n))
    return n, L, pos, vel, sp


def cpu_baseline(budget_s=15.0, ncell=40):
    """The FP64 oracle as it stands (single thread, cell search with Newton's third law),
    on a bounded sample of the workload: N = 4*40^3 of the same mixture and ramp."""
    import oracle

    n, L, pos, vel, sp = cpu_sample_state(ncell)
    st = oracle.MDState(pos, vel, sp, L, oracle.ka_params())
    oracle.md_run(st, 1, DT, thermo=(T_HIGH, T_HIGH, TAU), use_cells=True)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle.md_run(st, 1, DT, thermo=(ramp_T(steps), ramp_T(steps + 1), TAU), use_cells=True)
        steps += 1
    dt = time.perf_counter() - t0
    out = {"value": n * steps / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"N={n} (4*{ncell}^3 FCC, same mixture, rho=1.2, NH ramp), {steps} steps, "
                     f"{dt:.1f} s, FP64 cell search, single thread"}
    # second mode: the oracle's full-stencil force form on every core (same state, ramp)
    st = oracle.MDState(pos, vel, sp, L, oracle.ka_params())
    oracle.md_run(st, 1, DT, thermo=(T_HIGH, T_HIGH, TAU), use_cells="all_cores")
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s / 3:
        oracle.md_run(st, 1, DT, thermo=(ramp_T(steps), ramp_T(steps + 1), TAU),
                      use_cells="all_cores")
        steps += 1
    dt = time.perf_counter() - t0
    out["all_cores"] = {"value": n * steps / dt, "unit": "particle-steps/s",
                        "cores": oracle.threads(), "kind": "oracle",
                        "sample": f"the same N={n} state, {steps} steps, {dt:.1f} s, FP64 "
                                  "full-stencil forces over every core (OpenMP)"}
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return None
    import oracle

    n, L, pos, vel, sp = cpu_sample_state(20)
    st = oracle.MDState(pos, vel, sp, L, oracle.ka_params())
    for k in range(args.warmup):
        oracle.md_run(st, 1, DT, thermo=(ramp_T(k), ramp_T(k + 1), TAU), use_cells=True)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.md_run(st, 1, DT, thermo=(ramp_T(k), ramp_T(k + 1), TAU), use_cells=True)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    sample = (f"N={n} (4*20^3 FCC, same mixture, rho=1.2, NH ramp) per step, FP64 oracle, "
              f"single thread")
    # the config names what this arm timed: a bounded sample of the workload
    config = workload_config(args, ws)
    config["sample_of"] = config["workload"]
    config["workload"] = (f"bounded sample of the supercooling quench: N={n} (4*20^3 FCC, "
                          "80:20), rho=1.2, same Nose-Hoover ramp and dt, FP64 oracle, "
                          "single thread")
    config["n_particles"] = n
    config["box"] = L
    return {"impl": "reference", "metric": "particle-steps/s (binary LJ, 16M & 1.02B N) mixed vs "
            "FP64 GPU; % of roofline", "value": v, "unit": "particle-steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--skin", type=float, default=0.4,
                    help="Verlet skin of the 16 M workload and its FP64 and soft-sphere legs "
                         "(0.4: the fastest of 0.25-0.6 measured at 16 M; the 1.02 B cell-mode "
                         "step keeps 0.3, its fastest)")
    ap.add_argument("--equil", type=int, default=400,
                    help="untimed equilibration steps at T=2.0 before the ramp")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ncell", type=int, default=NCELL_FCC,
                    help="FCC cells per edge (N = 4 ncell^3); the workload is ncell = 160")
    ap.add_argument("--soft-steps", type=int, default=100,
                    help="timed steps of the soft-sphere / shifted-force variant (0 = skip)")
    ap.add_argument("--replicas", type=int, default=64,
                    help="number of replicas of the batched-replica leg (0 = skip)")
    ap.add_argument("--replica-steps", type=int, default=500)
    ap.add_argument("--replica-skin", type=float, default=0.3,
                    help="Verlet skin of the replicas (their boxes need 4 cells a side for the "
                         "batch's 2 x 2 x 4 blocks)")
    ap.add_argument("--large-steps", type=int, default=20,
                    help="timed mixed-precision steps of the 1.02e9-particle cell-mode step")
    ap.add_argument("--large-untimed", type=int, default=5,
                    help="untimed steps of the large step before its timed steps")
    ap.add_argument("--large-fp64-steps", type=int, default=1,
                    help="timed steps of the FP64 form of the large step")
    ap.add_argument("--large-ncell", type=int, default=635,
                    help="FCC cells per edge of the large step (N = 4 ncell^3)")
    ap.add_argument("--profile-cell", action="store_true",
                    help="profiling case in cell mode (forces from the stencil, no list)")
    ap.add_argument("--block-z", type=int, default=0,
                    help="block shape of the 16M handle (0 = autotuned at creation)")
    ap.add_argument("--profile-phases", type=int, default=0,
                    help="profiling case: equilibrate, rebuild, K phase-by-phase steps, exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
