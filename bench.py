"""Throughput benchmark: particle-steps/s of the full PIC-MCC step on one GB300.

One step = push + gather + walls + MCC + births + sort + deposit + circuit +
Poisson for every particle (the whole hot path).  Default workload: the
256 x 256 cell, 5 cm x 5 cm RZ discharge with the external circuit (V_s =
500 V, R_ext = 200 Ohm), FP64, EC-PIC, loaded with the synthetic developed
("grown") state of 4e7 macroparticles per species (uniform 1e15 m^-3 floor
plus a 1e16 m^-3 Gaussian racetrack ring near the cathode).

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica of the workload on its own GPU (the discharge does not
shard; replicas only), barrier + max-over-ranks timing, value = all ranks'
particle-steps / that time.

--impl reference times the CPU oracle (the plain FP64 C implementation the
GPU path is checked against) on the host cores, on a bounded sample of the
same workload.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pic_inputs  # noqa: E402

METRIC = "particle-steps/s (push+gather+deposit+MCC+Poisson), 1 GB300, vs plain FP64"
UNIT = "particle-steps/s"

# Algorithmic FP64 floating-point operations of one particle-step of the push
# kernel (gather + Boris + move + frame rotation + cell location + deposit
# weights), counted from the formulas (add/mul = 1, fma = 2, div/sqrt = 1);
# the derivation is listed with the design notes.
# kernels of one step of one discharge: field tables, queue set-up, push,
# births (sort, rank, commit), scan, scatter, charge, circuit, Poisson, step end,
# and the births append when full sorts are periodic; plus, once per pic_step
# call, the live-count kernel of the push's re-tuning check.  An ensemble step
# launches the same kernels once each over all its discharges.
KERNELS_PER_STEP = 12
KERNELS_PER_CALL = 1
# full cell sort period of the default runs (256 x 256, 4e7 per species,
# measured over 128 timed steps: FP64 7.84e9 / 7.92e9 / 7.95e9 particle-steps/s
# at 16 / 32 / 64; FP32 2.85e10 / 2.99e10 / 3.13e10 at 8 / 16 / 32)
SORT_EVERY_DEFAULT = {"fp64": 32, "fp32": 32}
FLOPS_PER_PARTICLE = {0: 69.0, 1: 77.0}   # EC, MC (h E and h B from per-species tables; positions in cell units)
# Algorithmic HBM bytes of one particle-step: read and write r, z, v_r,
# v_theta, v_z, id once (FP64).
BYTES_PER_PARTICLE = 96.0
# FP32 mode: read and write the two 16-byte records of a particle once.
BYTES_PER_PARTICLE_FP32 = 64.0
# DRAM traffic of one push launch per particle pushed, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on this workload at 1e7 per
# species, scaled by the particles of a launch (one pass over each particle)
# (profiles/traffic_push_one_rz256_ring_1e7.md); None until measured on the
# kernel as it stands.
TRAFFIC_PER_PARTICLE = {"fp64": 87.8, "fp32": 62.9}
# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA pipes-lanes per SM per clock x 2
# flop x 2.07 GHz = 1.26 TFLOP/s (nominal 1.25); scaled to the measured clock.
FP64_FLOP_PER_CLK = 152 * 2 * 2
# steps a new handle spends tuning the push (chunk size, then cell tile shape)
AUTOTUNE_STEPS = 6
TILE_NAMES = {1: "8x8", 2: "16x8", 3: "8x16"}   # cells, r x z (pic_tuned_tile)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n-per-species", type=float, default=4e7)
    ap.add_argument("--gather", default="ec", choices=["ec", "mc"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="particle arithmetic: fp64 (plain method) or fp32 (precision mode)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=float, default=8e6,
                    help="oracle sample size per species for the CPU baseline")
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--cpu-sample-per-core", type=float, default=2e6,
                    help="particles per species of each oracle process of the all-cores "
                         "CPU baseline (and of the reference arm)")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes of the all-cores CPU baseline (0: one per core "
                         "this process may run on)")
    ap.add_argument("--cpu-cores-steps", type=int, default=8,
                    help="timed oracle steps per process of the all-cores CPU baseline")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="only the headline FP64 line: skip the FP32, ensemble and learned "
                         "warm-start sub-records")
    ap.add_argument("--workload", default="rz256",
                    choices=["rz256", "sweep16", "learned", "combined", "unet", "precision"],
                    help="rz256: one 256x256 discharge; sweep16: the 16-discharge "
                         "SEY x R_ext ensemble on 128x128 grids; learned: the 256x512 "
                         "discharge with and without the learned Poisson warm start; "
                         "combined: the sweep as one FP32 ensemble with the learned warm "
                         "start; unet: the warm-start network alone on the 257x513 node grid")
    ap.add_argument("--phi-extrapolate", type=int, default=1, choices=(0, 1),
                    help="1: each step's Poisson solve starts from 2 phi^(n-1) - phi^(n-2) "
                         "(phi still solved to poisson_tol); 0: from phi^(n-1)")
    ap.add_argument("--sort-every", type=int, default=None,
                    help="full cell sort every this many steps (births appended in place "
                         "between; results do not depend on it); default 32 for both "
                         "precisions (the fastest measured)")
    ap.add_argument("--geometry", default="rz256", choices=["rz256", "paper"],
                    help="rz256 workload's chamber: rz256 = 5 x 5 cm, cathode disk r <= 2 cm, "
                         "other walls grounded; paper = the 3 x 3 cm chamber of Section 3 "
                         "(cathode to 0.85 L_r, insulating block on the rest of z = 0, "
                         "10 mTorr), same 256 x 256 grid and particle count")
    ap.add_argument("--unet-mode", type=int, default=1, choices=[0, 1],
                    help="learned: 0 = network maps (rho, r, V) to phi; 1 = network maps the "
                         "previous solution's residual to the change of phi")
    ap.add_argument("--snapshots", type=int, default=512,
                    help="learned: recorded steps (one snapshot per step)")
    ap.add_argument("--combined-snapshots", type=int, default=1024,
                    help="combined: snapshots recorded over the 16 discharges (16 per step)")
    ap.add_argument("--train-iters", type=int, default=1000)
    ap.add_argument("--train-batch", type=int, default=8)
    ap.add_argument("--energy-steps", type=int, default=100000,
                    help="precision: steps of the closed-system energy runs")
    ap.add_argument("--steady-steps", type=int, default=20000,
                    help="precision: steps of the FP64 / FP32 discharge comparison")
    args = ap.parse_args()
    if args.sort_every is None:
        args.sort_every = SORT_EVERY_DEFAULT[args.precision]
    return args


def workload(args):
    g = 0 if args.gather == "ec" else 1
    if args.geometry == "paper":
        p = pic_inputs.params_paper(gather=g, seed=args.seed, cells=256)
    else:
        p = pic_inputs.params_rz256(gather=g, seed=args.seed)
    n = int(args.n_per_species)
    p, parts = pic_inputs.grown_ring_state(p, n, seed=args.seed)
    p = pic_inputs.with_capacity(p, parts, factor=1.25, births=1 << 20)
    p["diag_every"] = 10      # diagnostics reduction every 10 steps
    p["precision"] = 1 if args.precision == "fp32" else 0
    p["sort_every"] = args.sort_every
    p["phi_extrapolate"] = args.phi_extrapolate
    return p, parts


def config_block(p, n, args):
    name = "rz256" if args.geometry == "rz256" else "paper256_insulating_block"
    return {"workload": f"{name}_ring_{n:.0e}_per_species_{args.precision}".replace("+", ""),
            "grid": [p["nr"], p["nz"]], "domain_m": [p["R"], p["L"]],
            "n_per_species": n, "gather": args.gather.upper() + "-PIC",
            "precision": args.precision, "circuit": {"Vs": p["Vs"], "Rext": p["Rext"]},
            "dt": p["dt"], "poisson_tol": p["poisson_tol"], "diag_every": p["diag_every"],
            "sort_every": p["sort_every"],
            "poisson_start": ("2 phi^(n-1) - phi^(n-2)" if p["phi_extrapolate"]
                              else "phi^(n-1)"),
            "insulating_boundary": {"z0_outside_cathode": p["gap_neumann"],
                                    "wall_r_R": p["wall_neumann"]},
            "poisson_precond": ("multigrid V-cycle" if p["poisson_precond"] == 1 or p["gap_neumann"]
                                or p["wall_neumann"] else
                                "sine transform along z + tridiagonal solves in r (FP32)"),
            "l2": "inputs larger than L2 (particle state 3.8 GB >> 129 MB)"}


# ---------------------------------------------------------------------------
# replicas (N > 1): one independent discharge per rank
# ---------------------------------------------------------------------------
def aggregate_replicas(t: float, psteps: float, world: int, device: str):
    """Whole-job numbers of N replicas: the timed region is the slowest rank's,
    the work is the sum of all ranks' particle-steps."""
    if world <= 1:
        return t, psteps
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([t], device=device, dtype=torch.float64)
    tot = torch.tensor([float(psteps)], device=device, dtype=torch.float64)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tmax.item()), float(tot.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.tmp = tempfile.TemporaryDirectory(prefix="pic_clocks_")
        self.path = os.path.join(self.tmp.name, "clocks.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            return self._summary()
        finally:
            self.tmp.cleanup()

    def _summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch, local: int = 0) -> str:
    props = torch.cuda.get_device_properties(local)
    return f"GPU-{props.uuid}" if hasattr(props, "uuid") else str(local)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def cpu_baseline(p, parts, sample: int, steps: int, seed: int):
    import oracle
    rng = np.random.default_rng(seed + 99)
    sub = {}
    taken = 0
    for k in ("e", "i"):
        n = parts[k]["r"].shape[0]
        idx = np.sort(rng.choice(n, size=min(sample, n), replace=False))
        sub[k] = {q: parts[k][q][idx].copy() for q in parts[k]}
        taken = max(taken, idx.size)
    orc = oracle.Oracle(p, sub)           # includes the one-time Cholesky factorisation
    t0 = time.perf_counter()
    total = 0
    for _ in range(steps):
        total += orc.count(0) + orc.count(1)
        orc.step(1)
    dt = time.perf_counter() - t0
    return {"value": total / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{taken:.0e} random particles per species of the same state, "
                      f"{steps} full steps (push, MCC, deposit, banded-Cholesky Poisson on "
                      f"{p['nr'] + 1}x{p['nz'] + 1}), single-threaded C, {dt:.1f} s"}


def host_cores() -> int:
    """Cores this process may run on (the affinity mask, not the machine's count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_replica(k, p, n, steps, warm, seed, barrier, queue):
    """One process of the all-cores oracle run: its own sample of the workload
    (the same synthetic state drawn with n particles per species), `warm`
    untimed steps, then `steps` timed ones started together with the others."""
    try:
        import oracle
        p2, parts = pic_inputs.grown_ring_state(p, n, seed=seed + 1000 + k)
        orc = oracle.Oracle(p2, parts)     # includes the one-time Cholesky factorisation
        del parts
        if warm:
            orc.step(warm)
        barrier.wait(timeout=600)
        t0 = time.time()
        total = 0
        for _ in range(steps):
            total += orc.count(0) + orc.count(1)
            orc.step(1)
        queue.put((k, total, t0, time.time(), None))
    except Exception as exc:   # reported by the parent
        queue.put((k, 0, 0.0, 0.0, repr(exc)))


def cpu_baseline_all_cores(p, n: int, steps: int, warm: int, seed: int, procs: int = 0):
    """The oracle as it stands on every host core: one single-threaded oracle
    process per core, each on its own n-per-species sample of the workload,
    timed together; value = all processes' particle-steps / the common wall
    time.  Processes are spawned (not forked: the parent holds a CUDA context)."""
    import multiprocessing as mp
    from oracle import build as oracle_build
    oracle_build.build()                   # built once, before the processes load it
    procs = procs or host_cores()
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    env_keep = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    workers = [ctx.Process(target=_oracle_replica,
                           args=(k, p, n, steps, warm, seed, barrier, queue), daemon=True)
               for k in range(procs)]
    for w in workers:
        w.start()
    if env_keep is None:
        os.environ.pop("OMP_NUM_THREADS")
    else:
        os.environ["OMP_NUM_THREADS"] = env_keep
    res = [queue.get(timeout=1800) for _ in workers]
    for w in workers:
        w.join(timeout=60)
    errors = [r[4] for r in res if r[4]]
    if errors:
        raise RuntimeError(f"oracle process failed: {errors[0]}")
    total = sum(r[1] for r in res)
    t = max(r[3] for r in res) - min(r[2] for r in res)
    cpu = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    cpu = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"value": total / t, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} single-threaded oracle processes, one per core, each on its own "
                      f"{n:.0e}-per-species draw of the same synthetic state, {steps} full "
                      f"steps each (push, MCC, deposit, banded-Cholesky Poisson on "
                      f"{p['nr'] + 1}x{p['nz'] + 1}) after {warm} untimed, {t:.1f} s wall",
            "ms_per_step": t / steps * 1e3, "particles_per_step": total / steps,
            "cpu_model": cpu, "nproc": os.cpu_count()}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on every host core, on a
    bounded sample of the workload (one sample per core)."""
    if rank != 0:
        return
    g = 0 if args.gather == "ec" else 1
    p = (pic_inputs.params_paper(gather=g, seed=args.seed, cells=256) if args.geometry == "paper"
         else pic_inputs.params_rz256(gather=g, seed=args.seed))
    p.update(precision=1 if args.precision == "fp32" else 0, sort_every=args.sort_every,
             phi_extrapolate=args.phi_extrapolate, diag_every=10)
    n = int(args.cpu_sample_per_core)
    res = cpu_baseline_all_cores(p, n, max(1, args.steps), max(0, args.warmup), args.seed,
                                 args.cpu_procs)
    v = res["value"]
    cfg = config_block(p, n * res["cores"], args)
    # the workload sampled is the GPU arm's (same grid, parameters and synthetic
    # state); n_per_species states the particles actually stepped
    cfg["workload"] = config_block(p, int(args.n_per_species), args)["workload"]
    cfg["sample"] = {"processes": res["cores"], "n_per_species_per_process": n,
                     "note": "n_per_species is the total over the processes; every process "
                             "steps its own discharge (same synthetic state, own draw)"}
    cfg["l2"] = "host run"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "cpu_baseline": res,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# ensemble workload: 16 discharges (gamma x R_ext sweep), uneven loads
# ---------------------------------------------------------------------------
def sweep_workload(args):
    g = 0 if args.gather == "ec" else 1
    plist = pic_inputs.params_rz128_sweep(gather=g, seed=args.seed)
    rng = np.random.default_rng(args.seed + 5)
    sizes = [int(1e6 * 8.0 ** (k / 15.0)) for k in range(16)]
    rng.shuffle(sizes)
    out = []
    for k, p in enumerate(plist):
        p, parts = pic_inputs.grown_ring_state(p, sizes[k], seed=args.seed + 31 * k)
        p = pic_inputs.with_capacity(p, parts, factor=1.25, births=1 << 18)
        p["diag_every"] = 10
        p["precision"] = 1 if args.precision == "fp32" else 0
        p["sort_every"] = args.sort_every
        p["phi_extrapolate"] = args.phi_extrapolate
        out.append((p, parts))
    return out


def run_sweep(args, torch, pg, emit: bool = True):
    insts = sweep_workload(args)
    ntot = sum(2 * parts["e"]["r"].shape[0] for _, parts in insts)
    warm = AUTOTUNE_STEPS + args.warmup

    def load(h, k, parts):
        for key, sp in (("e", 0), ("i", 1)):
            pg.pic_set_particles(h, k, sp, parts[key])
        pg.pic_solve_fields(h, k)

    def timed(h_list, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ps0 = sum(pg.pic_diagnostics(h, k)["particle_steps"] for h, k in h_list)
        torch.cuda.synchronize()
        ev0.record()
        for h in dict.fromkeys(h for h, _ in h_list):
            pg.pic_step(h, steps)
        ev1.record()
        torch.cuda.synchronize()
        ps1 = sum(pg.pic_diagnostics(h, k)["particle_steps"] for h, k in h_list)
        return ev0.elapsed_time(ev1), ps1 - ps0

    ens = pg.pic_create([p for p, _ in insts])
    for k, (_, parts) in enumerate(insts):
        load(ens, k, parts)
    pg.pic_step(ens, warm)
    pg.pic_sync(ens)
    with ClockSampler(gpu_uuid(torch)) as clk:
        ms_e, ps_e = timed([(ens, k) for k in range(len(insts))], args.steps)
    pg.pic_profile(ens, True)
    pg.pic_step(ens, min(args.steps, 5))
    prof = pg.pic_profile_read(ens)
    pg.pic_profile(ens, False)
    nprof = max(1, prof["push"]["launches"])
    tuned, tile = pg.pic_tuned_chunk(ens), pg.pic_tuned_tile(ens)
    graph = pg.pic_uses_graph(ens)
    pg.pic_destroy(ens)
    # the same 16 discharges as 16 sequential single-discharge runs
    singles = []
    for p, parts in insts:
        h = pg.pic_create(p)
        load(h, 0, parts)
        pg.pic_step(h, AUTOTUNE_STEPS + args.warmup)
        singles.append(h)
    pg.pic_sync(singles[0])
    ms_s, ps_s = timed([(h, 0) for h in singles], args.steps)
    # Poisson time of the 16 sequential runs per step of all 16
    seq_poisson = 0.0
    for h in singles:
        pg.pic_profile(h, True)
        pg.pic_step(h, min(args.steps, 5))
        pr = pg.pic_profile_read(h)
        pg.pic_profile(h, False)
        seq_poisson += pr["poisson"]["total_ms"] / max(1, pr["push"]["launches"])
    for h in singles:
        pg.pic_destroy(h)
    value = ps_e / (ms_e / 1e3)
    seq = ps_s / (ms_s / 1e3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": warm, "ms_per_step": ms_e / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": f"sweep16_rz128_{args.precision}", "sort_every": args.sort_every,
                       "instances": len(insts), "grid": [128, 128], "domain_m": [0.05, 0.05],
                       "particles_per_species": [parts["e"]["r"].shape[0] for _, parts in insts],
                       "total_particles": ntot,
                       "gamma_x_Rext": [[p["gamma_i"], p["Rext"]] for p, _ in insts],
                       "l2": "inputs larger than L2"},
            "clocks": clk.summary(),
            "sequential_16_value": seq, "ensemble_over_sequential": value / seq,
            "sequential_16_poisson_ms_per_step": seq_poisson,
            "autotuned_particles_per_thread": tuned, "autotuned_cell_tile": TILE_NAMES[tile],
            "cuda_graph": graph,
            "per_kernel_ms_per_step": {k: v["total_ms"] / nprof for k, v in prof.items()}}
    if emit:
        print(json.dumps(line), flush=True)
    return line


# ---------------------------------------------------------------------------
# learned warm start workload: 256 x 512 cells, 10 cm long, 5e7 per species
# ---------------------------------------------------------------------------
def run_learned(args, torch, pg, emit: bool = True):
    g = 0 if args.gather == "ec" else 1
    n = int(args.n_per_species) if args.n_per_species != 4e7 else int(5e7)
    p = pic_inputs.params_rz256x512(gather=g, seed=args.seed)
    p, parts = pic_inputs.grown_ring_state(p, n, seed=args.seed)
    p = pic_inputs.with_capacity(p, parts, factor=1.25, births=1 << 20)
    p["diag_every"] = 10
    p["precision"] = 1 if args.precision == "fp32" else 0
    p["sort_every"] = args.sort_every
    # the network proposes starts for the multigrid-preconditioned solve (the
    # sine-transform preconditioner reaches the tolerance in two iterations
    # from any start)
    p["poisson_precond"] = 1
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    del parts
    pg.pic_solve_fields(h, 0)
    pg.pic_unet_create(h, args.seed + 1, args.train_batch, args.unet_mode)
    # training data: one snapshot per step of the run itself
    pg.pic_unet_snapshots(h, args.snapshots, 1)
    t0 = time.perf_counter()
    pg.pic_step(h, args.snapshots)
    pg.pic_sync(h)
    t_rec = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss0, loss1 = pg.pic_unet_train(h, args.train_iters, args.train_batch, 2e-3, args.seed + 7)
    t_train = time.perf_counter() - t0
    pg.pic_unet_record(h, False)   # both arms below without the recording

    def measure(on: bool):
        pg.pic_unet_warm_start(h, on)
        pg.pic_step(h, args.warmup)
        pg.pic_sync(h)
        s0, d0 = pg.pic_unet_stats(h), pg.pic_diagnostics(h, 0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(gpu_uuid(torch)) as clk:
            ev0.record()
            pg.pic_step(h, args.steps)
            ev1.record()
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        s1, d1 = pg.pic_unet_stats(h), pg.pic_diagnostics(h, 0)
        pg.pic_profile(h, True)
        pg.pic_step(h, 10)
        prof = pg.pic_profile_read(h)
        pg.pic_profile(h, False)
        nprof = max(1, prof["push"]["launches"])
        return {"value": (d1["particle_steps"] - d0["particle_steps"]) / (ms / 1e3),
                "ms_per_step": ms / args.steps,
                "poisson_iters_per_step": (s1["poisson_iters"] - s0["poisson_iters"]) / args.steps,
                "starts": {k: s1[k] - s0[k] for k in ("starts_previous", "starts_network",
                                                       "starts_zero")},
                "poisson_ms_per_step": prof["poisson"]["total_ms"] / nprof,
                "warm_start_ms_per_step": prof["warm_start"]["total_ms"] / nprof,
                "cuda_graph": pg.pic_uses_graph(h), "clocks": clk.summary()}

    plain = measure(False)
    warm = measure(True)

    # cold starts (no previous solution: phi set to zero before the step), the
    # case the network is for; consecutive steps alternate plain / warm
    nodes = np.zeros((p["nr"] + 1, p["nz"] + 1))
    cold = {"plain_iters": [], "warm_iters": [], "warm_starts_network": 0}
    for _ in range(3):
        for on in (False, True):
            pg.pic_unet_warm_start(h, on)
            pg.pic_set_phi(h, 0, nodes)
            s0 = pg.pic_unet_stats(h)
            pg.pic_step(h, 1)
            s1 = pg.pic_unet_stats(h)
            cold["warm_iters" if on else "plain_iters"].append(s1["poisson_iters"] - s0["poisson_iters"])
            if on:
                cold["warm_starts_network"] += s1["starts_network"] - s0["starts_network"]
    line = {"metric": METRIC, "value": warm["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": warm["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": f"learned_rz256x512_{n:.0e}_per_species_mode{args.unet_mode}_"
                                   f"{args.precision}".replace("+", ""),
                       "grid": [p["nr"], p["nz"]], "domain_m": [p["R"], p["L"]],
                       "n_per_species": n, "unet_mode": args.unet_mode,
                       "snapshots": args.snapshots, "train_iters": args.train_iters,
                       "poisson_precond": "multigrid V-cycle (both arms)",
                       "train_batch": args.train_batch, "poisson_tol": p["poisson_tol"],
                       "sort_every": p["sort_every"],
                       "l2": "inputs larger than L2"},
            "plain": plain, "warm": warm, "cold_start": cold,
            "training": {"loss_first": loss0, "loss_last": loss1, "seconds": t_train,
                         "record_seconds": t_rec, "stats": pg.pic_unet_stats(h)}}
    if emit:
        print(json.dumps(line), flush=True)
    pg.pic_destroy(h)
    return line


# ---------------------------------------------------------------------------
# the three forms together: the 16-discharge sweep as one FP32 ensemble whose
# Poisson solves start from the learned warm start (one network for all 16,
# trained on the ensemble's own recorded steps), against the plain FP64 form
# (the same 16 discharges run one after the other, default solver)
# ---------------------------------------------------------------------------
def run_combined(args, torch, pg, emit: bool = True, plain_fp64=None):
    a = argparse.Namespace(**vars(args))
    a.precision, a.sort_every = "fp32", SORT_EVERY_DEFAULT["fp32"]
    insts = sweep_workload(a)
    for p, _ in insts:
        # the network proposes starts for the multigrid-preconditioned solve
        p["poisson_precond"] = 1
    n_inst = len(insts)
    h = pg.pic_create([p for p, _ in insts])
    for k, (_, parts) in enumerate(insts):
        for key, sp in (("e", 0), ("i", 1)):
            pg.pic_set_particles(h, k, sp, parts[key])
        pg.pic_solve_fields(h, k)
    del insts[:]
    pg.pic_unet_create(h, args.seed + 1, args.train_batch, 1)
    record = max(1, args.combined_snapshots // n_inst)
    pg.pic_unet_snapshots(h, record * n_inst, 1)
    t0 = time.perf_counter()
    pg.pic_step(h, record)
    pg.pic_sync(h)
    t_rec = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss0, loss1 = pg.pic_unet_train(h, args.train_iters, args.train_batch, 2e-3, args.seed + 7)
    t_train = time.perf_counter() - t0
    pg.pic_unet_record(h, False)   # both arms below without the recording

    def psteps():
        return sum(pg.pic_diagnostics(h, k)["particle_steps"] for k in range(n_inst))

    def measure(on: bool):
        pg.pic_unet_warm_start(h, on)
        pg.pic_step(h, args.warmup)
        pg.pic_sync(h)
        s0, p0 = pg.pic_unet_stats(h), psteps()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(gpu_uuid(torch)) as clk:
            ev0.record()
            pg.pic_step(h, args.steps)
            ev1.record()
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        s1, p1 = pg.pic_unet_stats(h), psteps()
        pg.pic_profile(h, True)
        pg.pic_step(h, 5)
        prof = pg.pic_profile_read(h)
        pg.pic_profile(h, False)
        nprof = max(1, prof["push"]["launches"])
        return {"value": (p1 - p0) / (ms / 1e3), "ms_per_step": ms / args.steps,
                "poisson_iters_per_instance_step":
                    (s1["poisson_iters"] - s0["poisson_iters"]) / (args.steps * n_inst),
                "starts": {k: s1[k] - s0[k] for k in ("starts_previous", "starts_network",
                                                       "starts_zero")},
                "poisson_ms_per_step": prof["poisson"]["total_ms"] / nprof,
                "warm_start_ms_per_step": prof["warm_start"]["total_ms"] / nprof,
                "cuda_graph": pg.pic_uses_graph(h), "clocks": clk.summary()}

    without = measure(False)
    warm = measure(True)
    line = {"metric": METRIC, "value": warm["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": warm["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sweep16_rz128_fp32_learned_mode1", "instances": n_inst,
                       "grid": [128, 128], "sort_every": a.sort_every,
                       "poisson_precond": "multigrid V-cycle",
                       "snapshots": record * n_inst, "train_iters": args.train_iters,
                       "train_batch": args.train_batch, "l2": "inputs larger than L2"},
            "warm": warm, "without_warm_start": without,
            "training": {"loss_first": loss0, "loss_last": loss1, "seconds": t_train,
                         "record_seconds": t_rec}}
    if plain_fp64 and "sequential_16_value" in plain_fp64:
        seq, seq_p = plain_fp64["sequential_16_value"], plain_fp64.get("sequential_16_poisson_ms_per_step")
        line["plain_fp64"] = {"value": seq, "poisson_ms_per_step": seq_p,
                              "form": "the 16 discharges as 16 sequential FP64 single-discharge "
                                      "runs (sine-transform preconditioner, extrapolated start)"}
        line["over_plain_fp64"] = warm["value"] / seq
        if seq_p:
            line["poisson_time_over_plain_fp64"] = warm["poisson_ms_per_step"] / seq_p
    if emit:
        print(json.dumps(line), flush=True)
    pg.pic_destroy(h)
    return line


# ---------------------------------------------------------------------------
# the warm-start network alone: forward (batch 1) and training pass (batch 8)
# on the 257 x 513 node grid, through the C ABI (host inputs)
# ---------------------------------------------------------------------------
def run_unet(args, torch, pg):
    p = pic_inputs.params_rz256x512(seed=args.seed)
    p.update(cap_e=4096, cap_i=4096, birth_cap=1024)
    h = pg.pic_create(p)
    pg.pic_unet_create(h, args.seed + 1, 8, args.unet_mode)
    H, W = p["nr"] + 1, p["nz"] + 1
    rng = np.random.default_rng(args.seed)
    x = rng.normal(size=(8, 3, H, W)).astype(np.float32)
    y = rng.normal(size=(8, H, W)).astype(np.float32)
    out = {}
    for name, B, yy in (("forward_b1", 1, None), ("forward_backward_b8", 8, y)):
        for _ in range(args.warmup):
            pg.pic_unet_loss_grad(h, x[:B], None if yy is None else yy[:B])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pg.pic_unet_loss_grad(h, x[:B], None if yy is None else yy[:B])
        torch.cuda.synchronize()
        out[name + "_ms"] = (time.perf_counter() - t0) / args.steps * 1e3
    gflop_fwd = 0.0
    C = (16, 32, 64, 64)
    for l in range(4):
        n = ((p["nr"] >> l) + 1) * ((p["nz"] >> l) + 1)
        cin_a = 16 if l == 0 else C[l - 1]
        gflop_fwd += 2 * 9 * n * (cin_a * C[l] + C[l] * C[l]) / 1e9
        if l < 3:
            gflop_fwd += 2 * 9 * n * ((C[l + 1] + C[l]) * C[l] + C[l] * C[l]) / 1e9
    line = {"metric": "U-Net forward time, 257x513 nodes, batch 1 (through the C ABI)",
            "value": out["forward_b1_ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "dtype": "bf16",
            "data": "synthetic", "config": {"workload": "unet_257x513", "mode": args.unet_mode,
                                            "params": pg.pic_unet_param_count()},
            "forward_backward_b8_ms": out["forward_backward_b8_ms"],
            "forward_gflop": gflop_fwd,
            "note": "host-to-device copy of the inputs and device-to-host copy of the output "
                    "are inside each timed call"}
    print(json.dumps(line), flush=True)
    pg.pic_destroy(h)


# ---------------------------------------------------------------------------
# precision mode on the 32 x 32 discharge: energy drift of a closed system and
# time-averaged diagnostics of the discharge, FP32 against FP64
# ---------------------------------------------------------------------------
def _run_series(pg, p, parts, steps, every):
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    out = []
    for _ in range(steps // every):
        pg.pic_step(h, every)
        out.append(pg.pic_diagnostics(h, 0))
    pg.pic_destroy(h)
    return out


def run_precision(args, torch, pg):
    res = {"energy": {}, "steady": {}}
    t0 = time.perf_counter()
    # closed system: no collisions, reflecting walls, all electrodes at 0 V
    for gname, g in (("EC", 0), ("MC", 1)):
        for prec in ("fp64", "fp32"):
            p = pic_inputs.params_rz32(gather=g, precision=1 if prec == "fp32" else 0, seed=args.seed)
            p.update(mcc_on=0, walls_reflect=1, circuit_mode=0, Vc_fixed=0.0, diag_every=100)
            p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 64, n0=1e15, seed=args.seed + 1)
            p = pic_inputs.with_capacity(p, parts, factor=1.1)
            ser = _run_series(pg, p, parts, args.energy_steps, 100)
            tot = np.array([d["W_field"] + d["K_e"] + d["K_i"] for d in ser])
            rel = tot / tot[0] - 1.0
            res["energy"][f"{gname}_{prec}"] = {
                "steps": args.energy_steps, "rel_change_end": float(rel[-1]),
                "max_abs_rel_change": float(np.abs(rel).max()),
                "rel_change_per_1e5_steps": float(rel[-1] * 1e5 / args.energy_steps)}
    # the cfg-1 discharge: -400 V cathode, collisions, secondary emission
    keys = ("I_cath", "n_e_peak", "n_i_peak", "W_field", "K_e", "K_i", "N_e", "N_i")
    means = {}
    for prec in ("fp64", "fp32"):
        acc = {k: [] for k in keys}
        for seed in (args.seed, args.seed + 1):
            p = pic_inputs.params_rz32(gather=0, precision=1 if prec == "fp32" else 0, seed=seed)
            p.update(diag_every=50)
            p, parts = pic_inputs.seed_plasma(p, 32 * 32 * 64, n0=1e15, seed=seed + 10)
            p = pic_inputs.with_capacity(p, parts, factor=4.0, births=1 << 16)
            ser = _run_series(pg, p, parts, args.steady_steps, 50)
            tail = ser[len(ser) // 2:]
            for k in keys:
                acc[k].append(float(np.mean([d[k] for d in tail])))
        means[prec] = {k: float(np.mean(v)) for k, v in acc.items()}
        res["steady"][prec] = {"per_seed": acc}
    res["steady"]["fp32_vs_fp64_rel_diff"] = {
        k: (means["fp32"][k] - means["fp64"][k]) / abs(means["fp64"][k]) if means["fp64"][k] else 0.0
        for k in keys}
    res["steady"]["seed_spread_fp64_rel"] = {
        k: (abs(res["steady"]["fp64"]["per_seed"][k][0] - res["steady"]["fp64"]["per_seed"][k][1]) /
            abs(means["fp64"][k]) if means["fp64"][k] else 0.0) for k in keys}
    line = {"metric": "precision mode on the 32x32 discharge (FP32 vs FP64)", "value": None,
            "unit": None, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "rz32_precision", "energy_steps": args.energy_steps,
                       "steady_steps": args.steady_steps, "steady_average": "second half, every 50 steps",
                       "seeds": [args.seed, args.seed + 1]},
            "seconds": time.perf_counter() - t0, **res}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# one discharge: create, load, tune, warm up, time K steps, per-kernel times
# ---------------------------------------------------------------------------
def timed_discharge(pg, torch, p, parts, args, local=0, world=1, barrier=lambda: None):
    """Time args.steps steps of one discharge (CUDA events on the handle's
    stream, graph replay), after the autotuner's steps and args.warmup warm-up
    steps; then per-kernel CUDA-event times over a second pass of the same
    step.  Returns the handle and a record."""
    h = pg.pic_create(p)
    for k, sp in (("e", 0), ("i", 1)):
        pg.pic_set_particles(h, 0, sp, parts[k])
    pg.pic_solve_fields(h, 0)
    # the first 4 steps of a handle tune the push's chunk size (eager, untimed)
    pg.pic_step(h, AUTOTUNE_STEPS)
    pg.pic_step(h, args.warmup)
    pg.pic_sync(h)
    d0 = pg.pic_diagnostics(h, 0)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(gpu_uuid(torch, local)) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        pg.pic_step(h, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = ev0.elapsed_time(ev1)
    d1 = pg.pic_diagnostics(h, 0)
    pg.pic_profile(h, True)
    pg.pic_step(h, min(args.steps, 10))
    prof = pg.pic_profile_read(h)
    pg.pic_profile(h, False)
    prof_steps = max(1, prof["push"]["launches"])
    per_kernel = {k: v["total_ms"] / prof_steps for k, v in prof.items()}
    return h, {"ms": ms, "psteps": d1["particle_steps"] - d0["particle_steps"], "d1": d1,
               "per_kernel": per_kernel, "clocks": clk.summary()}


def push_roofline(precision, gather, rec, n_pushed, peaks, peak_kind):
    """Roofline of the dominant kernel, the push of both species (one launch per
    step): algorithmic HBM bytes per particle-step (read and write the particle
    state once: 96 B FP64, 64 B FP32) x particles / its CUDA-event time against
    the measured copy bandwidth; for FP64 also the FP64-pipe view (algorithmic
    flops against 152 SMs x 4 flop/clk at the loaded clock), where that kernel
    is bound."""
    push_ms = rec["per_kernel"]["push"]
    bpp = BYTES_PER_PARTICLE if precision == "fp64" else BYTES_PER_PARTICLE_FP32
    hbm = peaks.get("hbm_gbs", 6800.0)
    bw = bpp * n_pushed / (push_ms / 1e3) / 1e9
    line = {"bound": "hbm", "kernel": ("k_push_one" if precision == "fp64" else "k_push32_one")
            + " (both species)", "achieved": bw, "peak": hbm, "unit": "GB/s",
            "frac": bw / hbm, "traffic": (TRAFFIC_PER_PARTICLE[precision] * n_pushed
                                          if TRAFFIC_PER_PARTICLE[precision] else None),
            "peak_kind": peak_kind, "bytes_per_particle": bpp, "particles_per_launch": n_pushed,
            "push_ms": push_ms, "per_kernel_ms_per_step": rec["per_kernel"]}
    if precision == "fp64":
        sm_mhz = rec["clocks"].get("sm_mhz") or 2070.0
        derived = FP64_FLOP_PER_CLK * sm_mhz * 1e6 / 1e12
        fl = FLOPS_PER_PARTICLE[gather] * n_pushed / (push_ms / 1e3) / 1e12
        measured = peaks.get("fp64_fma_tflops")
        fp64_peak = measured if measured else derived
        line["alu_view"] = {"bound": "alu", "achieved": fl, "peak": fp64_peak, "unit": "TFLOP/s",
                            "frac": fl / fp64_peak, "flops_per_particle": FLOPS_PER_PARTICLE[gather],
                            "peak_kind": "measured" if measured else "derived",
                            "peak_note": ("FP64 FMA throughput measured on this GPU by "
                                          "pic_fp64_fma_rate (independent FMA chains on every SM)"
                                          if measured else "FP64 pipes: 152 SMs x 4 flop/clk"),
                            "derived_peak": derived,
                            "derived_note": f"152 SMs x 4 flop/clk at the median loaded SM clock "
                                            f"{sm_mhz:.0f} MHz"}
    return line


def end_to_end(pg, torch, p, parts, args):
    """The metric through the C ABI with host buffers: upload of the state from
    pinned host memory, the field solve, then every step pic_step and a
    diagnostics read-back."""
    import ctypes
    pinned = {k: {q: torch.from_numpy(a).pin_memory() for q, a in parts[k].items()}
              for k in ("e", "i")}
    state_bytes = sum(v.numel() * v.element_size() for k in pinned for v in pinned[k].values())
    h2 = pg.pic_create(p)
    torch.cuda.synchronize()
    lib = pg.load_library()
    t0 = time.perf_counter()
    for k, sp in (("e", 0), ("i", 1)):
        a = pinned[k]
        rc = lib.pic_set_particles(h2.ptr, 0, sp, a["r"].numel(), a["r"].data_ptr(),
                                   a["z"].data_ptr(), a["vr"].data_ptr(), a["vt"].data_ptr(),
                                   a["vz"].data_ptr(), a["id"].data_ptr(), 0)
        assert rc == 0, rc
    pg.pic_solve_fields(h2, 0)
    ps0 = pg.pic_diagnostics(h2, 0)["particle_steps"]
    de = None
    for _ in range(args.steps):
        pg.pic_step(h2, 1)
        de = pg.pic_diagnostics(h2, 0)
    t_e2e = time.perf_counter() - t0
    pg.pic_destroy(h2)
    return {"value": (de["particle_steps"] - ps0) / t_e2e, "unit": UNIT,
            "h2d_bytes_per_step": state_bytes / args.steps,
            "d2h_bytes_per_step": float(ctypes.sizeof(pg.PicDiag)),
            "note": "whole job through the C ABI: state upload from pinned host buffers "
                    "(amortised over the steps), field solve, then per step pic_step + "
                    "pic_diagnostics read-back"}


def sub_records(args, torch, pg, p, parts, peaks, peak_kind, local, fp64_value):
    """The other forms, each timed on its own: the FP32 particle mode on the
    same workload and state, the 16-discharge ensemble against 16 sequential
    runs (both precisions), the learned Poisson warm start against the plain
    solver on the 256 x 512 workload, and the three together (FP32 ensemble
    with the learned warm start) against the plain FP64 form."""
    out = {}
    g = 0 if args.gather == "ec" else 1
    try:
        p32 = dict(p, precision=1, sort_every=SORT_EVERY_DEFAULT["fp32"])
        h, rec = timed_discharge(pg, torch, p32, parts, args, local)
        n_pushed = pg.pic_count(h, 0, 0) + pg.pic_count(h, 0, 1)
        out["fp32"] = {"value": rec["psteps"] / (rec["ms"] / 1e3), "unit": UNIT,
                       "ms_per_step": rec["ms"] / args.steps, "over_fp64": None,
                       "config": {"workload": f"rz256_ring_{int(args.n_per_species):.0e}_per_species_"
                                              "fp32".replace("+", ""),
                                  "sort_every": p32["sort_every"], "same_state_as_headline": True},
                       "push_particles_per_thread": pg.pic_tuned_chunk(h),
                       "cell_tile": TILE_NAMES[pg.pic_tuned_tile(h)],
                       "poisson": {"iters_last_step": rec["d1"]["poisson_iters"],
                                   "ms_per_step": rec["per_kernel"]["poisson"]},
                       "roofline": push_roofline("fp32", g, rec, n_pushed, peaks, peak_kind),
                       "clocks": rec["clocks"]}
        out["fp32"]["over_fp64"] = out["fp32"]["value"] / fp64_value
        pg.pic_destroy(h)
    except Exception as exc:   # a failed sub-record is reported, the headline stands
        out["fp32"] = {"error": repr(exc)}
    for prec in ("fp32", "fp64"):
        try:
            a = argparse.Namespace(**vars(args))
            a.precision, a.sort_every = prec, SORT_EVERY_DEFAULT[prec]
            out[f"sweep16_{prec}"] = run_sweep(a, torch, pg, emit=False)
        except Exception as exc:
            out[f"sweep16_{prec}"] = {"error": repr(exc)}
    try:
        a = argparse.Namespace(**vars(args))
        a.n_per_species = 5e7
        out["learned"] = run_learned(a, torch, pg, emit=False)
    except Exception as exc:
        out["learned"] = {"error": repr(exc)}
    try:
        out["combined"] = run_combined(args, torch, pg, emit=False,
                                       plain_fp64=out.get("sweep16_fp64"))
    except Exception as exc:
        out["combined"] = {"error": repr(exc)}
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    barrier()
    import paper_2507_10727_gb300 as pg

    # a side stream: pic_step captures one step into a CUDA graph and replays it
    side = torch.cuda.Stream()
    torch.cuda.set_stream(side)
    if args.workload == "sweep16":
        return run_sweep(args, torch, pg)
    if args.workload == "learned":
        return run_learned(args, torch, pg)
    if args.workload == "combined":
        return run_combined(args, torch, pg)
    if args.workload == "unet":
        return run_unet(args, torch, pg)
    if args.workload == "precision":
        return run_precision(args, torch, pg)

    p, parts = workload(args)
    n = int(args.n_per_species)
    peaks, peak_kind = measured_peaks()
    h, rec = timed_discharge(pg, torch, p, parts, args, local, world, barrier)
    t, psteps = aggregate_replicas(rec["ms"] / 1e3, rec["psteps"], world, "cuda")
    value = psteps / t
    ne, ni = pg.pic_count(h, 0, 0), pg.pic_count(h, 0, 1)
    g = 0 if args.gather == "ec" else 1
    if args.precision == "fp64":   # the FP64 push's ALU view (the FP32 push has none)
        try:
            peaks = dict(peaks, fp64_fma_tflops=pg.pic_fp64_fma_rate())
        except Exception:   # the derived FP64 peak stands in
            pass
    roofline = push_roofline(args.precision, g, rec, ne + ni, peaks, peak_kind)

    # region diagnostics sampler (Sections 4, 5): one warp per cell bin of the
    # sorted arrays; algorithmic bytes = the electron velocities (24 B FP64,
    # the 32 B FP32 record) + the bin ends and the per-cell accumulators
    stream = torch.cuda.current_stream()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pg.pic_region_sample(h, 0)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(5):
        pg.pic_region_sample(h, 0)
    r1.record(stream)
    torch.cuda.synchronize()
    reg_ms = r0.elapsed_time(r1) / 5
    ncell = p["nr"] * p["nz"]
    reg_bytes = ((24.0 if args.precision == "fp64" else 32.0) * ne
                 + 2 * 4.0 * ncell + 2 * (2 * 8.0 + 2 * 32.0) * ncell
                 + 2 * 8.0 * (p["nr"] + 1) * (p["nz"] + 1))
    regions_out = pg.pic_region_read(h, 0)
    region = {"ms_per_sample": reg_ms, "achieved_gbs": reg_bytes / (reg_ms / 1e3) / 1e9,
              "bytes_per_sample": reg_bytes, "Te_eV": regions_out["Te"],
              "z_sheath_m": regions_out["z_sheath"], "z_bulk_m": regions_out["z_bulk"]}
    graph, tuned, tile = pg.pic_uses_graph(h), pg.pic_tuned_chunk(h), pg.pic_tuned_tile(h)
    pg.pic_destroy(h)

    # end to end through the C ABI with host buffers: upload the state from
    # pinned host memory, then each step pic_step + a diagnostics read-back
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(pg, torch, p, parts, args)

    subs = {}
    cpu = None
    if rank == 0 and world == 1:
        if not args.no_subrecords:
            subs = sub_records(args, torch, pg, p, parts, peaks, peak_kind, local, value)
        del parts
        if not args.no_cpu_baseline:
            cpu = cpu_baseline_all_cores(p, int(args.cpu_sample_per_core), args.cpu_cores_steps,
                                         1, args.seed, args.cpu_procs)
            p1, parts1 = workload(args)
            cpu["single_thread"] = cpu_baseline(p1, parts1, int(args.cpu_sample), args.cpu_steps,
                                                args.seed)
            del parts1

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": rec["ms"] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic", "config": config_block(p, n, args),
                "gpu_launches": args.steps * (KERNELS_PER_STEP + (1 if args.sort_every > 1 else 0))
                                + KERNELS_PER_CALL,
                "cuda_graph": graph,
                "autotune_steps": AUTOTUNE_STEPS, "push_particles_per_thread": tuned,
                "cell_tile": TILE_NAMES[tile],
                "poisson": {"iters_last_step": rec["d1"]["poisson_iters"],
                            "resid_last_step": rec["d1"]["poisson_resid"],
                            "ms_per_step": rec["per_kernel"]["poisson"]},
                "roofline": roofline, "clocks": rec["clocks"], "e2e": e2e, "cpu_baseline": cpu,
                "region_diagnostics": region, **subs}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
