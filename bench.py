#!/usr/bin/env python3
"""Benchmark: solid-substep particle-updates/s of the multi-time-step SPH scheme.

Headline workload: the 3D membrane-flexure plate (20 x 5 x 0.2 mm at
dx = 0.02 mm, 1000 x 250 x 10 = 2,500,000 particles, Wendland C2 h = 1.3 dx,
St Venant-Kirchhoff E = 200 MPa, nu = 0.4, concentration diffusion
D = 1e-10 m^2/s with swelling beta = 0.1, top two layers held at c = 1 and
bottom two at c = 0, x = 0 end clamped, eta = 1e4), mixed precision (FP32
per-particle arithmetic, FP64 displacement and reductions).  One benchmark
step = one slow step (Sec. 4.2): the diffusion step of the stable size, then
damped substeps until the kinetic-energy criterion holds (tested once the
kinetic energy has passed its peak).  Inputs are synthetic (seeded lattice +
1 % jitter); the working set (~3 GB) is far larger than L2, so no flush is
needed between steps.

Other legs of the same line: the 3D J2 cylinder (252,800 particles) as a
second workload; the batched FP32 form against the plain FP64 GPU form to
equilibrium on instances of the batched workload; the 64-instance batch; the
reverse mode; the rows built after the hot path; the error against the FP64
oracle of every leg on a reduced twin the oracle can run; the oracle itself on
the host cores (one thread and all cores) as the CPU baseline.

--impl reference times the FP64 CPU oracle (the only reference there is: the
paper ships no code) on the host cores on a bounded sample of the headline
workload.  --profile-case runs a fixed small number of substeps of one
workload (the command under ncu).

Multi-GPU: one single body does not shard (halo exchanges every substep), so
N ranks run N independent replicas (weak scaling); the value is the sum over
ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solid-substep particle-updates/s; time-to-equilibrium vs plain FP64 at tol"
_T0 = time.monotonic()


def log(msg: str):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.monotonic() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)
UNIT = "particle-substeps/s"
STAGES = {1: "k_stress", 2: "k_force", 3: "k_damp", 4: "k_drift"}


def algo_bytes(dim: int, k: float, plastic: bool, diffusion: bool, rsize: int = 4):
    """Algorithmic bytes per particle per substep of each stage (each array
    streamed once per pass, CSR int32 indices 4 B per neighbour, kernel
    gradients recomputed from X, damping pairs owned once: k/2 pair indices of
    4 B each; u in FP64).  rsize: bytes of the per-particle reals (4 in mixed
    precision).  k: measured neighbours per particle."""
    d2 = dim * dim
    x = dim * rsize
    stress = 4 * k + x + 8 * dim + d2 * rsize + d2 * rsize      # idx, X, u, B0, write P B0
    if plastic:
        stress += 2 * 7 * rsize                                    # C_p^-1 (6) + alpha r/w
    if diffusion:
        stress += rsize                                            # c
    force = 4 * k + x + d2 * rsize + 2 * dim * rsize              # idx, X, P B0, v r/w
    damp = 2 * k + x + 2 * dim * rsize                             # pair idx, X, v r/w
    drift = dim * rsize + 2 * 8 * dim                              # v, u r/w (FP64)
    return {1: stress, 2: force, 3: damp, 4: drift}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--check-every", type=int, default=0,
                    help="0: device-side WHILE loop (production); k: host-checked chunks")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: launch shapes from the autotuner after the first warm-up step")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-substeps", type=int, default=30,
                    help="substeps of each oracle CPU-baseline sample (0 = skip)")
    ap.add_argument("--cpu-sample", default="80x40x10",
                    help="lattice of the plate sub-block the oracle baseline runs")
    ap.add_argument("--cylinder", type=int, default=1, help="the J2 cylinder leg (0 = skip)")
    ap.add_argument("--compare-instances", type=int, default=4,
                    help="instances (the smallest of the batched workload) of the batched-FP32 "
                         "vs plain-FP64 comparison (0 = skip)")
    ap.add_argument("--compare-steps", type=int, default=10,
                    help="relaxed slow steps of that comparison")
    ap.add_argument("--max-substeps", type=int, default=10000,
                    help="cap on substeps per slow step in the batch and comparison legs "
                         "(reported: steps that reach it are not converged)")
    ap.add_argument("--budget-s", type=float, default=480.0,
                    help="legs after the headline start only while the run is younger than this")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="instances of the batched workload (0 = skip)")
    ap.add_argument("--next-rows", type=int, default=1,
                    help="measure the droplet schedule, two-stage diffusion and equilibrium "
                         "adjoint (0 = skip)")
    ap.add_argument("--adjoint-steps", type=int, default=3,
                    help="slow steps reversed in the FP64 reverse-mode measurement (0 = skip)")
    ap.add_argument("--twins", type=int, default=1,
                    help="error against the FP64 oracle on reduced twins (0 = skip)")
    ap.add_argument("--ke-study", type=int, default=0,
                    help="slow steps of the strip's kinetic-energy criterion study (0 = skip)")
    ap.add_argument("--ref-substeps", type=int, default=2,
                    help="oracle substeps per reference-arm step")
    ap.add_argument("--profile-case", default=None,
                    choices=["bar2d", "cylinder3d", "strip2d", "plate3d", "membrane_droplet3d"],
                    help="instead of the benchmark: build this workload and run --substeps "
                         "substeps of its first slow step(s) (the command under ncu)")
    ap.add_argument("--substeps", type=int, default=2, help="substeps per slow step of --profile-case")
    ap.add_argument("--slow-steps", type=int, default=1, help="slow steps of --profile-case")
    ap.add_argument("--diffusion-mode", type=int, default=0, help="diffusion form of --profile-case")
    ap.add_argument("--reverse", action="store_true",
                    help="--profile-case: also reverse the last slow step (FP64 reverse mode)")
    ap.add_argument("--membrane-mm", type=float, default=10.0,
                    help="--profile-case membrane_droplet3d: in-plane size (the paper's is 10 mm)")
    ap.add_argument("--plate-size", default="1000x250x10",
                    help="--profile-case plate3d: lattice (a smaller plate for full ncu sets)")
    ap.add_argument("--tile", type=int, default=0,
                    help="--profile-case: particles per Morton tile (0 = default)")
    ap.add_argument("--damp-warps", type=int, default=0,
                    help="--profile-case: damping warps per CTA (0 = default)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cpu():
    """Core count and CPU model of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model or platform.processor() or platform.machine(),
            "machine": platform.machine()}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms; each line
    is stamped with the host clock so a window can be selected afterwards."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def wait_first(self, timeout: float = 5.0):
        """Block until the sampler has produced a line (so it covers what follows)."""
        t_end = time.monotonic() + timeout
        while self.proc is not None and not self.lines and time.monotonic() < t_end:
            time.sleep(0.01)

    def summary(self, a: float, b: float, label: str):
        """Median SM clock and the throttle reasons seen in [a, b] (host time)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, smax, reasons = [], None, set()
        for ts, ln in list(self.lines):
            if ts < a or ts > b:
                continue
            parts = [q.strip() for q in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "window": label}

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)


# sources of the substep kernels whose ncu traffic the roofline reports
TRAFFIC_SOURCES = ("mts_substep.cu", "mts_setup.cu", "mts_device.cuh", "mts_internal.cuh",
                   "mts_tiles.cuh")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2309_04010_gb300", "csrc")
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str, n: int):
    """DRAM bytes per substep of `kernel` from the committed ncu summary, scaled
    to n particles; None when the summary is missing or for other sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != source_hash():
            return None
        k = d["workloads"][workload]["kernels"][kernel]
        return k["dram_bytes_per_particle"] * n
    except Exception:
        return None


# ----------------------------------------------------------------------------
# FP64 oracle on the host cores
# ----------------------------------------------------------------------------
def plate_sample_case(spec: str):
    """A sub-block of the headline plate: same spacing, material, damping,
    diffusion and boundary conditions (clamped x = 0 end, held top and bottom
    layers), fewer particles."""
    from synth import bodies as B
    nx, ny, nz = (int(v) for v in spec.split("x"))
    return B.plate3d(nx=nx, ny=ny, nz=nz)


def _oracle_worker(spec, substeps, barrier, queue):
    """One host core: build the oracle body of the sample (not timed), wait for
    the others, then time `substeps` substeps of the first slow step."""
    import oracle
    case = plate_sample_case(spec)
    ob = oracle.body_from_case(case)
    dts = ob.diffusion_dt()[1]
    barrier.wait()
    t0 = time.time()
    ob.advance(dt_slow=dts, ke_tol=-1.0, ke_mode=1, max_substeps=substeps)
    queue.put((case.n * substeps, time.time() - t0, t0))


def oracle_baseline(spec: str, substeps: int, all_cores: bool = True):
    """The oracle as it stands on the host: one thread, and one process per core
    (spawned, so they are independent of the CUDA context) each running the
    same sample; value = particle-substeps / wall time."""
    import multiprocessing as mp
    import oracle
    case = plate_sample_case(spec)
    ob = oracle.body_from_case(case)
    dts = ob.diffusion_dt()[1]
    t0 = time.perf_counter()
    ob.advance(dt_slow=dts, ke_tol=-1.0, ke_mode=1, max_substeps=substeps)
    t1 = time.perf_counter() - t0
    one = case.n * substeps / t1
    del ob
    host = host_cpu()
    out = {"one_thread": {"value": one, "seconds": t1}, "host": host}
    ncore = host["nproc"] or 1
    if all_cores and ncore > 1:
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(ncore)
        q = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker, args=(spec, substeps, barrier, q))
                 for _ in range(ncore)]
        for p in procs:
            p.start()
        res = [q.get(timeout=900) for _ in procs]
        for p in procs:
            p.join(timeout=60)
        start = min(r[2] for r in res)
        end = max(r[2] + r[1] for r in res)
        out["all_cores"] = {"value": sum(r[0] for r in res) / (end - start), "processes": ncore,
                            "seconds": end - start}
    out["sample"] = (f"{substeps} substeps of the first slow step of a {spec} sub-block of the "
                     f"plate ({case.n} particles, same spacing, material and boundary "
                     f"conditions), FP64 oracle; set-up not timed")
    out["n"] = case.n
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    case = plate_sample_case(args.cpu_sample)
    ob = oracle.body_from_case(case)
    dts = ob.diffusion_dt()[1]
    total, t_all = 0, 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ob.advance(dt_slow=dts, ke_tol=-1.0, ke_mode=1, max_substeps=args.ref_substeps)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            total += case.n * args.ref_substeps
            t_all += dt
    value = total / t_all
    sample = (f"{args.ref_substeps} substeps of each of {args.steps} slow steps of a "
              f"{args.cpu_sample} sub-block ({case.n} particles) of the 2.5 M-particle plate, "
              f"FP64 oracle, 1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "plate3d-2500000", "n_particles": 2500000,
                   "sample": "bounded: a sub-block of the plate, oracle substeps per slow "
                             "step as stated"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------
def reduce_over_ranks(dist, ms: float, updates: float, device: str):
    """Whole-job timing of replicated ranks: the slowest rank's time (max) and
    the particle updates of all ranks (sum); dist = None for one process."""
    if dist is None:
        return ms, updates
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    dist.barrier()
    return float(t.item()), float(u.item())


def shard_instances(sizes, world: int):
    """Instances of a batch dealt to ranks by estimated work (particles),
    largest first onto the least-loaded rank; returns one index list per
    rank, each ascending.  Instances are independent: no collective is needed
    on the data path."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


def step_params(case, body, l, check_every=0, max_substeps=None):
    """Slow step l of a workload: the load increment l / n_ramp, or one
    diffusion step of the stable size; kinetic-energy criterion of the case."""
    plan = case.plan
    p = dict(ke_tol=plan.ke_tol, ke_ref=plan.ke_ref, ke_mode=plan.ke_mode,
             max_substeps=max_substeps or plan.max_substeps, check_every=check_every)
    if case.diffusion is not None:
        p["dt_slow"] = body.diffusion_dt()[1]
    else:
        p["ramp"] = l / max(plan.n_ramp, 1)
    return p


def rel_err(a, b):
    import numpy as np
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def twin_error(ctx, M, case, slow_steps: int, substeps: int, precision, diffusion_mode=0):
    """Error of the GPU form against the FP64 oracle on the same body: both run
    `slow_steps` slow steps of exactly `substeps` substeps (counts frozen, so
    the comparison does not depend on a threshold test); returns the relative
    max-norm errors of u (and c)."""
    import oracle
    gb = M.body_from_case(ctx, case, precision)
    if diffusion_mode:
        gb.set_diffusion_mode(diffusion_mode)
    ob = oracle.body_from_case(case, damp_layout=gb.damping_layout())
    if diffusion_mode:
        ob.set_diffusion_mode(diffusion_mode)
    for l in range(1, slow_steps + 1):
        p = step_params(case, gb, l, max_substeps=substeps)
        p["ke_tol"] = -1.0
        if "dt_slow" in p:     # the oracle's stable size (the library's agrees to rounding)
            p["dt_slow"] = ob.diffusion_dt()[1]
            p["force_dt"] = True
        rg = gb.advance_slow_step(**p)
        ro = ob.advance(dt_slow=p.get("dt_slow", 0.0), ramp=p.get("ramp", 0.0), ke_tol=-1.0,
                        ke_mode=p["ke_mode"], max_substeps=substeps, force_dt=True)
        if not (rg.substeps == ro.substeps == substeps):
            raise RuntimeError("twin runs took different substep counts")
    out = {"n": case.n, "slow_steps": slow_steps, "substeps_per_slow_step": substeps,
           "u_rel_err": rel_err(gb.read(M.F_U), ob.read(oracle.F_U))}
    if case.diffusion is not None:
        out["c_rel_err"] = rel_err(gb.read(M.F_C), ob.read(oracle.F_C))
    gb.close()
    return out


def stage_profile(gb, case, l, substeps: int = 24):
    """CUDA-event time per substep of each stage (all of its launches), measured
    inside the captured graph on the library stream over `substeps` substeps of
    a fixed-size replay of slow step l from the body's current state (restored
    afterwards)."""
    ck = gb.save_state()
    st = {}
    for s in (1, 2, 3, 4):
        gb.set_profiling(s)
        p = step_params(case, gb, l, check_every=4, max_substeps=substeps)
        p["ke_tol"] = -1.0
        p.pop("dt_slow", None)           # substeps only: no diffusion step in the replay
        p["ramp"] = p.get("ramp", 0.0)
        r = gb.advance_slow_step(**p)
        st[s] = r.prof_ms / max(r.prof_count, 1)
        gb.load_state(ck)
    gb.set_profiling(0)
    return st


def measure_workload(ctx, M, args, case, prec, name, steps, warmup, dist=None, clocks=None):
    """Warm-up slow steps (the autotuner after the first), then `steps` timed
    slow steps to the kinetic-energy criterion with CUDA events on the library
    stream; the stage profile and the roofline of the dominant stage."""
    import torch
    t0 = time.perf_counter()
    gb = M.body_from_case(ctx, case, prec)
    setup_s = time.perf_counter() - t0
    off, _ = gb.neighbors()
    k = int(off[-1]) / case.n
    tune, l = None, 0
    for w in range(warmup):
        l += 1
        gb.advance_slow_step(**step_params(case, gb, l, args.check_every))
        if w == 0 and args.autotune:
            t0 = time.perf_counter()
            tune = gb.autotune(substeps=8, ramp=(l + 1) / max(case.plan.n_ramp, 1)
                               if case.diffusion is None else 0.0)
            tune["seconds"] = time.perf_counter() - t0
    gb.set_profiling(0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    h0 = time.monotonic()
    e0.record(stream)
    reps = []
    for s in range(steps):
        l += 1
        reps.append(gb.advance_slow_step(**step_params(case, gb, l, args.check_every)))
    e1.record(stream)
    torch.cuda.synchronize()
    h1 = time.monotonic()
    ms = e0.elapsed_time(e1)
    clk = clocks.summary(h0, h1, f"{name}: timed region") if clocks else None
    substeps = sum(r.substeps for r in reps)
    st = stage_profile(gb, case, l)
    dom = max(st, key=st.get)
    ab = algo_bytes(case.dim, k, case.material.model == "j2", case.diffusion is not None,
                    4 if prec == M.MIXED else 8)
    hbm, peak_kind = peaks()
    achieved = ab[dom] * case.n / (st[dom] * 1e-3) / 1e9
    whole = sum(ab.values())
    whole_gbs = whole * case.n * substeps / (ms * 1e-3) / 1e9
    return {
        "gb": gb, "l": l, "ms": ms, "substeps": substeps, "reps": reps, "clocks": clk,
        "launches": sum(r.kernel_launches for r in reps), "k": k, "setup_s": setup_s,
        "tune": tune, "stage_ms": {STAGES[s]: st[s] for s in st},
        "roofline": {"bound": "hbm", "kernel": STAGES[dom], "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": ncu_traffic(name, STAGES[dom], case.n),
                     "peak_kind": f"{peak_kind} copy bandwidth",
                     "launch_ms": st[dom],
                     "algorithmic_bytes_per_particle": ab[dom],
                     "timing": "CUDA events recorded inside the captured graph on the library "
                               "stream around the stage (all of its launches in one substep), "
                               "over a 24-substep replay from the state after the timed region"},
        "whole_substep": {"algorithmic_bytes_per_particle": whole, "achieved_gbs": whole_gbs,
                          "frac": whole_gbs / hbm,
                          "per_stage_algorithmic_bytes": {STAGES[s]: ab[s] for s in ab}},
    }


def e2e_steps(gb, case, M, l0, steps, check_every):
    """End to end through the C ABI with host-resident state: upload the state
    fields (u, v, and c for a diffusion body) from pinned host memory, advance
    one slow step, read them back, every step; host wall clock."""
    import torch
    fields = [M.F_U, M.F_V] + ([M.F_C] if case.diffusion is not None else [])
    host = {f: torch.from_numpy(gb.read(f)).pin_memory().numpy() for f in fields}
    nbytes = sum(host[f].nbytes for f in fields)
    sub, t = 0, 0.0
    for s in range(steps):
        t0 = time.perf_counter()
        for f in fields:
            gb.write(f, host[f])
        r = gb.advance_slow_step(**step_params(case, gb, l0 + s + 1, check_every))
        for f in fields:
            gb.read(f, out=host[f])
        t += time.perf_counter() - t0
        sub += r.substeps
    return {"value": case.n * sub / t if t > 0 else None, "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "substeps": sub, "seconds": t,
            "fields": "u, v" + (", c" if case.diffusion is not None else "")}


def measure_compare(ctx, M, args):
    """North-star comparison: the batched FP32 (mixed) form against the plain
    FP64 GPU form, time to equilibrium over `compare_steps` relaxed slow steps
    of the same instances of the batched workload.  Both start warm (one
    untimed slow step each, graphs captured); mixed: all instances in one
    graph launch per slow step; FP64: each instance on its own, one after
    another.  Each form's error against the FP64 oracle is taken on the
    smallest J2 bar and the smallest strip of the set (twin runs with frozen
    substep counts)."""
    import torch
    from synth import bodies as B
    cases_all = B.batch_instances(count=64)
    strips = sorted([c for c in cases_all if c.diffusion is not None], key=lambda c: c.n)
    bars = sorted([c for c in cases_all if c.diffusion is None], key=lambda c: c.n)
    half = max(args.compare_instances // 2, 1)
    cases = strips[:half] + bars[:args.compare_instances - half]
    cap = args.max_substeps
    out = {"instances": len(cases), "particles": int(sum(c.n for c in cases)),
           "selection": "the smallest strips and J2 bars of the 64-instance workload",
           "slow_steps": args.compare_steps, "max_substeps": cap}
    # mixed, batched
    bodies = [M.body_from_case(ctx, c, M.MIXED) for c in cases]
    bt = M.Batch(ctx, bodies)
    bt.advance([step_params(c, b, 1, max_substeps=cap) for c, b in zip(cases, bodies)])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sub32, n32 = 0, []
    conv32 = 0
    for l in range(2, args.compare_steps + 2):
        reps = bt.advance([step_params(c, b, l, max_substeps=cap) for c, b in zip(cases, bodies)])
        sub32 += sum(c.n * r.substeps for c, r in zip(cases, reps))
        n32.append(sum(r.substeps for r in reps))
        conv32 += sum(r.converged for r in reps)
    torch.cuda.synchronize()
    t32 = time.perf_counter() - t0
    bt.close()
    tip32 = [list(r.tip_deflection[:c.dim]) for c, r in zip(cases, reps)]
    for b in bodies:
        b.close()
    # FP64, one instance after another
    bodies = [M.body_from_case(ctx, c, M.FP64) for c in cases]
    for c, b in zip(cases, bodies):
        b.advance_slow_step(**step_params(c, b, 1, max_substeps=cap))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sub64, n64, conv64 = 0, [], 0
    for l in range(2, args.compare_steps + 2):
        tot = 0
        for c, b in zip(cases, bodies):
            r = b.advance_slow_step(**step_params(c, b, l, max_substeps=cap))
            sub64 += c.n * r.substeps
            tot += r.substeps
            conv64 += r.converged
        n64.append(tot)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    tip64 = [list(b.read(M.F_U)[c.tip_ids].mean(axis=0)) for c, b in zip(cases, bodies)]
    for b in bodies:
        b.close()
    dtip = max(abs(a - b) / max(abs(b), 1e-300)
               for x, y in zip(tip32, tip64) for a, b in zip(x, y) if abs(b) > 1e-12)
    out.update({"batched_fp32_s": t32, "plain_fp64_s": t64,
                "time_to_equilibrium_speedup": t64 / t32 if t32 > 0 else None,
                "batched_fp32_substeps_per_slow_step": n32,
                "plain_fp64_substeps_per_slow_step": n64,
                "converged_slow_steps": {"batched_fp32": conv32, "plain_fp64": conv64,
                                         "of": len(cases) * args.compare_steps},
                "batched_fp32_value": sub32 / t32, "plain_fp64_value": sub64 / t64,
                "unit": UNIT,
                "tip_rel_difference_fp32_vs_fp64": float(dtip),
                "timing": "host wall clock around the slow steps, stream synchronised; both "
                          "forms warm (graphs captured in an untimed first slow step)"})
    if args.twins:
        bars = [c for c in cases if c.diffusion is None]
        strips = [c for c in cases if c.diffusion is not None]
        errs = {}
        for nm, group in (("bar", bars), ("strip", strips)):
            if not group:
                continue
            c = min(group, key=lambda z: z.n)
            errs[nm] = {"fp64": twin_error(ctx, M, c, 2, 60, M.FP64),
                        "mixed": twin_error(ctx, M, c, 2, 60, M.MIXED)}
        out["err_vs_oracle"] = errs
    return out


def measure_batch(ctx, args, M, rank=0, world=1, dist=None):
    """The batched mode on the 64-instance workload (uneven 2D strips and J2
    bars, mixed precision): slow step 2 of all bodies through one batch graph
    launch, against the same bodies advanced one after another from the same
    saved states.  With several ranks each takes a shard of the instances (no
    collective on the data path; max time and summed updates over ranks)."""
    import torch
    from synth import bodies as B
    cases_all = B.batch_instances(count=args.batch_count)
    mine = shard_instances([c.n for c in cases_all], world)[rank]
    cases = [cases_all[i] for i in mine]
    bodies = [M.body_from_case(ctx, c, M.MIXED) for c in cases]
    bt = M.Batch(ctx, bodies)
    cap = args.max_substeps
    bt.advance([step_params(c, b, 1, max_substeps=cap) for c, b in zip(cases, bodies)])  # warm-up
    t0 = time.perf_counter()
    shapes = bt.autotune(substeps=8, ramp=0.0)
    tune_s = time.perf_counter() - t0
    states = [b.save_state() for b in bodies]
    bt.advance([step_params(c, b, 2, max_substeps=cap) for c, b in zip(cases, bodies)])  # capture
    for b, s in zip(bodies, states):
        b.load_state(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    reps = bt.advance([step_params(c, b, 2, max_substeps=cap) for c, b in zip(cases, bodies)])
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    upd_b = sum(c.n * r.substeps for c, r in zip(cases, reps))
    for b, s in zip(bodies, states):
        b.load_state(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    upd_s = 0
    for c, b in zip(cases, bodies):
        r = b.advance_slow_step(**step_params(c, b, 2, max_substeps=cap))
        upd_s += c.n * r.substeps
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    bt.close()
    for b in bodies:
        b.close()
    tb, upd_b = reduce_over_ranks(dist, tb, float(upd_b), "cuda")
    ts, upd_s = reduce_over_ranks(dist, ts, float(upd_s), "cuda")

    def key(sh):
        return f"tile {sh['tile']}, {sh['damp_warps']} damping warps"
    return {"workload": f"batch_instances-{len(cases_all)}",
            "particles": int(sum(c.n for c in cases_all)), "n_gpus": world,
            "batched_value": upd_b / tb, "sequential_value": upd_s / ts,
            "speedup": (upd_b / tb) / (upd_s / ts), "unit": UNIT,
            "substeps_range": [int(min(r.substeps for r in reps)),
                               int(max(r.substeps for r in reps))],
            "converged": int(sum(r.converged for r in reps)), "max_substeps": cap,
            "shapes": {k: sum(1 for sh in shapes if key(sh) == k)
                       for k in sorted({key(sh) for sh in shapes})},
            "autotune_s": tune_s,
            "err_vs_oracle": "batch members compute what single bodies compute, bit for bit "
                             "(tested); the members' error is compare_fp32_batched_vs_fp64's",
            "timing": "host wall clock around slow step 2 of every instance, batched and then "
                      "one body after another from the same saved states, stream "
                      "synchronised, max over ranks"}


def measure_adjoint(ctx, args, M, case):
    """Reverse mode (FP64) on the cylinder: forward slow steps, then their
    reversal (recompute with tape + transposed substeps)."""
    import numpy as np
    import torch
    gb = M.body_from_case(ctx, case, M.FP64)
    plan = case.plan
    steps = [dict(ramp=l / plan.n_ramp, ke_tol=plan.ke_tol, ke_ref=plan.ke_ref,
                  ke_mode=plan.ke_mode, max_substeps=plan.max_substeps)
             for l in range(1, args.adjoint_steps + 1)]
    ckpts, counts = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p in steps:
        ckpts.append(gb.save_state())
        counts.append(gb.advance_slow_step(**p).substeps)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    gb.adjoint_enable(max(counts))
    gb.adjoint_seed(tip_bar=[1.0, 0.0, 0.0], force_bar=[1.0, 0.0, 0.0])
    th = np.zeros(7)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, ck, k in zip(reversed(steps), reversed(ckpts), reversed(counts)):
        gb.load_state(ck)
        th += gb.adjoint_slow_step(k, **p)
    torch.cuda.synchronize()
    ta = time.perf_counter() - t0
    gb.close()
    sub = sum(counts)
    out = {"workload": f"cylinder3d-j2-{case.n}", "precision": "f64", "slow_steps": len(steps),
           "substeps": sub, "forward_s": tf, "reverse_s": ta,
           "reverse_value": case.n * sub / ta, "unit": UNIT, "reverse_over_forward": ta / tf,
           "dtheta_nonzero": [bool(x != 0) for x in th],
           "timing": "host wall clock, stream synchronised; the reverse time includes the "
                     "taped recomputation of the step"}
    if args.twins:
        out["err_vs_oracle"] = adjoint_twin_error(ctx, M)
    out["batch_mixed"] = adjoint_batch_mixed(ctx, M)
    return out


def adjoint_batch_mixed(ctx, M, count: int = 8, nsub: int = 20):
    """Reverse mode of a mixed-precision batch: `count` instances of the
    batched workload advanced together (one graph launch per slow step, two
    slow steps of `nsub` substeps), then every member's two slow steps
    reversed one after another (FP64 adjoint on each member's FP64 twin);
    gradients of tip deflection and end force for all seven parameters."""
    import numpy as np
    import torch
    from synth import bodies as B
    cases = B.batch_instances(count=count, n_min=5_000, n_max=50_000, seed=B.SEED_BASE + 52)
    bodies = [M.body_from_case(ctx, c, M.MIXED) for c in cases]
    bt = M.Batch(ctx, bodies)
    ck = [[] for _ in cases]
    steps = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for l in (1, 2):
        ps = [dict(dt_slow=b.diffusion_dt()[1] if c.diffusion is not None else 0.0,
                   ramp=l / max(c.plan.n_ramp, 1), ke_tol=-1.0, ke_ref=c.plan.ke_ref,
                   max_substeps=nsub) for c, b in zip(cases, bodies)]
        for k, b in enumerate(bodies):
            ck[k].append(b.save_state())
        bt.advance(ps)
        steps.append(ps)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    bt.close()
    t0 = time.perf_counter()
    nonzero = 0
    for k, (c, b) in enumerate(zip(cases, bodies)):
        b.adjoint_enable(nsub)
        b.adjoint_seed(tip_bar=np.ones(c.dim), force_bar=np.ones(c.dim))
        th = np.zeros(7)
        for l in (1, 0):
            b.load_state(ck[k][l])
            th += b.adjoint_slow_step(nsub, **steps[l][k])
        nonzero += int(np.count_nonzero(th))
    torch.cuda.synchronize()
    ta = time.perf_counter() - t0
    for b in bodies:
        b.close()
    return {"instances": len(cases), "particles": int(sum(c.n for c in cases)),
            "slow_steps": 2, "substeps_per_slow_step": nsub, "forward_batched_s": tf,
            "reverse_s": ta, "nonzero_gradients": nonzero,
            "err_vs_oracle": "mixed members against the reverse-mode oracle: <= 1e-3 (tested; "
                             "2.4e-6 on the small cylinder above)",
            "timing": "host wall clock, stream synchronised; the reverse time includes the "
                      "members' FP64 twins' set-up on first use and the taped recomputations"}


def adjoint_twin_error(ctx, M):
    """Parameter gradients of the reverse mode (FP64 and mixed bodies) against
    the PyTorch reverse-mode oracle on a small J2 cylinder (4 x 2 mm, two slow
    steps of 8 substeps): the largest relative difference over the five
    parameters the objective depends on (E and the hardening law)."""
    import numpy as np
    import torch
    import oracle
    from oracle import adjoint as A
    from synth import bodies as B
    case = B.cylinder3d(L=4e-3, R=1e-3, dx=0.25e-3, n_slow=10)
    rng = np.random.default_rng(11)
    w_tip, w_f = rng.normal(size=3), rng.normal(size=3)
    nsub, out = 8, {"n": case.n, "slow_steps": 2, "substeps_per_slow_step": 8}
    th_o = None
    for prec, name in ((M.FP64, "fp64"), (M.MIXED, "mixed")):
        gb = M.body_from_case(ctx, case, prec)
        steps = [dict(ramp=l / case.plan.n_ramp, ke_tol=-1.0, max_substeps=nsub) for l in (1, 2)]
        ck = []
        for p in steps:
            ck.append(gb.save_state())
            gb.advance_slow_step(**p)
        gb.adjoint_enable(nsub)
        gb.adjoint_seed(tip_bar=w_tip, force_bar=w_f)
        th = np.zeros(7)
        for p, c in zip(reversed(steps), reversed(ck)):
            gb.load_state(c)
            th += gb.adjoint_slow_step(nsub, **p)
        if th_o is None:
            ob = oracle.body_from_case(case, damp_layout=gb.damping_layout())
            tb = A.TorchBody(case, ob)
            tt = tb.theta0().clone().requires_grad_(True)
            st = tb.initial_state()
            for p in steps:
                st, ef, tip, _ = tb.slow_step(st, tt, p["ramp"], nsub)
            L = (torch.from_numpy(w_tip) * tip).sum() + (torch.from_numpy(w_f) * ef).sum()
            th_o = torch.autograd.grad(L, tt)[0].numpy()
        gb.close()
        out[f"{name}_theta_rel_err"] = float(max(abs(th[k] - th_o[k]) / abs(th_o[k])
                                                 for k in range(5)))
    return out


def measure_next_rows(ctx, M, args):
    """The rows built after the hot path: the droplet-contact membrane
    (Sec. 5.4 schedule, 819,200 particles, mixed) with the one-pass and the
    two-stage diffusion step, and the equilibrium adjoint of a relaxed bar
    (FP64) against the unrolled reverse of the same slow step."""
    import torch
    from synth import bodies as B
    out = {}
    case = B.membrane_droplet3d(Lx=5e-3, Ly=5e-3)
    for mode in (0, 1):
        gb = M.body_from_case(ctx, case, M.MIXED)
        if mode:
            gb.set_diffusion_mode(1)
        kw = dict(ke_tol=-1.0, ke_ref=case.plan.ke_ref, ke_mode=1,
                  max_substeps=50)                        # fixed substeps per slow step
        gb.advance_slow_step(dt_slow=gb.diffusion_dt()[1], **kw)   # warm-up (graph capture)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sub = 0
        for _ in range(2):
            dts = gb.diffusion_dt()[1]
            sub += gb.advance_slow_step(dt_slow=dts, **kw).substeps
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        key = "membrane_two_stage" if mode else "membrane_one_pass"
        out[key] = {"particles": case.n, "slow_steps": 2, "substeps": sub, "seconds": dt,
                    "value": case.n * sub / dt, "unit": UNIT, "dt_slow": dts}
        gb.close()
        if args.twins:
            twin = B.membrane_droplet3d(Lx=0.6e-3, Ly=0.6e-3)
            out[key]["err_vs_oracle"] = twin_error(ctx, M, twin, 2, 20, M.MIXED,
                                                   diffusion_mode=mode)
    beam = B.bar2d(nx=24, ny=6, n_slow=4, eta=1e3)
    gb = M.body_from_case(ctx, beam, M.FP64)
    ck = gb.save_state()
    p = dict(ramp=0.25, ke_tol=1e-22, ke_ref=beam.plan.ke_ref, max_substeps=60000)
    k = gb.advance_slow_step(**p).substeps
    gb.adjoint_enable(k)
    gb.adjoint_seed(force_bar=[1.0, 0.0])            # d(end force)/d theta
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th_eq, iters = gb.adjoint_equilibrium(max_iters=200000, tol=1e-10)
    torch.cuda.synchronize()
    t_eq = time.perf_counter() - t0
    gb.adjoint_reset()
    gb.adjoint_seed(force_bar=[1.0, 0.0])
    gb.load_state(ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th_un = gb.adjoint_slow_step(k, **p)
    torch.cuda.synchronize()
    t_un = time.perf_counter() - t0
    gb.close()
    out["equilibrium_adjoint"] = {
        "workload": f"bar2d-{beam.n}-svk-relaxed", "forward_substeps": k,
        "equilibrium_iterations": iters, "equilibrium_s": t_eq, "unrolled_s": t_un,
        "dE_rel_difference": float(abs(th_eq[0] - th_un[0]) / abs(th_un[0]))}
    return out


def measure_ke_study(ctx, M, steps: int):
    """The kinetic-energy criterion study of the strip (the paper's procedure,
    Sec. 5.1 and 5.3): the same slow steps under criteria lowered by decades;
    tip displacement and substeps per slow step of each."""
    import torch
    from synth import bodies as B
    case = B.strip2d()
    out = {}
    for tol in (5e-4, 5e-6, 5e-8, 5e-10):
        gb = M.body_from_case(ctx, case, M.MIXED)
        dts = gb.diffusion_dt()[1]
        subs = []
        t0 = time.perf_counter()
        for _ in range(steps):
            r = gb.advance_slow_step(dt_slow=dts, ke_tol=tol, ke_ref=case.plan.ke_ref, ke_mode=1,
                                     max_substeps=400000)
            subs.append(int(r.substeps))
        torch.cuda.synchronize()
        out[f"{tol:g}"] = {"tip": [float(x) for x in r.tip_deflection[:2]],
                           "substeps_mean": sum(subs) / len(subs), "substeps_max": max(subs),
                           "seconds": time.perf_counter() - t0}
        gb.close()
    return {"workload": f"strip2d-{case.n}", "slow_steps": steps, "criteria": out}


def run_ours(args, rank, world, local):
    import torch

    from paper_2309_04010_gb300 import _build
    _build.build()
    from paper_2309_04010_gb300 import mtssph as M
    from synth import bodies as B

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    prec = M.MIXED if args.precision == "mixed" else M.FP64
    ctx = M.Context(local)
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()

    # ---- headline: the 2.5 M-particle plate
    log("plate: set-up, warm-up, timed slow steps")
    case = B.plate3d()
    h = measure_workload(ctx, M, args, case, prec, "plate3d", args.steps, args.warmup, dist, clocks)
    gb = h["gb"]
    ms, total_updates = reduce_over_ranks(dist, h["ms"], float(h["substeps"]) * case.n, "cuda")
    value = total_updates / (ms * 1e-3)
    log(f"plate: {value:.3e} {UNIT}; end to end")
    e2e = e2e_steps(gb, case, M, h["l"], args.e2e_steps, args.check_every)
    shapes = gb.shapes()
    gb.close()
    err = None
    if args.twins and rank == 0:
        log("plate twin against the oracle")
        err = twin_error(ctx, M, B.plate3d(nx=40, ny=20, nz=10), 2, 40, prec)
        err["twin"] = "40 x 20 x 10 sub-block of the plate (same spacing, material, BCs)"

    def within_budget(name):
        ok = time.monotonic() - _T0 < args.budget_s
        log(f"{name}: " + ("start" if ok else "skipped (time budget)"))
        return ok

    # ---- other legs (rank 0)
    cyl = None
    if args.cylinder and rank == 0 and within_budget("cylinder"):
        cc = B.cylinder3d()
        c = measure_workload(ctx, M, args, cc, prec, "cylinder3d", args.steps + 2, args.warmup,
                             None, clocks)
        cyl = {"workload": f"cylinder3d-j2-{cc.n}",
               "value": cc.n * c["substeps"] / (c["ms"] * 1e-3),
               "unit": UNIT, "ms_per_step": c["ms"] / (args.steps + 2),
               "substeps_per_step": [r.substeps for r in c["reps"]],
               "converged": [r.converged for r in c["reps"]],
               "roofline": dict(c["roofline"], stage_ms_per_substep=c["stage_ms"]),
               "whole_substep": c["whole_substep"], "launch_shapes": c["gb"].shapes(),
               "autotune": c["tune"], "clocks": c["clocks"], "neighbours_per_particle": c["k"]}
        c["gb"].close()
        if args.twins:
            cyl["err_vs_oracle"] = twin_error(ctx, M, B.cylinder3d(L=6e-3, R=1.5e-3, n_slow=500),
                                              2, 30, prec)
    def leg(name, run):
        """One side leg with the clocks seen during it (median SM clock, reasons)."""
        h0 = time.monotonic()
        out = run()
        if isinstance(out, dict):
            out["clocks"] = clocks.summary(h0, time.monotonic(), name)
        return out

    compare = (leg("compare", lambda: measure_compare(ctx, M, args))
               if args.compare_instances > 0 and rank == 0 and within_budget("compare") else None)
    batch = (leg("batch", lambda: measure_batch(ctx, args, M, rank, world, dist))
             if args.batch_count > 0 and (world > 1 or within_budget("batch")) else None)
    adjoint = (leg("adjoint", lambda: measure_adjoint(ctx, args, M, B.cylinder3d()))
               if args.adjoint_steps > 0 and rank == 0 and within_budget("adjoint") else None)
    nxt = (leg("next rows", lambda: measure_next_rows(ctx, M, args))
           if args.next_rows > 0 and rank == 0 and within_budget("next rows") else None)
    study = (leg("criterion study", lambda: measure_ke_study(ctx, M, args.ke_study))
             if args.ke_study > 0 and rank == 0 and within_budget("criterion study") else None)
    clocks.stop()
    if rank != 0:
        return
    cpu = None
    if args.cpu_substeps > 0 and world == 1:
        log("oracle on the host cores")
        ob = oracle_baseline(args.cpu_sample, args.cpu_substeps)
        best = ob.get("all_cores", ob["one_thread"])
        cpu = {"value": best["value"], "unit": UNIT,
               "cores": ob.get("all_cores", {}).get("processes", 1), "kind": "oracle",
               "sample": ob["sample"] + "; value: one process per core, all started together",
               "one_thread_value": ob["one_thread"]["value"], "host": ob["host"]}
    plan = case.plan
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == M.MIXED else "f64", "data": "synthetic",
        "config": {"workload": "plate3d-2500000", "n_particles": case.n,
                   "neighbours_per_particle": h["k"], "precision": args.precision,
                   "precision_note": "f32 per-particle arithmetic; f64 displacement and "
                                     "kinetic-energy/max reductions" if prec == M.MIXED else "f64",
                   "slow_steps": f"{args.warmup + 1}..{args.warmup + args.steps} of the schedule "
                                 f"(diffusion step of the stable size each)",
                   "ke_criterion": f"density kinetic energy <= {plan.ke_tol:g} x 3 K beta, "
                                   "tested once E_k has passed its peak",
                   "substeps_per_step": [r.substeps for r in h["reps"]],
                   "converged": [r.converged for r in h["reps"]],
                   "l2": "working set larger than L2 (no flush)",
                   "parallelism": "replicas" if world > 1 else "single",
                   "setup_s": h["setup_s"], "launch_shapes": shapes, "autotune": h["tune"]},
        "gpu_launches": h["launches"],
        "roofline": dict(h["roofline"], stage_ms_per_substep=h["stage_ms"]),
        "whole_substep": h["whole_substep"],
        "err_vs_oracle": err,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "cylinder": cyl,
        "compare_fp32_batched_vs_fp64": compare,
        "batch": batch,
        "adjoint": adjoint,
        "next_rows": nxt,
        "ke_study": study,
        "clocks": h["clocks"],
    }
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A known, small number of launches for an ncu capture: build the
    workload's body (set-up), apply its first load increment (or, for the
    diffusion workloads, one diffusion step of the stable size) and run
    --substeps substeps with the kinetic-energy stop disabled; --reverse then
    reverses the last slow step.  Prints one line with the substep count."""
    from paper_2309_04010_gb300 import _build
    _build.build()
    from paper_2309_04010_gb300 import mtssph as M
    from synth import bodies as B

    if args.profile_case == "membrane_droplet3d":
        case = B.membrane_droplet3d(Lx=args.membrane_mm * 1e-3, Ly=args.membrane_mm * 1e-3)
    elif args.profile_case == "plate3d":
        nx, ny, nz = (int(v) for v in args.plate_size.split("x"))
        case = B.plate3d(nx=nx, ny=ny, nz=nz)
    else:
        case = getattr(B, args.profile_case)()
    ctx = M.Context(0)
    prec = M.MIXED if args.precision == "mixed" else M.FP64
    gb = M.body_from_case(ctx, case, prec)
    if args.tile or args.damp_warps:
        gb.set_shapes(tile=args.tile, damp_warps=args.damp_warps)
    if args.diffusion_mode:
        gb.set_diffusion_mode(args.diffusion_mode)
    off, _ = gb.neighbors()
    total, p, ck = 0, None, None
    for l in range(1, args.slow_steps + 1):
        ramp = l / case.plan.n_ramp if case.plan.n_ramp else 0.0
        p = dict(ramp=ramp, ke_tol=-1.0, max_substeps=args.substeps, check_every=args.substeps)
        if case.diffusion is not None:
            p.update(dt_slow=gb.diffusion_dt()[1], ke_mode=1, force_dt=True)
        ck = gb.save_state()
        total += gb.advance_slow_step(**p).substeps
    if args.reverse:
        gb.adjoint_enable(args.substeps)
        gb.adjoint_seed(tip_bar=[1.0] * case.dim, force_bar=[1.0] * case.dim)
        gb.load_state(ck)
        gb.adjoint_slow_step(args.substeps, **p)
    print(f"profile_case workload={args.profile_case} n={case.n} nnz={int(off[-1])} "
          f"precision={args.precision} substeps={total} shapes={gb.shapes()}")
    gb.close()
    ctx.close()


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
