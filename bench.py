"""Benchmark of the explicit PIC step on one GB300 (or N, one process each).

Workload (default): thermal_tsc_256 -- a 256^3 periodic box, one electron
species at 8 particles per cell (134,217,728 particles), Maxwellian
u_th = 0.05 c, TSC shape, density 0.01 over a fixed neutralising
background, dt = 0.5 x the 3D Courant limit; synthetic, seeded.

Metric: particle updates per second in push+deposit (field gather, Boris,
move, Esirkepov deposition, frame maintenance) of the mixed form
(int32 cell + FP32 offsets in supercell frames), with the whole step
captured in a CUDA graph.  Reported alongside: the plain FP64 GPU form on
the same workload, the full-step rate (adds the Yee update), the HBM
roofline fraction of the push+deposit kernel, an end-to-end number through
the C ABI from pinned host buffers, and the FP64 oracle timed on a bounded
sample on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle updates/sec (push+deposit) at 1 GB300 and % of HBM roofline, batched FP32 vs plain"
UNIT = "particle updates/s"
FALLBACK_HBM_GBS = 6800.0
# algorithmic HBM bytes per unit (mixed form): particle read 32 B + write 28 B
# (the weight is read-only); fields: E, B read 24 B/cell, J written 12 B/cell
MIXED_BYTES_PER_PARTICLE = 60.0
MIXED_BYTES_PER_CELL = 36.0
# plain FP64 form: particle read 56 B + write 48 B; fields 48 + 24 B/cell
PLAIN_BYTES_PER_PARTICLE = 104.0
PLAIN_BYTES_PER_CELL = 72.0
PUSH_KERNEL_SRC = os.path.join(ROOT, "paper_1606_02862_gb300", "csrc", "k_push.cu")
# machine-readable figures of the committed ncu summary of the push kernel
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "push_deposit_thermal_tsc.json")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001 - absent on a machine without the driver's file
        return FALLBACK_HBM_GBS, "fallback"


def push_profile():
    """Per-particle DRAM bytes, L1 data-pipe wavefronts (shared memory and
    global LSU traffic) and FP32 operations of the push kernel from the
    committed ncu figures (thermal TSC, 8x4x4 supercells, 256 threads, a
    JSON file beside the summary), or Nones when the file is absent or the
    kernel source changed since the counters were taken."""
    none = {"tpp": None, "wpp": None, "fpp": None, "wkind": None}
    try:
        with open(PUSH_KERNEL_SRC, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        with open(TRAFFIC_SUMMARY) as f:
            prof = json.load(f)
        if prof.get("kernel_source_sha256") != sha:
            return none
        l1 = prof.get("l1_wavefronts_per_particle")
        return {"tpp": float(prof["dram_bytes_per_particle"]),
                "wpp": float(l1 if l1 is not None else prof["shared_wavefronts_per_particle"]),
                "wkind": "l1" if l1 is not None else "smem",
                "fpp": float(prof["fp32_ops_per_particle"]) if "fp32_ops_per_particle" in prof else None}
    except Exception:  # noqa: BLE001
        return none


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:  # noqa: BLE001
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:  # noqa: BLE001
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        busy = [r for r in rows if r[0] > 0]
        sm = sorted(r[0] for r in busy) or [0.0]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- ours

def binding_roofline(result, npart):
    """The roofline that binds the TSC push kernel: L1 data-pipe wavefronts
    (shared memory plus global LSU traffic; ncu count per particle from the
    committed profile) per second against one wavefront per cycle per SM at
    the SM clock sampled during the run."""
    wpp = result.get("wpp")
    mhz = (result.get("clocks") or {}).get("sm_mhz")
    if not wpp or not mhz:
        return None
    try:
        import torch

        nsm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:  # noqa: BLE001
        return None
    achieved = wpp * npart / (result["push_ms"] * 1e-3) / 1e9
    peak = nsm * mhz * 1e6 / 1e9
    return {"bound": "l1_data_pipe" if result.get("wkind") == "l1" else "smem", "achieved": achieved,
            "peak": peak, "unit": "G wavefronts/s",
            "frac": achieved / peak, "kernel": "k_push_deposit",
            "per_particle": wpp, "peak_source": f"1 wavefront/clk/SM x {nsm} SMs x {mhz:.0f} MHz sampled"}

def alu_roofline(result, npart):
    """The FP32 arithmetic bound of the push kernel: FP32 operations (FFMA,
    FMUL, FADD; a packed f32x2 instruction counts two) per particle (ncu,
    committed profile) per second against 128 FP32 lanes per SM per cycle at
    the sampled SM clock."""
    fpp = result.get("fpp")
    mhz = (result.get("clocks") or {}).get("sm_mhz")
    if not fpp or not mhz:
        return None
    try:
        import torch

        nsm = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:  # noqa: BLE001
        return None
    achieved = fpp * npart / (result["push_ms"] * 1e-3) / 1e12
    peak = nsm * 128 * mhz * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T FP32 operations/s",
            "frac": achieved / peak, "kernel": "k_push_deposit", "per_particle": fpp,
            "peak_source": f"128 FP32 lanes/clk/SM x {nsm} SMs x {mhz:.0f} MHz sampled"}


def make_state(torch, n, ppc, u_th, pinned=True):
    from paper_1606_02862_gb300 import workloads as W

    npart = n * n * n * ppc
    X = torch.empty((npart, 3), dtype=torch.float64, pin_memory=pinned)
    U = torch.empty((npart, 3), dtype=torch.float64, pin_memory=pinned)
    Wt = torch.empty((npart,), dtype=torch.float64, pin_memory=pinned)
    W.fill_thermal(X.numpy(), U.numpy(), Wt.numpy(), n, n, n, ppc, u_th)
    return X, U, Wt


SHAPE = {"tsc": 2, "cic": 1, "pcs": 3}


GATHER = {"momentum": 0, "energy": 1}


def new_ctx(pic, n, precision, sc, threads, shape=2, gather=0, sort_every=0):
    from paper_1606_02862_gb300 import workloads as W

    ctx = pic.Context([(n, n, n)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT,
                      [pic.Species(-1.0, 1.0, shape, True, gather)], precision=precision, sc=sc,
                      threads_per_sc=threads, use_graph=True, sort_every=sort_every)
    ctx.set_background(0, 0.01)
    return ctx


def load(ctx, X, U, Wt):
    n = X.shape[0]
    ctx.load_particles_ptr(0, 0, n, X.data_ptr(), U.data_ptr(), Wt.data_ptr())


def cpu_baseline_oracle(steps=15, n=32, ppc=8):
    """The FP64 oracle on a bounded sample of the same recipe (n^3 box)."""
    import oracle
    from paper_1606_02862_gb300 import workloads as W

    oracle.build()
    wl = W.thermal_tsc(n=n, ppc=ppc, u_th=0.05)
    b = wl.boxes[0]
    x, u, w = b.particles[0]
    st = oracle.State(n, n, n, wl.dt, species=[oracle.Species(-1.0, 1.0, 2, x, u, w)], rho_bg=b.rho_bg)
    t0 = time.perf_counter()
    st.step(steps)
    dt = time.perf_counter() - t0
    return {"value": x.shape[0] * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"thermal_tsc recipe on a {n}^3 box ({x.shape[0]} particles, TSC, 8 ppc), "
                      f"{steps} full steps, single-threaded FP64 C oracle ({dt:.1f} s)",
            "cpu": cpu_model(), "threads_used": 1}


# Arm CPU part numbers (/proc/cpuinfo "CPU part") of the hosts this may run on
ARM_PARTS = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
             "0xd49": "Arm Neoverse-N2", "0xd84": "Arm Neoverse-V3"}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo; Arm part numbers
    are named), its architecture, and the cores this process may run on."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    if not name:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    key = line.split(":", 1)[0].strip().lower()
                    if key in ("model name", "cpu part", "hardware"):
                        v = line.split(":", 1)[1].strip()
                        name = ARM_PARTS.get(v, v)
                        break
        except Exception:  # noqa: BLE001
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001
        usable = os.cpu_count()
    return {"model": name or os.uname().machine, "arch": os.uname().machine, "nproc": usable,
            "logical_cpus": os.cpu_count()}


def run_batched(args, pic, torch, sc, threads, hbm, rank=0, world=1, dist=None):
    """Batched uneven boxes: 64 periodic boxes of edge 16..96 and 1..16 ppc in
    one context (one launch per stage for all boxes) against the plain FP64
    form (one box per launch), push+deposit rate of each.  With several ranks
    the boxes are partitioned over them (no data exchange) and the rate is
    all particles / slowest rank."""
    from paper_1606_02862_gb300 import shard
    from paper_1606_02862_gb300 import workloads as W

    allb = list(W.iter_batched_uneven())
    costs = [shard.box_cost(b[0] ** 3, b[3].shape[0]) for b in allb]
    mine = shard.partition(costs, world)[rank]
    boxes = [allb[i] for i in mine]
    del allb
    grids = [(b[0],) * 3 for b in boxes]
    npart_mine = sum(b[3].shape[0] for b in boxes)
    npart, ncell = shard.sum_over_ranks([npart_mine, sum(b[0] ** 3 for b in boxes)], dist,
                                        device="cuda")
    npart, ncell = int(npart), int(ncell)
    out = {"workload": f"batched_uneven: {len(boxes)} periodic boxes, edges 16..96, ppc 1..16, "
                       f"u_th 0.01..0.1c, TSC ({npart} particles, {ncell} cells)"}
    if getattr(args, "auto", False):
        sc, threads = (0, 0, 0), 0  # libpic tunes on this state at its first step
    for prec, steps, name in ((pic.PRECISION_MIXED, max(10, args.steps // 5), "mixed"),
                              (pic.PRECISION_FP64_PLAIN, 2, "plain_fp64")):
        if prec == pic.PRECISION_FP64_PLAIN and args.no_plain:
            continue
        ctx = pic.Context(grids, (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2)],
                          precision=prec, sc=sc, threads_per_sc=threads)
        for bi, (_n, _ppc, _uth, x, u, w) in enumerate(boxes):
            ctx.set_background(bi, 0.01)
            ctx.load_particles(bi, 0, x, u, w)
        ctx.step(3 if prec == pic.PRECISION_MIXED else 1)
        cfg = ctx.config() if prec == pic.PRECISION_MIXED else None
        ctx.stage_timing(True)
        ctx.step(steps)
        ms, nst = ctx.stage_times()
        ctx.close()
        pd, push_ms, step_ms = shard.max_over_ranks([(ms[0] + ms[1]) / nst, ms[0] / nst, ms[3] / nst],
                                                    dist, device="cuda")
        per_p = MIXED_BYTES_PER_PARTICLE if prec == pic.PRECISION_MIXED else PLAIN_BYTES_PER_PARTICLE
        per_c = MIXED_BYTES_PER_CELL if prec == pic.PRECISION_MIXED else PLAIN_BYTES_PER_CELL
        out[name] = {"value": npart / (pd * 1e-3), "unit": UNIT, "push_deposit_ms": pd,
                     **({"supercell": "x".join(map(str, cfg[0])), "threads": cfg[1]} if cfg else {}),
                     "step_ms": step_ms, "steps": nst,
                     "hbm_frac": (npart * per_p + ncell * per_c) / world / (push_ms * 1e-3) / 1e9 / hbm}
        log(f"[rank {rank}] batched {name}: push+deposit {pd:.3f} ms, step {step_ms:.3f} ms")
    if "plain_fp64" in out:
        out["mixed_over_plain"] = out["mixed"]["value"] / out["plain_fp64"]["value"]
    return out


def run_ours(args, rank, world, dist):
    import torch

    from paper_1606_02862_gb300 import build as libbuild
    from paper_1606_02862_gb300 import pic, shard

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(pic.LIB_PATH):
        libbuild.build()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    n, ppc, u_th = args.n, 8, 0.05
    # --sc auto: zeros, so that libpic tunes supercell and threads on the
    # loaded state at the first (warm-up) step
    args.auto = args.sc == "auto"
    sc, threads = ((0, 0, 0), 0) if args.auto else (tuple(int(v) for v in args.sc.split("x")), args.threads)
    ncell = n ** 3
    t0 = time.perf_counter()
    X, U, Wt = make_state(torch, n, ppc, u_th)
    npart = X.shape[0]
    log(f"[rank {rank}] generated {npart} particles in {time.perf_counter() - t0:.1f} s")

    hbm, hbm_src = measured_hbm()
    result = {}

    # ---------------- mixed form, device-resident inputs, graph replay
    ctx = new_ctx(pic, n, pic.PRECISION_MIXED, sc, threads, SHAPE[args.shape], GATHER[args.gather],
                  args.sort_every)
    t0 = time.perf_counter()
    load(ctx, X, U, Wt)
    log(f"[rank {rank}] loaded in {time.perf_counter() - t0:.1f} s")
    t0 = time.perf_counter()
    ctx.step(args.warmup)
    sc, threads = ctx.config()
    tune_trials = ctx.info(pic.INFO_TUNE_TRIALS)
    args.threads = threads
    args.sc = "x".join(str(v) for v in sc)
    log(f"[rank {rank}] supercell {args.sc}, {threads} threads ({tune_trials} configurations timed by "
        f"libpic's tuner); warm-up {time.perf_counter() - t0:.1f} s")
    ctx.stage_timing(True)
    fused0 = ctx.info(pic.INFO_FUSED_STEPS)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        ctx.step_async(args.steps)
        ev1.record(stream)
        ctx.sync()
        torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    stage_ms, nst = ctx.stage_times()
    graph = bool(ctx.info(pic.INFO_GRAPH_ACTIVE))
    # launches per step of the field update in use (libpic times the fused
    # and the in-place form at the first step and keeps the faster); with
    # the fused one an in-place step (an odd last one) makes two more
    kernels = ctx.info(pic.INFO_KERNELS_PER_STEP)
    field_update = ctx.info(pic.INFO_FIELD_UPDATE)
    fused_in = ctx.info(pic.INFO_FUSED_STEPS) - fused0
    launches = kernels * args.steps + (2 * (args.steps - fused_in) if field_update == pic.FIELD_UPDATE_FUSED else 0)
    assert nst == args.steps, (nst, args.steps)
    ctx.stage_timing(False)
    ctx.close()
    push_ms = stage_ms[0] / args.steps
    frames_ms = stage_ms[1] / args.steps
    yee_ms = stage_ms[2] / args.steps
    step_ms = total_ms / args.steps
    pd_ms = push_ms + frames_ms
    pd_ms_max, step_ms_max = shard.max_over_ranks([pd_ms, step_ms], dist, device="cuda")
    value = world * npart / (pd_ms_max * 1e-3)
    push_bytes = npart * MIXED_BYTES_PER_PARTICLE + ncell * MIXED_BYTES_PER_CELL
    achieved = push_bytes / (push_ms * 1e-3) / 1e9
    # the committed counters hold for the configuration they were taken on
    prof = push_profile() if (args.shape == "tsc" and args.gather == "momentum" and tuple(sc) == (8, 4, 4)
                              and threads in (0, 256)) else {"tpp": None, "wpp": None, "fpp": None,
                                                             "wkind": None}
    tpp = prof["tpp"]
    result.update(value=value, step_ms=step_ms_max, push_ms=push_ms, frames_ms=frames_ms,
                  yee_ms=yee_ms, graph=graph, kernels=kernels, launches=launches, achieved=achieved,
                  field_update="fused two-buffer kernel" if field_update == pic.FIELD_UPDATE_FUSED
                  else "three in-place kernels",
                  traffic=None if tpp is None else tpp * npart, clocks=clk.summary(), wpp=prof["wpp"],
                  wkind=prof["wkind"],
                  fpp=prof["fpp"])
    log(f"[rank {rank}] mixed: push {push_ms:.3f} ms, frames {frames_ms:.3f} ms, yee {yee_ms:.3f} ms,"
        f" step {step_ms:.3f} ms, graph={graph}")

    # ---------------- end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        Xo = torch.empty_like(X, pin_memory=True)
        Uo = torch.empty_like(U, pin_memory=True)
        Wo = torch.empty_like(Wt, pin_memory=True)
        Eo_t = torch.empty((3, n, n, n), dtype=torch.float64, pin_memory=True)
        Eo = Eo_t.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = new_ctx(pic, n, pic.PRECISION_MIXED, sc, args.threads, SHAPE[args.shape], GATHER[args.gather])
        t1 = time.perf_counter()
        load(ctx, X, U, Wt)
        t2 = time.perf_counter()
        ctx.step(args.steps)
        t3 = time.perf_counter()
        nout = ctx.read_particles_ptr(0, 0, npart, Xo.data_ptr(), Uo.data_ptr(), Wo.data_ptr())
        ctx.read_fields_ptr(0, pic.FIELD_E, Eo.ctypes.data)
        t_e2e = time.perf_counter() - t0
        log(f"[rank {rank}] e2e phases: create {t1 - t0:.3f} s, load {t2 - t1:.3f} s, "
            f"{args.steps} steps {t3 - t2:.3f} s, read back {t0 + t_e2e - t3:.3f} s")
        ctx.close()
        h2d = npart * 56.0
        d2h = nout * 56.0 + Eo.nbytes
        result["e2e"] = {"value": world * npart * args.steps / t_e2e, "unit": UNIT,
                         "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                         "seconds": t_e2e,
                         "what": "pic_create + pic_load_particles (pinned FP64 host) + K x pic_step "
                                 "+ pic_read_particles + pic_read_fields(E), wall clock"}
        log(f"[rank {rank}] e2e {t_e2e:.2f} s")
        del Xo, Uo, Wo

    # ---------------- plain FP64 GPU form, same workload
    if not args.no_plain:
        ctx = new_ctx(pic, n, pic.PRECISION_FP64_PLAIN, sc, 0, SHAPE[args.shape], GATHER[args.gather])
        load(ctx, X, U, Wt)
        ctx.step(1)
        ctx.stage_timing(True)
        ctx.step(args.plain_steps)
        ms, nst = ctx.stage_times()
        ctx.close()
        p_ms = ms[0] / nst
        p_bytes = npart * PLAIN_BYTES_PER_PARTICLE + ncell * PLAIN_BYTES_PER_CELL
        result["plain"] = {"value": world * npart / (p_ms * 1e-3), "unit": UNIT,
                           "push_ms": p_ms, "step_ms": ms[3] / nst, "steps": nst,
                           "hbm_frac": p_bytes / (p_ms * 1e-3) / 1e9 / hbm,
                           "bytes_per_particle": PLAIN_BYTES_PER_PARTICLE}
        log(f"[rank {rank}] plain fp64: push {p_ms:.2f} ms")

    # ---------------- batched uneven boxes, mixed vs plain
    if not args.no_batched:
        del X, U, Wt
        result["batched"] = run_batched(args, pic, torch, sc, threads, hbm, rank, world, dist)
        if world > 1:
            result["batched"]["parallelism"] = f"boxes partitioned over {world} ranks"
            result["batched"]["scaling"] = "strong"

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": result["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": result["step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": thermal_workload_name(args, n, ppc),
                   "form": f"mixed: int32 cell + FP32 offsets, supercell frames {args.sc}, "
                           f"{args.threads} threads/supercell"
                           + (f" (tuned by libpic over {tune_trials} configurations)" if tune_trials else ""),
                   "graph": result["graph"],
                   "field_update": result["field_update"],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (particles 4.3 GB/GPU)"},
        "push_deposit_ms_per_step": result["push_ms"] + result["frames_ms"],
        "stage_ms_per_step": {"push_deposit_kernel": result["push_ms"],
                              "frame_maintenance": result["frames_ms"], "yee": result["yee_ms"]},
        "full_step_rate": world * npart / (result["step_ms"] * 1e-3),
        "roofline": {"bound": "hbm", "achieved": result["achieved"], "peak": hbm, "unit": "GB/s",
                     "frac": result["achieved"] / hbm, "traffic": result["traffic"],
                     "kernel": "k_push_deposit", "peak_source": hbm_src,
                     "bytes_per_launch": npart * MIXED_BYTES_PER_PARTICLE + ncell * MIXED_BYTES_PER_CELL},
        "binding": binding_roofline(result, npart),
        "alu": alu_roofline(result, npart),
        "gpu_launches": int(result["launches"]),
        "clocks": result["clocks"],
    }
    if "plain" in result:
        line["plain_fp64"] = result["plain"]
    if "e2e" in result:
        line["e2e"] = result["e2e"]
    if "batched" in result:
        line["batched"] = result["batched"]
    if world == 1 and not args.no_legs:
        # short runs of the other synthetic configurations, so that one
        # default run records them all (each after its own warm-up)
        line["workloads"] = {}
        for name, plain in (("small_cic_32", 5), ("laser_ramp", 2), ("foil_overdense", 2), ("khi_128", 2)):
            leg = workload_leg(name, args.leg_steps, 3, plain_steps=plain)
            line["workloads"][name] = leg
            log(f"leg {name}: {leg['value']:.3e} {UNIT}, push+deposit {leg['push_deposit_ms']:.3f} ms, "
                f"plain FP64 {leg['plain_fp64']['value']:.3e}")
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_oracle()
    return line


# ----------------------------------------------------------------------------- one box over N GPUs

def run_decomposed(args, rank, world, dist):
    """The headline thermal box split into z slabs, one per rank (GPU); per
    step each slab exchanges its J guard planes, the particles leaving
    through its z faces and its E and B planes with the two neighbouring
    slabs (NCCL point-to-point; a one-slab run exchanges with itself).
    Push+deposit time = push kernel + J / migrant exchange + frame
    maintenance, CUDA events on the slab's stream, max over ranks; the rate
    is the whole box's particles over that time (strong scaling: the box is
    fixed, the slabs shrink as N grows)."""
    import torch

    from paper_1606_02862_gb300 import build as libbuild
    from paper_1606_02862_gb300 import decomp, pic, shard
    from paper_1606_02862_gb300 import workloads as W

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(pic.LIB_PATH):
        libbuild.build()
    if dist is not None:
        dist.barrier()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n, ppc, u_th = args.n, 8, 0.05
    sc = (8, 4, 4) if args.sc == "auto" else tuple(int(v) for v in args.sc.split("x"))
    threads = args.threads or 256
    layout = decomp.SlabLayout(n, world, sc[2])
    z0, nzl = layout.extent(rank)
    m = n * n * nzl * ppc
    X = torch.empty((m, 3), dtype=torch.float64, pin_memory=True)
    U = torch.empty((m, 3), dtype=torch.float64, pin_memory=True)
    Wt = torch.empty((m,), dtype=torch.float64, pin_memory=True)
    W.fill_thermal(X.numpy(), U.numpy(), Wt.numpy(), n, n, n, ppc, u_th, z_lo=z0, z_hi=z0 + nzl)
    X[:, 2] -= z0
    ring = decomp.DistRing(dist) if dist is not None else decomp.LocalRing(1)

    def new_slab():
        ctx = pic.Context([(n, n, nzl)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT,
                          [pic.Species(-1.0, 1.0, SHAPE[args.shape], True, GATHER[args.gather])],
                          sc=sc, threads_per_sc=threads, use_graph=False)
        ctx.set_background(0, 0.01)
        slab = decomp.LibpicSlab(ctx)
        load(ctx, X, U, Wt)
        stepper = decomp.SlabStepper([slab], ring, decomp.torch_buffers("cuda"))
        stepper.prime()
        return ctx, stepper

    ctx, stepper = new_slab()
    stepper.step(args.warmup)
    marks = {k: [] for k in ("push", "exchange", "frames", "fields", "end")}

    def mark(label):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        marks[label].append(e)

    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    hbm, hbm_src = measured_hbm()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        stepper.step(args.steps, mark=mark)
        ctx.sync()
        torch.cuda.synchronize()

    def span(a, b):
        return sum(x.elapsed_time(y) for x, y in zip(marks[a], marks[b])) / args.steps

    push_ms, exch_ms = span("push", "exchange"), span("exchange", "frames")
    frames_ms, fields_ms = span("frames", "fields"), span("fields", "end")
    step_ms = span("push", "end")
    pd_ms = push_ms + exch_ms + frames_ms
    pd_max, step_max, push_max = shard.max_over_ranks([pd_ms, step_ms, push_ms], dist, device="cuda")
    npart = n ** 3 * ppc
    mine_bytes = m * MIXED_BYTES_PER_PARTICLE + n * n * nzl * MIXED_BYTES_PER_CELL
    achieved = mine_bytes / (push_ms * 1e-3) / 1e9
    ctx.close()

    # end to end: create, load from pinned host memory, K steps, read back
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    cap = m + m // 4 + 4096  # the slab's count drifts by the particles crossing its faces
    Xo = torch.empty((cap, 3), dtype=torch.float64, pin_memory=True)
    Uo = torch.empty((cap, 3), dtype=torch.float64, pin_memory=True)
    Wo = torch.empty((cap,), dtype=torch.float64, pin_memory=True)
    Eo = torch.empty((3, nzl, n, n), dtype=torch.float64, pin_memory=True).numpy()
    t0 = time.perf_counter()
    ctx, stepper = new_slab()
    stepper.step(args.steps)
    ctx.sync()
    nout = ctx.read_particles_ptr(0, 0, cap, Xo.data_ptr(), Uo.data_ptr(), Wo.data_ptr())
    ctx.read_fields_ptr(0, pic.FIELD_E, Eo.ctypes.data)
    t_e2e = time.perf_counter() - t0
    kernels = ctx.info(pic.INFO_KERNELS_PER_STEP)
    ctx.close()
    (t_max,) = shard.max_over_ranks([t_e2e], dist, device="cuda")
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": npart / (pd_max * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_max, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": thermal_workload_name(args, n, ppc).replace(f"({npart} particles/GPU)",
                                                                           f"({npart} particles)"),
                   "form": f"mixed, supercell {'x'.join(map(str, sc))}, {threads} threads/supercell",
                   "parallelism": f"domain decomposition: {world} z slabs of {layout.extent(0)[1]} "
                                  "planes, NCCL point-to-point halo and particle exchange"
                                  if world > 1 else "one slab exchanging with itself",
                   "l2": "inputs larger than L2"},
        "push_deposit_ms_per_step": pd_max,
        "stage_ms_per_step": {"push_deposit_kernel": push_ms, "j_and_migrant_exchange": exch_ms,
                              "frame_maintenance": frames_ms, "yee_with_exchanges": fields_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "kernel": "k_push_deposit (rank 0's slab)",
                     "peak_source": hbm_src},
        "gpu_launches": int(kernels * args.steps), "clocks": clk.summary(),
        "e2e": {"value": npart * args.steps / t_max, "unit": UNIT,
                "h2d_bytes_per_step": m * 56.0 / args.steps,
                "d2h_bytes_per_step": (nout * 56.0 + Eo.nbytes) / args.steps, "seconds": t_max,
                "what": "per rank: pic_create + load (pinned FP64 host) + K staged steps with exchanges "
                        "+ read back particles and E, wall clock, max over ranks; bytes of rank 0"},
    }


# ----------------------------------------------------------------------------- other workloads

WORKLOADS = {
    "small_cic_32": "32^3 periodic, electrons 2 ppc, u_th 0.01c, B_z 0.1, CIC",
    "laser_ramp": "128x1024x128, e- + p+ 4 ppc each in a density ramp to 0.01 n_c, Gaussian pulse a0 3",
    "foil_overdense": "256x2048x256, 20-cell foil of e- + C6+ at 30 n_c, 16 ppc each, Gaussian pulse a0 10",
    "khi_128": "128^3, e- + p+ 16 ppc each, shear slabs at +-0.2c, TSC (the paper's evaluation size)",
    "laser_window": "128x1024x128, e- + p+ 4 ppc each in a density ramp to 0.01 n_c; open y: 32-cell "
                    "absorbers, particles leaving through y removed, antenna-injected pulse a0 3, moving "
                    "window advanced by 4 cells whenever c t passes them, fresh plasma loaded at the top",
}


def workload_leg(name, steps, warmup, sc=(8, 4, 4), threads=256, plain_steps=0, diag_every=0, log_fn=log):
    """Push+deposit rate of one synthetic workload (mixed form, graph replay,
    in-graph stage events) as a dict; plain_steps > 0 also times the plain
    FP64 form (the paper runs its KHI case in single and double precision);
    diag_every > 0 records the FP64 diagnostics every diag_every steps (the
    timing then covers the steps between them)."""
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    t0 = time.perf_counter()
    wl = W.khi() if name == "khi_128" else getattr(W, name)()
    log_fn(f"generated {name} in {time.perf_counter() - t0:.1f} s")
    ctx = pic.from_workload(wl, sc=sc, threads_per_sc=threads)
    npart = sum(ctx.count_particles(b, s) for b in range(len(wl.boxes)) for s in range(len(wl.species))
                if wl.species[s].mobile)
    ncell = wl.ncells
    ctx.step(warmup)
    diags = []
    ctx.stage_timing(True)
    if diag_every > 0:
        diags.append([warmup] + ctx.diagnostics(0).tolist())
        for k in range(0, steps, diag_every):
            ctx.step(min(diag_every, steps - k))
            diags.append([warmup + min(k + diag_every, steps)] + ctx.diagnostics(0).tolist())
    else:
        ctx.step(steps)
    ms, nst = ctx.stage_times()
    fused = ctx.info(pic.INFO_FIELD_UPDATE) == pic.FIELD_UPDATE_FUSED
    ctx.close()
    out = {"workload": f"{name}: {WORKLOADS[name]}", "particles": npart, "cells": ncell, "steps": nst,
           "warmup": warmup, "value": npart / ((ms[0] + ms[1]) / nst * 1e-3), "unit": UNIT,
           "push_deposit_ms": (ms[0] + ms[1]) / nst,
           "stage_ms_per_step": {"push_deposit_kernel": ms[0] / nst, "frame_maintenance": ms[1] / nst,
                                 "yee": ms[2] / nst},
           "step_ms": ms[3] / nst,
           "hbm_frac": (npart * MIXED_BYTES_PER_PARTICLE + ncell * MIXED_BYTES_PER_CELL)
           / (ms[0] / nst * 1e-3) / 1e9 / measured_hbm()[0],
           "form": f"mixed, supercell {'x'.join(map(str, sc))}, {threads} threads, "
                   + ("fused two-buffer field update" if fused else "in-place field update")}
    if diags:
        out["diagnostics"] = {"columns": ["step", "field_energy", "kinetic_energy", "charge",
                                          "max_abs_divE_minus_rho"], "rows": diags}
    if plain_steps > 0:
        pctx = pic.from_workload(wl, precision=pic.PRECISION_FP64_PLAIN)
        pctx.step(1)
        pctx.stage_timing(True)
        pctx.step(plain_steps)
        pms, pn = pctx.stage_times()
        pctx.close()
        out["plain_fp64"] = {"value": npart / (pms[0] / pn * 1e-3), "unit": UNIT, "push_ms": pms[0] / pn,
                             "step_ms": pms[3] / pn, "steps": pn,
                             "hbm_frac": (npart * PLAIN_BYTES_PER_PARTICLE + ncell * PLAIN_BYTES_PER_CELL)
                             / (pms[0] / pn * 1e-3) / 1e9 / measured_hbm()[0]}
        out["fp32_over_fp64_step"] = (pms[3] / pn) / (ms[3] / nst)
    del wl
    return out


def run_workload(args):
    """One of the other synthetic workloads as its own JSON line."""
    import torch

    from paper_1606_02862_gb300 import build as libbuild

    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sc = (8, 4, 4) if args.sc == "auto" else tuple(int(v) for v in args.sc.split("x"))
    threads = args.threads or 256
    leg = workload_leg(args.workload, args.steps, args.warmup, sc, threads,
                       plain_steps=0 if args.no_plain or args.workload != "khi_128" else args.plain_steps,
                       diag_every=args.diag_every)
    hbm, hbm_src = measured_hbm()
    line = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": 1,
            "steps": leg["steps"], "warmup": args.warmup, "ms_per_step": leg["step_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{leg['workload']} ({leg['particles']} particles, {leg['cells']} cells)",
                       "form": leg["form"]},
            "stage_ms_per_step": leg["stage_ms_per_step"],
            "roofline": {"bound": "hbm", "achieved": leg["hbm_frac"] * hbm, "peak": hbm, "unit": "GB/s",
                         "frac": leg["hbm_frac"], "traffic": None, "kernel": "k_push_deposit",
                         "peak_source": hbm_src}}
    for k in ("plain_fp64", "fp32_over_fp64_step", "diagnostics"):
        if k in leg:
            line[k] = leg[k]
    return line


def run_yee(args):
    """The field update alone (scope row a5): an n^3 box without particles,
    random E, stage events around the field update of each step.  The
    headline form is the fused two-buffer kernel (PIC_FIELD_UPDATE_FUSED:
    one kernel per step, pairs of steps, so the step count is rounded up to
    an even number); the three in-place kernels (B half, E, B half) are timed
    beside it.  Rate in cell updates/s; roofline against the algorithmic 60
    B/cell of DRAM traffic per field update (E, B, J read, E, B written; the
    in-place kernels move 120: E, B read and B written twice, plus B, E, J
    read and E written)."""
    import torch

    from paper_1606_02862_gb300 import build as libbuild
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n = args.n
    steps = args.steps + (args.steps % 2)
    warm = max(2, args.warmup + (args.warmup % 2))

    def timed(field_update):
        ctx = pic.Context([(n, n, n)], (1.0, 1.0, 1.0), W.DT_HALF_COURANT, [pic.Species(-1.0, 1.0, 2, True)],
                          sc=(8, 4, 4), threads_per_sc=256, use_graph=True, field_update=field_update)
        rng = np.random.default_rng(W.BASE_SEED + 7)
        ctx.write_fields(0, pic.FIELD_E, rng.normal(0.0, 0.01, (3, n, n, n)))
        ctx.step(warm)
        ctx.stage_timing(True)
        ctx.step(steps)
        ms, nst = ctx.stage_times()
        fused = ctx.info(pic.INFO_FUSED_STEPS)
        ctx.close()
        return ms, nst, fused

    ms, nst, fused_steps = timed(pic.FIELD_UPDATE_FUSED)
    ms_ip, nst_ip, _ = timed(pic.FIELD_UPDATE_IN_PLACE)
    yee_ms = ms[2] / nst
    ip_ms = ms_ip[2] / nst_ip
    cells = n ** 3
    hbm, hbm_src = measured_hbm()
    achieved = 60.0 * cells / (yee_ms * 1e-3) / 1e9
    return {"metric": "cell updates/sec of the Yee field update (B half, E, B half) at 1 GB300",
            "value": cells / (yee_ms * 1e-3), "unit": "cell updates/s", "n_gpus": 1, "steps": nst,
            "warmup": warm, "ms_per_step": ms[3] / nst, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"yee_{n}: {n}^3 periodic cells, fields only (random E), FP32, guard-padded",
                       "form": f"fused two-buffer field update ({fused_steps} of {warm + nst} steps)",
                       "l2": "fields larger than L2" if 9 * 4 * cells > 129e6 else "fields fit in L2"},
            "stage_ms_per_step": {"yee": yee_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "kernel": "k_yee_fused",
                         "peak_source": hbm_src, "bytes_per_cell": 60},
            "in_place": {"kernels": "k_yee_b, k_yee_e, k_yee_b", "ms_per_update": ip_ms,
                         "value": cells / (ip_ms * 1e-3), "unit": "cell updates/s",
                         "frac_of_60B": 60.0 * cells / (ip_ms * 1e-3) / 1e9 / hbm,
                         "frac_of_own_120B": 120.0 * cells / (ip_ms * 1e-3) / 1e9 / hbm}}


def run_window(args):
    """The open-boundary laser workload with a moving window: push+deposit
    rate from the in-graph stage events (steps only), and the whole cycle per
    step including the window shifts and the loading of fresh plasma, timed
    with CUDA events around the loop (slabs generated before the timed region)."""
    import torch

    from paper_1606_02862_gb300 import build as libbuild
    from paper_1606_02862_gb300 import pic
    from paper_1606_02862_gb300 import workloads as W

    libbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t0 = time.perf_counter()
    wl = W.laser_window()
    b = wl.boxes[0]
    log(f"generated laser_window in {time.perf_counter() - t0:.1f} s")
    sc = (8, 4, 4) if args.sc == "auto" else tuple(int(v) for v in args.sc.split("x"))
    threads = args.threads or 256
    ctx = pic.from_workload(wl, sc=sc, threads_per_sc=threads)
    step_cells = sc[1]
    rng = np.random.default_rng(wl.extra["seed"] + 1)
    total = args.warmup + args.steps
    nshift = int(total * wl.dt / step_cells) + 1
    slabs = [W.window_slab(rng, b.nx, b.nz, b.ny - step_cells, b.ny, wl.extra["ppc"], wl.extra["density"],
                           y_shift=float((k + 1) * step_cells)) for k in range(nshift)]
    state = {"shifts": 0}

    def advance(k):
        ctx.step_async(1)
        if (k + 1) * wl.dt >= (state["shifts"] + 1) * step_cells:
            ctx.shift_window(0, step_cells)
            for si, (x, u, w) in enumerate(slabs[state["shifts"]]):
                ctx.load_particles(0, si, x, u, w)
            state["shifts"] += 1

    for k in range(args.warmup):
        advance(k)
    ctx.sync()
    npart = sum(ctx.count_particles(0, s) for s in range(2))
    shifts0 = state["shifts"]
    ctx.stage_timing(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.warmup, total):
        advance(k)
    e1.record(stream)
    torch.cuda.synchronize()
    cycle_ms = e0.elapsed_time(e1) / args.steps
    ms, nst = ctx.stage_times()
    npart1 = sum(ctx.count_particles(0, s) for s in range(2))
    ctx.close()
    del wl, slabs
    npart_avg = 0.5 * (npart + npart1)
    pd = (ms[0] + ms[1]) / nst
    hbm, hbm_src = measured_hbm()
    achieved = (npart_avg * MIXED_BYTES_PER_PARTICLE + b.ncells * MIXED_BYTES_PER_CELL) / (ms[0] / nst * 1e-3) / 1e9
    return {"metric": METRIC, "value": npart_avg / (pd * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": nst, "warmup": args.warmup, "ms_per_step": ms[3] / nst, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"laser_window: {WORKLOADS['laser_window']} (~{int(npart_avg)} particles, "
                                   f"{b.ncells} cells)",
                       "form": f"mixed, supercell {'x'.join(map(str, sc))}, {threads} threads"},
            "stage_ms_per_step": {"push_deposit_kernel": ms[0] / nst, "frame_maintenance": ms[1] / nst,
                                  "yee_and_absorber": ms[2] / nst},
            "window": {"shifts": state["shifts"] - shifts0, "cycle_ms_per_step": cycle_ms,
                       "what": "CUDA events around the loop: steps, window shifts and fresh-plasma loads "
                               "from host FP64 arrays"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "kernel": "k_push_deposit",
                         "peak_source": hbm_src}}


# ----------------------------------------------------------------------------- reference arm

def thermal_workload_name(args, n, ppc=8):
    """The config.workload string of the thermal benchmark (both arms)."""
    return (f"thermal_{args.shape}_{n}: {n}^3 periodic cells, electrons {ppc} ppc "
            f"({n ** 3 * ppc} particles/GPU), u_th 0.05c, {args.shape.upper()}, "
            "dt = 0.5 Courant, neutralising background"
            + (", energy-conserving gather" if args.gather == "energy" else ""))


def run_reference(args, rank):
    """The FP64 oracle as it stands, on this host's cores: each step is one
    full PIC step of a bounded sample (16^3 box, same recipe)."""
    if rank != 0:
        return None
    import oracle
    from paper_1606_02862_gb300 import workloads as W

    oracle.build()
    n = 16
    wl = W.thermal_tsc(n=n, ppc=8, u_th=0.05)
    b = wl.boxes[0]
    x, u, w = b.particles[0]
    st = oracle.State(n, n, n, wl.dt, species=[oracle.Species(-1.0, 1.0, 2, x, u, w)], rho_bg=b.rho_bg)
    st.step(args.warmup)
    t0 = time.perf_counter()
    st.step(args.steps)
    dt = time.perf_counter() - t0
    v = x.shape[0] * args.steps / dt
    sample = (f"thermal_tsc recipe on a {n}^3 box ({x.shape[0]} particles, TSC, 8 ppc) per step, "
              "single-threaded FP64 C oracle")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": thermal_workload_name(args, args.n),
                       "form": "FP64 CPU oracle, one host thread; each step a bounded sample (see cpu_baseline)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="box edge in cells")
    ap.add_argument("--sc", default="auto", help="supercell edges, e.g. 8x8x4, or auto")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the short runs of the other configurations in the default line")
    ap.add_argument("--leg-steps", type=int, default=20)
    ap.add_argument("--sort-every", type=int, default=0,
                    help="steps between sort passes of the push (0: the library's default, 4)")
    ap.add_argument("--diag-every", type=int, default=0,
                    help="--workload runs: FP64 diagnostics every this many steps")
    ap.add_argument("--shape", default="tsc", choices=["tsc", "cic", "pcs"],
                    help="particle shape of the headline thermal workload")
    ap.add_argument("--gather", default="momentum", choices=["momentum", "energy"],
                    help="gather variant of the headline thermal workload")
    ap.add_argument("--decomp", action="store_true",
                    help="one box split into z slabs over the ranks (the default with --gpus > 1); "
                         "with one GPU the single slab exchanges with itself")
    ap.add_argument("--replicas", action="store_true",
                    help="with --gpus > 1: one independent box per rank instead of one decomposed box")
    ap.add_argument("--workload", default="thermal_tsc_256",
                    choices=["thermal_tsc_256", "small_cic_32", "laser_ramp", "foil_overdense",
                             "khi_128", "laser_window", "yee"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.shape == "pcs":
        args.no_plain = True  # the plain FP64 form has CIC and TSC only

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        if args.impl == "ours":
            import torch

            # each rank's GPU before the NCCL group forms, so that its
            # communicator binds to that device
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist_mod.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = dist_mod
    if args.impl == "reference":
        line = run_reference(args, rank)
    elif args.workload == "laser_window":
        line = run_window(args) if rank == 0 else None
    elif args.workload == "yee":
        line = run_yee(args) if rank == 0 else None
    elif args.workload != "thermal_tsc_256":
        line = run_workload(args) if rank == 0 else None
    elif args.decomp or (world > 1 and not args.replicas):
        line = run_decomposed(args, rank, world, dist)
    else:
        line = run_ours(args, rank, world, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
