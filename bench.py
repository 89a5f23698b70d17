#!/usr/bin/env python3
"""Trotter steps/s and HBM roofline of the 27-qubit gauge-Higgs evolution on GB300.

Workload: 3x3 periodic gauge-Higgs lattice (18 link + 9 vertex = 27 qubits),
complex64 state (1.07 GB, larger than L2), H(s) = (1-s) H0 + s H1 with
J = h = 1, (g, lambda) = (0.6, 0.6), linear ramp over T = 20 in 1000 second-order
Trotter steps (dt = 0.02); the timed steps are a window of that schedule.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  `value` = Trotter steps/s over all ranks (each rank
evolves its own replica: the single-state path does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="gh3x3_27q_c64_fused_order2", Lx=3, Ly=3, form="gh", dtype="c64",
                g=0.6, lam=0.6, T=20.0, total_steps=1000, order=2)
METRIC = "trotter_steps_per_sec"
UNIT = "steps/s"


def linear_midpoints(T, n):
    # s_k = t_k / T at t_k = (k - 1/2) dt: a schedule input, computed identically by the oracle
    dt = T / n
    return (np.arange(1, n + 1) - 0.5) * dt / T


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_config(world: int) -> dict:
    """The bench workload's `config` (the same for both arms)."""
    W = WORKLOAD
    return {"workload": W["name"], "lattice": "3x3 periodic", "form": "gauge-Higgs", "qubits": 27,
            "g": W["g"], "lambda": W["lam"], "J": 1.0, "h": 1.0, "T": W["T"], "dt": W["T"] / W["total_steps"],
            "order": W["order"], "state_bytes": 8 << 27,
            "l2": "inputs larger than L2 (1.07 GB state, 129 MB L2)",
            "parallelism": "replicas" if world > 1 else "single"}


def kernel_source_hash(kernel_name: str = "") -> str:
    """sha256 (16 hex digits) of the X-pass kernel sources (the warp-local shared pass
    adds its own header)."""
    import hashlib
    d = hashlib.sha256()
    files = ["kernels.cuh", "xpass_tma.cuh"] + (["xpass_wl.cuh"] if kernel_name.startswith("k_xpass_wl") else [])
    for f in files:
        d.update(open(os.path.join(ROOT, "paper_2108_13410_gb300", "csrc", f), "rb").read())
    return d.hexdigest()[:16]


def profile_traffic(kernel_tag: str, kernel_name: str = ""):
    """dram read+write bytes per launch from the committed ncu summary, if it was
    taken on the current kernel source and on the same kernel instantiation (the
    summary's first line starts with its name)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.txt")
    if not os.path.exists(path):
        return None
    if kernel_name and not open(path).readline().startswith(kernel_name):
        return None
    h = kernel_source_hash(kernel_name)
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != h:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND") != "gloo" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_throughput(world: int, steps_per_rank: int, ms_max: float) -> float:
    """Whole-job steps/s: every rank evolves its own replica for steps_per_rank steps;
    the job takes as long as the slowest rank."""
    return world * steps_per_rank / (ms_max / 1000.0)


def max_over_ranks(world, x: float, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(budget_s: float, max_steps: float = 1e9):
    """Time the FP64 oracle on the 27-qubit workload for about budget_s seconds.

    The oracle applies the Trotter step factor by factor (81 Pauli factors per
    second-order step at 27 qubits); a bounded sample is a run of whole factors,
    scaled to steps.  Returns (steps_per_s, cores, description)."""
    from oracle import OracleLattice, Couplings
    from oracle import core as O
    lat = OracleLattice(WORKLOAD["Lx"], WORKLOAD["Ly"], True, WORKLOAD["form"])
    c = Couplings(WORKLOAD["g"], WORKLOAD["lam"])
    n = lat.n_qubits
    dt = WORKLOAD["T"] / WORKLOAD["total_steps"]
    s = linear_midpoints(WORKLOAD["T"], WORKLOAD["total_steps"])
    psi = O.plus_state(n)
    xs, zs = O._terms(lat)
    factors = []                                    # one second-order step: X/2, Z, X/2
    coef = O.coefficients(c, float(s[0]))
    factors += [(k, t, coef[key] * 0.5 * dt) for k, t, key in xs]
    factors += [(k, t, coef[key] * dt) for k, t, key in zs]
    factors += [(k, t, coef[key] * 0.5 * dt) for k, t, key in xs]
    per_step = len(factors)
    done = 0
    t0 = time.perf_counter()
    while True:
        k, tgt, th = factors[done % per_step]
        O._apply(psi, n, k, tgt, th)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s or done >= max_steps * per_step:
            break
    steps = done / per_step
    return steps / el, O.max_threads(), (f"{done} Pauli factors ({steps:.3f} second-order steps) of the "
                                         f"27-qubit workload, FP64, {el:.1f} s")


def run_reference(args):
    world, rank, local = dist_setup(args.gpus)
    if rank != 0:
        return 0
    # warm-up: one factor-sized sample per warm-up step
    budget_total = 150.0
    per = budget_total / max(1, args.steps + args.warmup)
    oracle_sample(min(per, 2.0))
    rates, descs = [], []
    for _ in range(args.steps):
        r, cores, d = oracle_sample(per)
        rates.append(r)
        descs.append(d)
    value = float(np.mean(rates))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(1),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step: {descs[-1]}"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2108_13410_gb300 import Simulator, QS_OPT_PROFILE
    from paper_2108_13410_gb300 import qsim as Q

    W = WORKLOAD
    dt = W["T"] / W["total_steps"]
    sched = linear_midpoints(W["T"], W["total_steps"])
    K, Wu = args.steps, args.warmup
    assert K + Wu <= W["total_steps"], "steps + warmup must fit the 1000-step schedule"
    cpl = [(W["g"], W["lam"])]
    sim = Simulator(W["Lx"], W["Ly"], form=W["form"], dtype=W["dtype"], device=f"cuda:{local}")
    stream = torch.cuda.current_stream(dev)
    # autotuner: pass plan (qubits fused per X pass), then the X-pass kernel configuration
    if args.no_autotune:
        from paper_2108_13410_gb300.qsim import qs_plan
        tune = {"plan": qs_plan(sim.h), "xpass": 0, "buffers": 3, "store": 1, "shared_buffers": 0,
                "shared_kernel": 1, "ms_per_step": None}
    else:
        tune = sim.autotune(n_steps=20, cache=False)
    sim.init_plus()
    # warm-up
    sim.evolve(cpl, sched[:Wu], dt, W["order"])
    torch.cuda.synchronize(dev)
    sim.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.evolve(cpl, sched[Wu:Wu + K], dt, W["order"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = e0.elapsed_time(e1)
    launches = sim.launch_count()
    # per-kernel launch durations: the same K steps once more with CUDA events around
    # every X-pass launch on the launching stream (the events break the programmatic
    # overlap of consecutive launches, so they stay out of the timed region above)
    sim.set_option(QS_OPT_PROFILE, 1)
    sim.profile_read()
    sim.evolve(cpl, sched[Wu:Wu + K], dt, W["order"])
    torch.cuda.synchronize(dev)
    kinds = sim.profile_read_kinds()          # (single-group passes, shared passes)
    sim.set_option(QS_OPT_PROFILE, 0)
    clk = clocks.stop()
    ms_max = max_over_ranks(world, ms, dev)
    value = job_throughput(world, K, ms_max)

    state_bytes = sim.state_bytes
    alg_bytes = 2.0 * state_bytes                     # one read + one write of the state per pass
    peak, peak_kind = peaks()
    # the two X-pass kernels the tuned configuration runs (tangent form; shared passes
    # default to two tile buffers in the gauge-Higgs form)
    tb = lambda v: "true" if v else "false"
    names = ("k_xpass_tma<%d, %s, false, true>" % (tune["buffers"], tb(tune["store"])),
             "k_xpass_tma<%d, %s, true, true>" % (tune["shared_buffers"] or 2, tb(tune["store"])))
    tags = ("k_xpass_tma_c64_27q", "k_xpass_tma_shared_c64_27q")
    if tune["shared_kernel"] == 1 and tune["store"]:  # warp-local shared passes
        geom = {0: "6, 24, 1, false", 2: "2, 8, 3, false", 3: "3, 8, 2, false"}[tune["shared_buffers"]]
        names = (names[0], "k_xpass_wl<%s>" % geom)
        tags = (tags[0], "k_xpass_wl_c64_27q")
    if tune["xpass"] == 1:                            # the register-staged kernel (no shared passes)
        names = ("k_xpass<float>", "k_xpass<float>")
    dom = 0 if kinds[0][0] >= kinds[1][0] else 1     # dominant kernel: larger total time
    per_kind = {}
    for kd in (0, 1):
        kms, kn = kinds[kd]
        if kn:
            per_kind[names[kd]] = {"launches": kn, "avg_launch_ms": kms / kn,
                                   "achieved_gbs": alg_bytes / (kms / kn / 1000.0) / 1e9,
                                   "share_of_xpass_time": kms / max(1e-12, kinds[0][0] + kinds[1][0])}
    xpass_n = kinds[0][1] + kinds[1][1]
    avg_ms = kinds[dom][0] / max(1, kinds[dom][1])
    achieved = alg_bytes / (avg_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": profile_traffic(tags[dom], names[dom]),
                "kernel": names[dom], "launches": kinds[dom][1], "avg_launch_ms": avg_ms,
                "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind,
                "launch_timing": "CUDA events around each X-pass launch on its stream, over a repeat "
                                 "of the timed steps",
                "xpass_kernels": per_kind, "passes_per_step": xpass_n / K,
                "step_hbm_gbs": (xpass_n / K) * alg_bytes / (ms / K / 1000.0) / 1e9}

    # ---- end to end through the public API with host buffers ----
    host_state = torch.empty(sim.state.shape, dtype=sim.state.dtype, pin_memory=True)
    host_state[0].fill_(2 ** (-sim.n / 2))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim.upload(host_state)                                   # h2d: initial state
    sim.evolve(cpl, sched[Wu:Wu + K], dt, W["order"])        # h2d: per-step operator records
    e_fin = sim.energy(cpl)                                  # d2h: reduction records
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(world, e2e_s, dev)
    e2e = {"value": world * K / e2e_s, "unit": UNIT,
           # initial state + the schedule value of every step + one coupling record
           "h2d_bytes_per_step": (state_bytes + 8 * K + 32) / K,
           "d2h_bytes_per_step": (1 + sim.n) * 4 * 8 / K,
           "final_energy": float(e_fin[0])}

    extra = {}
    if rank == 0 and not args.no_pergate:
        # the plain complex128 per-gate form on the same GPU, a few steps
        del host_state
        torch.cuda.empty_cache()
        sp = Simulator(W["Lx"], W["Ly"], form=W["form"], dtype="c128", device=f"cuda:{local}", method="pergate")
        sp.init_plus()
        sp.evolve(cpl, sched[:1], dt, W["order"])
        torch.cuda.synchronize(dev)
        kp = 3
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        sp.evolve(cpl, sched[1:1 + kp], dt, W["order"])
        a1.record(stream)
        torch.cuda.synchronize(dev)
        pg = kp / (a0.elapsed_time(a1) / 1000.0)
        extra["pergate_c128"] = {"value": pg, "unit": UNIT, "steps": kp,
                                 "fused_c64_speedup": value / world / pg}
        del sp
        torch.cuda.empty_cache()
        # the fused complex128 passes (the paper's precision): double-float arithmetic
        # (default) and FP64, each over one call of kf steps
        from paper_2108_13410_gb300.qsim import QS_OPT_C128_DF
        fused = {}
        for name, df, kf in (("double_float", 1, 40), ("fp64", 0, 10)):
            sf = Simulator(W["Lx"], W["Ly"], form=W["form"], dtype="c128", device=f"cuda:{local}")
            sf.set_option(QS_OPT_C128_DF, df)
            sf.init_plus()
            sf.evolve(cpl, sched[:3], dt, W["order"])
            torch.cuda.synchronize(dev)
            a0.record(stream)
            sf.evolve(cpl, sched[3:3 + kf], dt, W["order"])
            a1.record(stream)
            torch.cuda.synchronize(dev)
            fused[name] = {"value": kf / (a0.elapsed_time(a1) / 1000.0), "unit": UNIT, "steps": kf}
            del sf
            torch.cuda.empty_cache()
        fused["double_float"]["over_pergate"] = fused["double_float"]["value"] / pg
        extra["fused_c128"] = fused

    if rank == 0 and not args.no_accuracy:
        extra["accuracy"] = accuracy_leg(local, dev)

    if rank == 0 and not args.no_scan:
        extra["scan"] = scan_leg(local, dev)

    if rank == 0 and args.adjoint_steps > 0:
        extra["adjoint"] = adjoint_leg(args.adjoint_steps, local, dev, stream)

    if rank == 0 and not args.no_ug32:
        extra["ug32"] = ug32_leg(local, dev, stream)

    if rank == 0 and not args.no_protocol:
        extra["protocol"] = protocol_leg(local, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, cores, desc = oracle_sample(args.cpu_budget)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
               "warmup": Wu, "ms_per_step": ms_max / K, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
               "config": workload_config(world),
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk,
               "tuning": {"plan_qubits_per_pass": tune["plan"], "xpass_kernel": tune["xpass"],
                          "tile_buffers": tune["buffers"], "bulk_store": tune["store"],
                          "shared_pass_buffers": tune["shared_buffers"],
                          "shared_pass_kernel": "warp-local" if tune["shared_kernel"] == 1 else "cta-staged",
                          "tuned_ms_per_step": tune["ms_per_step"]}}
        out.update(extra)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def accuracy_leg(local, dev, n_steps=1000):
    """Error of the complex64 27-qubit evolution against the FP64 oracle over the full
    1000-step schedule.  The oracle runs the 18-qubit unitary-gauge image: a
    gauge-invariant gauge-Higgs state restricted to tau = 0 and scaled by 2^{9/2} is
    the unitary-gauge state, and both have the same energy."""
    import torch
    from oracle import OracleLattice, Couplings
    from oracle import core as O
    from paper_2108_13410_gb300 import Simulator
    W = WORKLOAD
    dt = W["T"] / W["total_steps"]
    s = linear_midpoints(W["T"], W["total_steps"])[:n_steps]
    cpl = [(W["g"], W["lam"])]
    ug = OracleLattice(W["Lx"], W["Ly"], True, "ug")
    c = Couplings(W["g"], W["lam"])
    t0 = time.perf_counter()
    ref = O.evolve(ug, c, s, dt, W["order"])
    e_ref = O.energy(ref, ug, c)
    oracle_s = time.perf_counter() - t0
    out = {"steps": n_steps, "oracle": "18-qubit unitary-gauge FP64 oracle", "oracle_seconds": oracle_s,
           "oracle_energy": e_ref}
    for renorm in (0, 50):
        sim = Simulator(W["Lx"], W["Ly"], form=W["form"], dtype="c64", device=f"cuda:{local}",
                        renorm_every=renorm)
        sim.init_plus()
        sim.evolve(cpl, s, dt, W["order"])
        e = float(sim.energy(cpl)[0])
        sl = sim.state[0, : 1 << 18].to(torch.complex128).cpu().numpy() * 2 ** 4.5
        rel = float(np.linalg.norm(sl - ref) / np.linalg.norm(ref))
        mx = float(np.max(np.abs(sl - ref)) / np.max(np.abs(ref)))
        out[f"c64_renorm{renorm}"] = {"amp_rel_l2": rel, "amp_rel_max": mx, "energy": e,
                                     "energy_abs_err": abs(e - e_ref)}
        del sim
        torch.cuda.empty_cache()
    return out


def scan_leg(local, dev, slots=304, baseline_points=4):
    """Phase-diagram scan: 1024 (g, lambda) points on a 32 x 32 grid of [0, 1.5]^2, even flat
    index -> 2x2 periodic gauge-Higgs (12 qubits), odd -> 3x2 open unitary gauge (17
    qubits), all in one persistent launch (qs_scan_mixed: a 12-qubit point on chip, a
    17-qubit point on its CTA's scratch slot), replayed as a CUDA graph; complex64, linear
    ramp T = 10, 200 second-order steps.  Reported next to the same points run one at a
    time through qs_evolve and the observables (per-point launches, a few points timed)."""
    import torch
    import synth
    from paper_2108_13410_gb300 import Simulator, QS_OPT_GRAPH, QS_ENERGY
    from paper_2108_13410_gb300.qsim import qs_scan_mixed
    grid = synth.coupling_grid(32, 0.0, 1.5)
    pts = [tuple(p) for p in grid]
    even, odd = pts[0::2], pts[1::2]
    T, n = 10.0, 200
    s = linear_midpoints(T, n)
    out = {"points": len(pts), "steps": n, "T": T, "launches": 1, "graph": True}
    sim12 = Simulator(2, 2, form="gh", dtype="c64", device=f"cuda:{local}")
    sim17 = Simulator(3, 2, form="ug", dtype="c64", boundary="open", batch=slots, device=f"cuda:{local}")
    sim17.set_option(QS_OPT_GRAPH, 1)
    qs_scan_mixed(sim12.h, even, sim17.h, odd, s, T / n, 2)          # warm-up (captures the graph)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r12, r17 = qs_scan_mixed(sim12.h, even, sim17.h, odd, s, T / n, 2)
    sec = time.perf_counter() - t0
    state17 = 8 << 17
    out.update({"seconds": sec, "point_steps_per_s": len(pts) * n / sec,
                "amplitude_updates_per_s": (len(even) * 4096 + len(odd) * (1 << 17)) * n / sec,
                "scratch_slots": slots,
                # 17-qubit points: two Walsh-Hadamard passes per factor group, each a read
                # and a write of the 1 MiB state (L2-resident slots)
                "state_traffic_gbs_17q": len(odd) * (n + 1) * 2 * 2 * state17 / sec / 1e9,
                "energy_range_12q": [float(r12[:, 0].min()), float(r12[:, 0].max())],
                "energy_range_17q": [float(r17[:, 0].min()), float(r17[:, 0].max())]})
    # per-point launches: each point through qs_evolve (one launch per pass) and the energy
    base = {}
    for name, sim, plist in (("gh2x2_12q", Simulator(2, 2, form="gh", dtype="c64", device=f"cuda:{local}"), even),
                             ("ug3x2open_17q", Simulator(3, 2, form="ug", dtype="c64", boundary="open",
                                                         device=f"cuda:{local}"), odd)):
        sim.init_plus()
        sim.evolve([plist[0]], s[:3], T / n, 2)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for p in plist[:baseline_points]:
            sim.init_plus()
            sim.evolve([p], s, T / n, 2)
            sim.expect(QS_ENERGY, 0, [p], 1.0)
        el = time.perf_counter() - t0
        base[name] = {"points_timed": baseline_points, "seconds_per_point": el / baseline_points,
                      "point_steps_per_s": baseline_points * n / el}
        del sim
    out["per_point_launches"] = base
    out["speedup_vs_per_point_launches"] = (out["point_steps_per_s"] / (len(pts) * n / (
        len(even) * base["gh2x2_12q"]["seconds_per_point"] + len(odd) * base["ug3x2open_17q"]["seconds_per_point"])))
    del sim12, sim17
    torch.cuda.empty_cache()
    return out


def ug32_leg(local, dev, stream):
    """4x4 torus in the unitary gauge: 32 link qubits, complex64 (32 GiB) and complex128
    (64 GiB) states, (g, lambda) = (0.5, 0.5), J = h = 1, linear ramp T = 20, dt = 0.02,
    second order; steps from the start of the 1000-step schedule after two warm-up
    steps.  Reports steps/s, X passes per step and the mean GB/s of each X-pass kernel
    (2 x state bytes per launch, CUDA events) against the measured HBM peak."""
    import torch
    from paper_2108_13410_gb300 import Simulator, QS_OPT_PROFILE, QS_NORM
    s = linear_midpoints(20.0, 1000)
    cpl = [(0.5, 0.5)]
    peak, _ = peaks()
    out = {"lattice": "4x4 periodic", "form": "unitary gauge", "qubits": 32, "g": 0.5, "lambda": 0.5,
           "dt": 0.02, "order": 2}
    from paper_2108_13410_gb300.qsim import QS_OPT_C128_DF
    # complex128: the double-float passes (default) and the FP64 register kernel
    # one call of n steps each (the schedule's 1000 steps run as one call; every call adds
    # the passes of its first and last factor groups)
    for key, dtype, n, df in (("c64", "c64", 30, 1), ("c128", "c128", 20, 1), ("c128_fp64", "c128", 2, 0)):
        sim = Simulator(4, 4, form="ug", dtype=dtype, device=f"cuda:{local}")
        if dtype == "c128":
            sim.set_option(QS_OPT_C128_DF, df)
        sim.init_plus()
        sim.evolve(cpl, s[:2], 0.02, 2)
        torch.cuda.synchronize(dev)
        sim.set_option(QS_OPT_PROFILE, 1)
        sim.profile_read_kinds()
        sim.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.evolve(cpl, s[2:2 + n], 0.02, 2)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        kinds = sim.profile_read_kinds()
        launches = sim.launch_count()
        sim.set_option(QS_OPT_PROFILE, 0)
        alg = 2.0 * sim.state_bytes
        kern = {}
        for name, (kms, kn) in zip(("plain", "shared"), kinds):
            if kn:
                gbs = alg / (kms / kn / 1000.0) / 1e9
                kern[name] = {"launches": kn, "avg_launch_ms": kms / kn, "achieved_gbs": gbs, "frac": gbs / peak}
        npass = kinds[0][1] + kinds[1][1]
        out[key] = {"steps": n, "steps_per_s": n / (ms / 1000.0), "ms_per_step": ms / n,
                    "state_bytes": sim.state_bytes, "passes_per_step": npass / n, "launches": launches,
                    "xpass": kern, "step_hbm_gbs": npass * alg / (ms / 1000.0) / 1e9,
                    "norm_minus_1": float(sim.expect(QS_NORM)[0] - 1.0)}
        if key == "c128":
            # the in-place split into the blocked double-float layout and the join back run
            # once per call, inside the time above: the call time minus the X-pass
            # launches' own event times is the split, the join and the launch gaps
            xpass_ms = kinds[0][0] + kinds[1][0]
            out[key]["arithmetic"] = "double-float (two floats per real number, FP32 pipes)"
            out[key]["xpass_ms_per_step"] = xpass_ms / n
            out[key]["split_join_and_gaps_ms_per_call"] = ms - xpass_ms
        elif key == "c128_fp64":
            out[key]["arithmetic"] = "FP64"
        del sim
        torch.cuda.empty_cache()
    return out


def protocol_leg(local, dev):
    """The hysteresis experiment of Sec. IV on the 3x3 unitary-gauge torus (18 qubits,
    J = h = 1/2, dg = 1e-5, dt = 0.02, second order, complex64) at p = 0.12 (deconfined)
    and p = 0.5: psi_1 carried O -> P -> P' and psi_1' carried O -> P' -> P, both energy
    curves sampled along the blue path; E (psi_1 at P) and E' (psi_1' arrived at P) next
    to the printed ones, with the crossing points.  Then the broken red paths of Sec. V
    (r = 0.05, 0.15, 0.25): minimum of d^2E/dg^2 next to the printed one."""
    import torch
    from paper_2108_13410_gb300.reproduce import hysteresis, red_path_curvature
    torch.cuda.synchronize(dev)
    out = {}
    for p in (0.12, 0.5):
        r = hysteresis(p, 1e-5, 0.02)
        r.pop("curve")
        if len(r["crossings"]) > 4:
            r["crossings"] = "%d sign changes of a difference below %.1e" % (len(r["crossings"]),
                                                                             r["max_abs_difference"])
        r["steps_per_s"] = 2 * r["steps_per_state"] / r["seconds"]
        out["hysteresis_p%03d" % round(100 * p)] = r
    red = []
    for rr in (0.05, 0.15, 0.25):
        c = red_path_curvature(rr)
        red.append({k: c[k] for k in ("r", "g_min", "printed_g_min", "d2E_min", "steps", "seconds")})
    out["red_paths"] = red
    return out


def adjoint_leg(n_steps, local, dev, stream):
    """Adjoint-gradient time / forward time on the 27-qubit lattice with the Fourier
    schedule s(t) = t/T + sum_{m<=16} a_m sin(m pi t/T), a_m ~ N(0, 0.01^2) (seed 2108),
    T = 20, second order; complex64 forward, FP64 reductions.  The complex64 gradient
    dE/da_m is compared with the complex128 adjoint on the same GPU."""
    import torch
    import synth
    from paper_2108_13410_gb300 import Simulator
    from paper_2108_13410_gb300.autograd import fourier_schedule
    W = WORKLOAD
    T = W["T"]
    dt = T / n_steps
    a = synth.fourier_coeffs(16, seed=2108, std=0.01)
    s, jac = fourier_schedule(a, T, n_steps)
    cpl = [(W["g"], W["lam"])]
    out = {"steps": n_steps, "M": 16, "T": T}
    grads = {}
    from paper_2108_13410_gb300.qsim import QS_OPT_C128_DF
    for dtype in ("c64", "c128"):
        sim = Simulator(W["Lx"], W["Ly"], form=W["form"], dtype=dtype, device=f"cuda:{local}", aux=True)
        if dtype == "c128":
            # the reference: FP64 forward and FP64 reverse sweep (the reverse passes have
            # no double-float form)
            sim.set_option(QS_OPT_C128_DF, 0)
        sim.init_plus()
        sim.evolve(cpl, s[:3], dt, 2)
        torch.cuda.synchronize(dev)
        sim.init_plus()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.evolve(cpl, s, dt, 2)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fwd_ms = e0.elapsed_time(e1)
        sim.init_plus()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        val, g = sim.adjoint_grad(cpl, s, dt, 2)
        adj_ms = (time.perf_counter() - t0) * 1000.0
        grads[dtype] = jac @ g[0]
        out[dtype] = {"forward_ms": fwd_ms, "adjoint_ms": adj_ms, "adjoint_over_forward": adj_ms / fwd_ms,
                      "energy": float(val[0])}
        if dtype == "c128":
            out[dtype]["arithmetic"] = "FP64"
        del sim
        torch.cuda.empty_cache()
    ref = grads["c128"]
    out["c64_grad_max_abs_err_vs_c128"] = float(np.max(np.abs(grads["c64"] - ref)))
    out["grad_max_abs_c128"] = float(np.max(np.abs(ref)))
    out["adjoint_over_forward"] = out["c64"]["adjoint_over_forward"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--no-scan", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-pergate", action="store_true")
    ap.add_argument("--no-ug32", action="store_true", help="skip the 32-qubit unitary-gauge leg")
    ap.add_argument("--no-protocol", action="store_true", help="skip the hysteresis-protocol leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default X-pass configuration (fewer launches before the timed steps)")
    ap.add_argument("--source-hash", action="store_true",
                    help="print the X-pass kernel source hashes (CTA-staged kernels, warp-local shared pass)")
    args = ap.parse_args()
    if args.source_hash:
        print(kernel_source_hash(), kernel_source_hash("k_xpass_wl"))
        return 0
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
