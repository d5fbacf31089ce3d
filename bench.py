#!/usr/bin/env python
"""Throughput benchmark of the checkerboard Metropolis XY path; prints one JSON line.

A step is one pass of the whole hot path over one lattice: the Philox hot
start followed by 1000 red/black Metropolis sweeps of an L = 4096 lattice at
beta = 1.12 (seed 7), each sweep with its fused per-sweep reductions.  With
N > 1 (torchrun, one rank per GPU) every rank runs its own independent chain
(lattice_id = rank): replicas, no collective on the data path.

  value  spin updates per second over all ranks, inputs resident on the
         device, CUDA events around each step on the lattice's stream, L2
         flushed (256 MiB write) before every timed step;
  e2e    the same metric through the C ABI with host buffers: every step
         copies the start configuration from pinned host memory (xy_set_state),
         sweeps, reads the records (xy_measure) and the final angles
         (xy_get_state); wall clock around each step.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "XY spin-updates/s on 1 GB300 (L=4096 and batched) and % of roofline"
UNIT = "spin-updates/s"
FLUSH_BYTES = 256 << 20

# Algorithmic instruction count per site update (one issue slot each), the
# work the method itself requires on this GPU:
#   Philox4x32-10: 20 wide multiplies + 20 three-input xors, 2 + 2 of them shared
#     by all sites of a sweep -> 36 per block, and one block serves two updates
#     (the sites x and x + 2 of a row share it) -> 18;
#   proposal theta + (delta 2^-23) ((w0 >> 8) - 2^23) and wrap -> 5;
#   neighbour sums (2 x 3 adds) -> 6;
#   two unit vectors (own + proposal; neighbours reuse their own): 2 x 25 with the
#     polynomial (reduction 4, minimax polynomials 9, quadrant 6, shared square
#     and products), 2 x 3 with the SFU intrinsics, 2 x 27 with CUDA's sincosf;
#   dE, Boltzmann factor, accept test and select: 22 (expf) / 14 (__expf);
#   per-sweep sums: 12 products and sums, 5 roundings to fixed point and 2.5
#     integer adds per black site -> 9.75 per update.
ALG_INSTR_PER_UPDATE = {"accurate": 110.75, "libm": 114.75, "fast": 58.75}
SMS, SMSP_PER_SM, LANES = 152, 4, 32       # GB300: 152 SMs x 4 schedulers x 32 lanes
TIMING_EVERY = 50          # kernel events on every 50th sweep of the timed region


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sincos", choices=["accurate", "fast", "libm"], default="accurate")
    ap.add_argument("--algorithm", choices=["auto", "fused", "two_pass", "persistent", "fused2"],
                    default="auto")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["large", "huge", "batch", "hmc", "quad", "peaks"],
                    default="large",
                    help="large: L=4096, 1000 sweeps/step; huge: L=16384, 200 sweeps/step; "
                         "batch: 256 lattices with replica exchange, 100 rounds/step; "
                         "hmc: HMC at L=4096, 10 trajectories of 80 leap-frog steps per step; "
                         "quad: four replicas per site at L=4096, 200 sweeps per step; "
                         "peaks: the instruction-rate microbenchmarks alone")
    ap.add_argument("--ctas-per-sm", type=int, default=0, choices=[0, 2, 3, 4],
                    help="work plan of the fused sweep: tile CTAs per SM (0: the library's "
                         "default)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary workloads reported beside the main line")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="override sweeps per step (profiling runs only)")
    ap.add_argument("--side", type=int, default=None,
                    help="override the lattice side L of the large workload (e.g. the "
                         "paper's Table 1 sides; profiling and scaling runs, not the headline)")
    return ap.parse_args()


def workload(args):
    import dataclasses
    from paper_0811_2111_gb300 import workloads as WL
    w = {"large": WL.LARGE, "huge": WL.HUGE, "batch": WL.LARGE}[args.workload]
    if args.sweeps is not None:
        w = dataclasses.replace(w, sweeps=args.sweeps)
    if args.side is not None:
        w = dataclasses.replace(w, L=args.side,
                                name=f"xy_L{args.side}_beta{w.beta}_seed{w.seed}_{w.sweeps}sweeps")
    return w


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value, world, device=None):
    """Max of a float over ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def alu_roofline(updates_per_s, sincos, clk_mhz, issue_per_sm_clk=None):
    """Issue-slot roofline of a Metropolis workload: algorithmic instructions per
    update x updates/s against SMs x the measured issue rate per SM and clock
    (xy_peak_measure's issue kind; nominal 4 schedulers x 32 lanes if unmeasured)
    x the SM clock."""
    instr = ALG_INSTR_PER_UPDATE[sincos]
    per_clk = issue_per_sm_clk or SMSP_PER_SM * LANES
    peak = SMS * per_clk * clk_mhz * 1e6 / 1e12
    achieved = instr * updates_per_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
            "frac": achieved / peak, "algorithmic_instr_per_update": instr,
            "peak_kind": "measured" if issue_per_sm_clk else "nominal",
            "basis": "whole-run throughput (launch gaps included)"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Loop iterations per thread of each instruction-rate microbenchmark
# (include/xy_peaks.h), sized for launches of a few milliseconds on GB300.
PEAK_ITERS = {"ffma": 32768, "imad": 16384, "imad_wide": 8192, "imad_hi": 16384,
              "lop3": 16384, "iadd": 16384, "mufu_sin": 4096, "mufu_ex2": 4096, "f2i": 4096,
              "dfma": 512, "issue": 16384, "philox": 512, "unit_vector": 1536,
              "unit_vector_sfu": 2048, "expf": 3072}


def measure_peaks(dev, kinds=None, reps=5):
    """Measured instruction rates of this GPU (xy_peak_measure): per kind the
    operations per second over the GPU and per SM per clock at the median SM
    clock sampled while they ran."""
    from paper_0811_2111_gb300 import _lib as X
    import torch
    kinds = kinds or list(PEAK_ITERS)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sampler = ClockSampler(str(dev.index or 0))
    sampler.start()
    raw = {}
    for k in kinds:
        rate, ms, ops = X.xy_peak_measure(k, PEAK_ITERS[k], reps, C.c_void_p(stream.cuda_stream))
        raw[k] = (rate, ms)
    clocks = sampler.stop()
    clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    out = {"sm_mhz": clk, "sms": sms, "clock_reasons": clocks.get("reasons"), "kinds": {}}
    for k, (rate, ms) in raw.items():
        out["kinds"][k] = {"ops_per_s": rate, "per_sm_per_clock": rate / (sms * clk * 1e6),
                           "best_ms": ms}
    return out


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    from paper_0811_2111_gb300 import build as B
    if d.get("source_hash") != B.source_hash():
        return None          # kernels changed since the counters were taken
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_sample(w, target_s, nthreads):
    """Time the FP64 oracle on the L x L workload: sweeps from the hot start."""
    import oracle
    t = time.perf_counter()
    oracle.run(w.L, w.L, w.beta, 1, seed=w.seed, nthreads=nthreads)
    one = time.perf_counter() - t
    n = max(1, min(50, int(target_s / max(one, 1e-9))))
    t = time.perf_counter()
    oracle.run(w.L, w.L, w.beta, n, seed=w.seed, nthreads=nthreads)
    dt = time.perf_counter() - t
    return w.sites * n / dt, n, dt


def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    w = workload(args)
    nthreads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.run(w.L, w.L, w.beta, 1, seed=w.seed, nthreads=nthreads)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.run(w.L, w.L, w.beta, 1, seed=w.seed, nthreads=nthreads)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = w.sites * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "L": w.L, "beta": w.beta, "seed": w.seed,
                   "sweeps_per_step": 1, "note": f"each step: one oracle sweep of the "
                   f"full L={w.L} lattice from the hot start (bounded sample of the "
                   f"{w.sweeps}-sweep workload)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": f"{args.steps} x 1 sweep of L={w.L} from the seed-{w.seed} "
                                   "hot start, OpenMP over the sites of one colour"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Batched workload: 256 lattices, 8 replica-exchange ladders
# ---------------------------------------------------------------------------

def measure_batch(dev, steps, warmup, sincos, rounds_per_step=100):
    """Updates/s of the batched engine on the replica-exchange workload, next to the
    same lattices swept one context at a time with the single-lattice kernels."""
    import torch
    from paper_0811_2111_gb300 import autotune
    from paper_0811_2111_gb300 import workloads as WL
    from paper_0811_2111_gb300.lattice import Batch, Lattice

    Ls, betas, ladders = WL.batch_layout()
    plan = autotune.tune_batch(Ls, betas, ladders, sweeps_per_round=10, sincos=sincos,
                               device=dev, use_cache=False)
    sweeps = rounds_per_step * 10
    sites = sum(L * L for L in Ls)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with Batch(Ls, betas, WL.BATCH_SEED, ladders=ladders, sweeps_per_round=10, sincos=sincos,
               target_band_sites=plan["target_band_sites"], group_ctas=plan["group_ctas"],
               ctas_per_sm=plan["ctas_per_sm"], device=dev) as b:
        b.reserve(rounds_per_step * (steps + max(1, warmup)))
        for _ in range(max(1, warmup)):
            b.run(rounds_per_step)
        torch.cuda.synchronize(dev)
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.run(rounds_per_step)
            e1.record(b.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        slots, acc, att = b.exchange_stats()
        n_ctas = b.info()[3]
        launches_per_round = b.launches_per_round()
    value = sites * sweeps * steps / (sum(ms) * 1e-3)
    # the same work as separate single-lattice contexts, one lattice at a time
    per_L = {}
    for L in sorted(set(Ls)):
        with Lattice(L, 1.1, 1, sincos=sincos, device=dev) as lat:
            lat.reserve(200)
            lat.sweep(20)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.sweep(100)
            e1.record(lat.stream)
            e1.synchronize()
            per_L[L] = e0.elapsed_time(e1) / 100          # ms per sweep
    single_ms_per_sweep = sum(per_L[L] for L in Ls)
    single_value = sites / (single_ms_per_sweep * 1e-3)
    return {"workload": "xy_batch_256_lattices_L16-256_64beta_x4_exchange_every_10",
            "value": value, "unit": UNIT, "ms_per_step": sum(ms) / steps,
            "sweeps_per_step": sweeps, "lattices": len(Ls), "sites": sites,
            "ctas_per_launch": n_ctas, "target_band_sites": plan["target_band_sites"],
            "plan": {"group_ctas": plan["group_ctas"], "ctas_per_sm": plan["ctas_per_sm"],
                     "target_band_sites": plan["target_band_sites"],
                     "candidates_ms_per_round": plan["ms_per_round"]},
            "exchange_acceptance": float(acc.sum() / max(att.sum(), 1)),
            "single_lattice_kernels_value": single_value,
            "speedup_vs_single_lattice_kernels": value / single_value,
            "launches_per_step": launches_per_round * rounds_per_step}


def measure_differentiation(dev, sincos, therm=10000, meas=100000):
    """The differentiated workload: 41 chains (beta 0.90 .. 1.30) of L=256, therm +
    meas sweeps in one batch, then the backward kernel over the device series."""
    import torch
    from paper_0811_2111_gb300 import workloads as WL
    from paper_0811_2111_gb300.autograd import chain_averages

    # warm the path once on a tiny case: torch loads its float64 elementwise
    # kernels lazily on first use, which would otherwise land in the timed backward
    wb = torch.tensor([1.0, 1.1], dtype=torch.float64, device=dev, requires_grad=True)
    we, _ = chain_averages(wb, 8, 1, 100, 100, sweeps_per_round=100, sincos=sincos)
    torch.autograd.grad(we.sum(), wb)
    betas = torch.tensor(WL.DIFF_BETAS, dtype=torch.float64, device=dev, requires_grad=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    e, u = chain_averages(betas, WL.DIFF_L, WL.DIFF_SEED, therm, meas, sweeps_per_round=1000,
                          sincos=sincos)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    stream = torch.cuda.current_stream(dev)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    # retain_graph keeps the forward's batch (and its device series) alive, so
    # its release is not timed as part of the backward
    (g,) = torch.autograd.grad(e.sum(), betas, retain_graph=True)
    b1.record(stream)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    backward_device_ms = b0.elapsed_time(b1)
    updates = len(WL.DIFF_BETAS) * WL.DIFF_L ** 2 * (therm + meas)
    gb = g.detach().cpu().numpy()
    b = np.array(WL.DIFF_BETAS)
    cv = -(b ** 2) * gb
    return {"workload": f"xy_diff_L{WL.DIFF_L}_41beta_{therm}+{meas}sweeps", "value":
            updates / (t1 - t0), "unit": UNIT, "forward_s": t1 - t0, "backward_ms": 1e3 * (t2 - t1),
            "backward_device_ms": backward_device_ms,
            "specific_heat_peak": {"beta": float(b[int(np.argmax(cv))]), "c_v": float(cv.max())},
            "timing": "wall clock around forward (chains + series kept on the device) and "
                      "backward (FP64 covariance kernel)"}


def measure_table1_sizes(dev, sincos, cpu_seconds=1.0):
    """The lattice sides of the paper's Table 1 (L = 128 ... 2048): fused-kernel
    Metropolis updates/s and HMC leap-frog site-steps/s on the GPU against the
    FP64 oracle on one host core; the HMC ratio is the analogue of the paper's
    "gain" over its serial HMC code (2008 GPU against one Conroe core: context,
    not a target)."""
    import torch
    import oracle
    from paper_0811_2111_gb300.lattice import Lattice

    out = {}
    for L in (128, 256, 512, 1024, 2048):
        sweeps = max(50, int(2e9 // (L * L)))
        with Lattice(L, 1.0, 3, sincos=sincos, device=dev) as lat:
            lat.reserve(sweeps + 10)
            lat.sweep(10)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.sweep(sweeps)
            e1.record(lat.stream)
            e1.synchronize()
            gpu = L * L * sweeps / (e0.elapsed_time(e1) * 1e-3)
        n = 1
        t = time.perf_counter()
        oracle.run(L, L, 1.0, n, seed=3, nthreads=1)
        dt = time.perf_counter() - t
        while dt < cpu_seconds and n < 4096:
            n *= 2
            t = time.perf_counter()
            oracle.run(L, L, 1.0, n, seed=3, nthreads=1)
            dt = time.perf_counter() - t
        cpu = L * L * n / dt
        out[str(L)] = {"gpu": gpu, "oracle_1core": cpu, "gain": gpu / cpu}
        if L <= 256:
            # a single lattice through the batched engine: one graph launch runs 100
            # sweeps of fused tiles (bit-identical to the single-lattice kernels)
            from paper_0811_2111_gb300.lattice import Batch
            rounds = max(2, int(2e9 // (L * L * 100)))
            with Batch([L], [1.0], 3, sweeps_per_round=100, sincos=sincos, device=dev) as b:
                b.reserve(rounds + 2)
                b.run(2)
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(b.stream)
                b.run(rounds)
                e1.record(b.stream)
                e1.synchronize()
                out[str(L)]["gpu_batched_engine_100_sweeps_per_launch"] = (
                    L * L * 100 * rounds / (e0.elapsed_time(e1) * 1e-3))
        # four replicas per site (the RGBA packing of Sec. 3.2), two-pass kernels
        from paper_0811_2111_gb300.lattice import Quad
        qs = max(20, int(2e9 // (4 * L * L)))
        with Quad(L, [1.0, 1.0, 1.0, 1.0], 3, sincos=sincos, device=dev) as qd:
            qd.sweep(5)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(qd.stream)
            qd.sweep(qs)
            e1.record(qd.stream)
            e1.synchronize()
            out[str(L)]["gpu_quad_4_replicas"] = 4 * L * L * qs / (e0.elapsed_time(e1) * 1e-3)
        # the paper's own algorithm: HMC trajectories (unit length, eps ~ N^-1/4)
        from paper_0811_2111_gb300 import workloads as WL
        from paper_0811_2111_gb300.hmc import HMC
        eps, n_md = WL.hmc_step_for(L)
        n_traj = max(5, int(4e9 // (L * L * n_md)))
        with HMC(L, 1.0, 3, eps, n_md, sincos=sincos, device=dev) as h:
            h.run(5)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(h.stream)
            h.run(n_traj)
            e1.record(h.stream)
            e1.synchronize()
            hmc_gpu = L * L * n_md * n_traj / (e0.elapsed_time(e1) * 1e-3)
            acc = float(h.observables(5)["accepted"].mean())
        rng = np.random.default_rng(2)
        th = rng.uniform(0, 2 * np.pi, L * L)
        pm = rng.normal(size=L * L)
        n = 1
        while True:
            t = time.perf_counter()
            oracle.hmc_leapfrog(th, pm, L, L, 1.0, eps, n)
            dt = time.perf_counter() - t
            if dt >= cpu_seconds or n >= 4096:
                break
            n *= 2
        hmc_cpu = L * L * n / dt
        out[str(L)]["hmc"] = {"eps": eps, "n_md": n_md, "acceptance": acc,
                              "gpu_site_steps": hmc_gpu, "oracle_1core_site_steps": hmc_cpu,
                              "gain": hmc_gpu / hmc_cpu}
    return {"unit": UNIT, "beta": 1.0, "sizes": out,
            "paper_cuda_gain_for_context": {"128": 33, "256": 37, "512": 38, "1024": 30,
                                            "2048": 30}}


# ---------------------------------------------------------------------------
# Hybrid Monte Carlo (the paper's own algorithm)
# ---------------------------------------------------------------------------

# The full kick-drift steps run two per launch (k_hmc_tile2): each launch reads
# and writes the angle and the momentum of every site once, 16 B per site for
# two steps.
HMC_BYTES_PER_SITE_STEP = 8.0
# Algorithmic thread-instructions of one site-step: the new angle's unit
# vector (25 accurate, 3 SFU, 27 libm, as for a Metropolis update), the two
# neighbour sums 6, the force 3, kick and drift 2, the wrap into [0, 2 pi) 8.
HMC_ALG_INSTR_PER_SITE_STEP = {"accurate": 44.0, "fast": 22.0, "libm": 46.0}
# DRAM bytes of one L = 4096 two-step launch (ncu, caches flushed before the
# capture: 134.4 MB read, 83.9 MB written; profiles/hmc_tile2_L4096_full.md),
# per step.
HMC_DRAM_BYTES_PER_STEP = 218.2e6 / 2


def measure_hmc(dev, sincos, trajectories=40, cpu_seconds=2.0, issue_per_sm_clk=None,
                clk_mhz=2070.0):
    """Leap-frog site-steps/s of HMC at L = 4096, beta = 1.12 (trajectories of 80
    steps of 0.0125, from a state thermalised by 2000 Metropolis sweeps and 30
    HMC trajectories), the step kernel's duration and HBM roofline, and the FP64
    oracle's leap-frog on one host core."""
    import torch
    import oracle
    from paper_0811_2111_gb300 import workloads as WL
    from paper_0811_2111_gb300.hmc import HMC

    from paper_0811_2111_gb300.lattice import Lattice

    L, N = WL.HMC_L, WL.HMC_L * WL.HMC_L
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # thermalise with the Metropolis engine (cheap), then hand the state over
    with Lattice(L, WL.HMC_BETA, WL.HMC_SEED, sincos=sincos, device=dev) as lat:
        lat.reserve(WL.HMC_METROPOLIS_THERM)
        lat.sweep(WL.HMC_METROPOLIS_THERM)
        therm_state, _ = lat.state()
    with HMC(L, WL.HMC_BETA, WL.HMC_SEED, WL.HMC_EPS, WL.HMC_NMD, sincos=sincos,
             device=dev) as h:
        h.set_state(therm_state, None, 0)
        h.run(WL.HMC_THERM)
        h.synchronize()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(h.stream)
        h.run(trajectories)
        e1.record(h.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        o = h.observables(WL.HMC_THERM, trajectories)
        # the step kernel alone: integrate(21) - integrate(1) = ten two-step launches
        reps = 20
        t = {}
        for n in (1, 21):
            e0.record(h.stream)
            for _ in range(reps):
                h.integrate(n)
            e1.record(h.stream)
            e1.synchronize()
            t[n] = e0.elapsed_time(e1) / reps
    step_ms = (t[21] - t[1]) / 20
    achieved = HMC_BYTES_PER_SITE_STEP * N / (step_ms * 1e-3) / 1e9
    per_clk = issue_per_sm_clk or SMSP_PER_SM * LANES
    alu_peak = SMS * per_clk * clk_mhz * 1e6 / 1e12
    alu_achieved = HMC_ALG_INSTR_PER_SITE_STEP[sincos] * N / (step_ms * 1e-3) / 1e12
    hbm, peak_kind = measured_peaks()
    # FP64 oracle leap-frog on one core (L = 512 sample)
    Ls = 512
    rng = np.random.default_rng(1)
    th = rng.uniform(0, 2 * np.pi, Ls * Ls)
    p = rng.normal(size=Ls * Ls)
    n, dt = 1, 0.0
    while True:
        t0 = time.perf_counter()
        oracle.hmc_leapfrog(th, p, Ls, Ls, WL.HMC_BETA, 0.05, n)
        dt = time.perf_counter() - t0
        if dt >= cpu_seconds or n >= 256:
            break
        n *= 2
    cpu = Ls * Ls * n / dt
    value = N * WL.HMC_NMD * trajectories / (ms * 1e-3)
    return {"workload": f"xy_hmc_L{L}_beta{WL.HMC_BETA}_eps{WL.HMC_EPS}_nmd{WL.HMC_NMD}",
            "metric": "leap-frog site-steps/s", "value": value, "unit": "site-steps/s",
            "trajectories_per_s": trajectories / (ms * 1e-3), "ms_per_trajectory": ms / trajectories,
            "begin_final_accept_ms": t[1], "acceptance": float(o["accepted"].mean()),
            "mean_exp_minus_dH": float(np.exp(-o["dH"]).mean()), "e": float(o["e"].mean()),
            "roofline": {"kernel": "k_hmc_tile2 (two leap-frog steps per launch)",
                         "bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                         "unit": "Tinstr/s", "frac": alu_achieved / alu_peak,
                         "peak_kind": "measured" if issue_per_sm_clk else "nominal",
                         "algorithmic_instr_per_site_step": HMC_ALG_INSTR_PER_SITE_STEP[sincos],
                         "ms_per_step": step_ms,
                         "hbm": {"achieved": achieved, "peak": hbm, "peak_kind": peak_kind,
                                 "unit": "GB/s", "frac": achieved / hbm,
                                 "bytes_per_site_step": HMC_BYTES_PER_SITE_STEP,
                                 "dram_bytes_per_step": HMC_DRAM_BYTES_PER_STEP,
                                 "dram_achieved": HMC_DRAM_BYTES_PER_STEP / (step_ms * 1e-3) / 1e9,
                                 "dram_frac": HMC_DRAM_BYTES_PER_STEP / (step_ms * 1e-3) / 1e9 / hbm}},
            "cpu_baseline": {"value": cpu, "unit": "site-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"FP64 leap-frog, L={Ls}, {n} steps"},
            "gain_vs_oracle_1core": value / cpu}


def _time_quad(dev, L, sincos, algorithm, sweeps, flush):
    import torch
    from paper_0811_2111_gb300.lattice import Quad

    with Quad(L, [1.0, 1.06, 1.12, 1.18], 7, sincos=sincos, algorithm=algorithm, device=dev) as q:
        q.sweep(10)
        torch.cuda.synchronize(dev)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(q.stream)
        q.sweep(sweeps)
        e1.record(q.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        acc = [float(q.observables(r, 10)["accepted"].mean()) / (L * L) for r in range(4)]
        algo = q.algorithm
    return 4 * L * L * sweeps / (ms * 1e-3), ms / sweeps, acc, algo


def measure_quad(dev, sincos, sweeps=200):
    """Four replicas per site at L = 4096 (betas 1.00, 1.06, 1.12, 1.18): updates/s
    over all replicas with the one-launch sweep, the two-pass kernels beside it."""
    import torch

    L = 4096
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    value, ms, acc, algo = _time_quad(dev, L, sincos, "auto", sweeps, flush)
    value2, ms2, _, _ = _time_quad(dev, L, sincos, "two_pass", sweeps, flush)
    fused = algo == "fused"
    bpu = 8.0 if fused else 12.0
    return {"workload": "xy_quad_L4096_4replicas_beta1.00-1.18", "value": value, "unit": UNIT,
            "algorithm": algo, "ms_per_sweep": ms, "acceptance": acc,
            "bytes_per_update": bpu,
            "hbm_achieved_gbs": bpu * value / 1e9,
            "launches_per_sweep": 1 if fused else 2,
            "two_pass": {"value": value2, "ms_per_sweep": ms2, "bytes_per_update": 12.0}}


def measure_precision(dev, sweeps=200):
    """The precision workload: L=16384 (1 GiB of angles), beta=1.12, seed 7,
    `sweeps` sweeps per variant; updates/s of each sincos / reduction variant."""
    import torch
    from paper_0811_2111_gb300 import workloads as WL
    from paper_0811_2111_gb300.lattice import Lattice

    w = WL.HUGE
    out = {"workload": w.name, "unit": UNIT, "variants": {}}
    for sincos, reduce in (("accurate", "exact"), ("fast", "exact"), ("libm", "exact"),
                           ("accurate", "compensated")):
        with Lattice(w.L, w.beta, w.seed, sincos=sincos, reduce=reduce, device=dev) as lat:
            lat.reserve(sweeps + 3)
            lat.sweep(3)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(lat.stream)
            lat.sweep(sweeps)
            e1.record(lat.stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            obs = lat.observables(3, sweeps)
        out["variants"][f"{sincos}/{reduce}"] = {
            "value": w.sites * sweeps / (ms * 1e-3), "ms_per_sweep": ms / sweeps,
            "e_last": float(obs["e"][-1]), "upsilon_last": float(obs["upsilon"][-1])}
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    from paper_0811_2111_gb300 import build as B
    from paper_0811_2111_gb300 import _lib as X
    from paper_0811_2111_gb300.lattice import Lattice

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.build()
    if args.workload == "batch":
        return run_batch_line(args, dev, world, rank)
    if args.workload == "hmc":
        return run_hmc_line(args, dev, world, rank)
    if args.workload == "quad":
        return run_quad_line(args, dev, world, rank)
    if args.workload == "peaks":
        p = measure_peaks(dev)
        if rank == 0:
            print(json.dumps({"metric": "instruction rates (xy_peak_measure)", "peaks": p}),
                  flush=True)
        return 0

    w = workload(args)
    stream = torch.cuda.current_stream(dev)
    # the work plan: timed candidates (autotune.tune_lattice) unless both the
    # algorithm and the CTAs per SM were given
    tuned = None
    algorithm, ctas = args.algorithm, args.ctas_per_sm
    if args.algorithm == "auto" or args.ctas_per_sm == 0:
        from paper_0811_2111_gb300 import autotune
        tuned = autotune.tune_lattice(w.L, w.beta, args.sincos, device=dev, use_cache=False)
        if args.algorithm == "auto" and tuned["algorithm"] != "two_pass":
            algorithm = tuned["algorithm"]
        if args.ctas_per_sm == 0:
            ctas = tuned["ctas_per_sm"]
    lat = Lattice(w.L, w.beta, w.seed, device=dev, stream=stream, lattice_id=rank,
                  sincos=args.sincos, algorithm=algorithm, ctas_per_sm=ctas)
    persistent = lat.algorithm == "persistent"        # what AUTO resolved to
    two = lat.algorithm == "fused2"                     # two sweeps per launch
    fused = lat.algorithm in ("fused", "persistent", "fused2")
    lat.reserve(w.sweeps)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        lat.reset(w.seed)
        lat.sweep(w.sweeps)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    # the instruction-rate microbenchmarks: the roofline's measured peaks
    peaks = measure_peaks(dev)
    issue_clk = peaks["kinds"]["issue"]["per_sm_per_clock"]

    props = torch.cuda.get_device_properties(dev)
    gpu_id = getattr(props, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None else str(local)
    sampler = ClockSampler(gpu_id)

    lat.timing(TIMING_EVERY)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler.start()
    for k in range(args.steps):
        flush.fill_(float(k))                         # evict the lattice from L2
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kt = {k: lat.kernel_time(k) for k in (0, 1)}
    lat.timing(0)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    updates = w.updates * args.steps * world
    value = updates / (total_ms * 1e-3)

    # e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        lat.reset(w.seed)
        start_state, _ = lat.state()
        host_in = torch.from_numpy(start_state.reshape(-1).copy()).pin_memory()
        host_out = torch.empty(w.sites, dtype=torch.float32).pin_memory()
        recs = (X.xy_obs * w.sweeps)()
        nxt = C.c_uint64()
        lib = X.lib()
        wall = []
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            X.check(lib.xy_set_state(lat.ctx, C.c_void_p(host_in.data_ptr()), 0), lat.ctx)
            X.check(lib.xy_sweep(lat.ctx, w.sweeps), lat.ctx)
            X.check(lib.xy_measure(lat.ctx, 0, w.sweeps, recs), lat.ctx)
            X.check(lib.xy_get_state(lat.ctx, C.c_void_p(host_out.data_ptr()), C.byref(nxt)),
                    lat.ctx)
            wall.append(time.perf_counter() - t)
        e2e_s = max_over_ranks(sum(wall), world, dev)
        e2e = {"value": w.updates * args.steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 4 * w.sites,
               "d2h_bytes_per_step": 4 * w.sites + C.sizeof(X.xy_record) * w.sweeps}

    # roofline of the dominant kernel (the one with the larger device time)
    kern = max((0, 1), key=lambda k: kt[k][0])
    kms, klaunch = kt[kern]
    avg_s = kms * 1e-3 / max(klaunch, 1)
    sweeps_per_launch = w.sweeps if persistent else (2 if two else 1)
    updates_per_launch = (w.sites if fused else w.sites // 2) * sweeps_per_launch
    alg_bytes = 8.0 * updates_per_launch     # 8 B per update: one read + one write of the angle
    hbm_peak, peak_kind = measured_peaks()
    hbm_achieved = alg_bytes / avg_s / 1e9
    names = (["sweep_fused_persist"] if persistent else ["sweep_fused2"] if two else
             ["sweep_fused"] if fused else ["red_half_sweep", "black_half_sweep_measure"])
    # issue-slot roofline: the measured issue rate per SM and clock
    # (xy_peak_measure, issue kind) x SMs x the median SM clock sampled during
    # the timed region (max clock if unsampled)
    clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    alu_peak = SMS * issue_clk * clk * 1e6 / 1e12                     # T instr/s
    nominal_peak = SMS * SMSP_PER_SM * LANES * clk * 1e6 / 1e12
    instr = ALG_INSTR_PER_UPDATE[args.sincos]
    alu_achieved = instr * updates_per_launch / avg_s / 1e12
    roofline = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Tinstr/s",
                "frac": alu_achieved / alu_peak, "traffic": profiled_traffic(),
                "kernel": names[kern], "kernel_avg_us": avg_s * 1e6,
                "algorithmic_instr_per_update": instr,
                "peak_kind": "measured",
                "peak_basis": (f"{SMS} SMs x {issue_clk:.2f} thread-instructions per SM and clock "
                               f"(xy_peak_measure issue kind, measured at "
                               f"{peaks['sm_mhz']:.0f} MHz in this run) x {clk:.0f} MHz"),
                "peak_nominal": nominal_peak,
                "frac_of_nominal": alu_achieved / nominal_peak,
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": hbm_achieved / hbm_peak, "peak_kind": peak_kind,
                        "algorithmic_bytes_per_launch": alg_bytes},
                "kernel_timing": ("CUDA events around every launch (all sweeps of a step) "
                                  "inside the timed region" if persistent else
                                  f"CUDA events around the launches of every {TIMING_EVERY}th "
                                  "sweep inside the timed region"),
                "sweeps_per_launch": sweeps_per_launch,
                "kernel_avg_ms": {names[k]: kt[k][0] / max(kt[k][1], 1)
                                  for k in range(len(names))}}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nthreads = os.cpu_count() or 1
        v, n, dt = oracle_sample(w, args.cpu_seconds, nthreads)
        cpu = {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"{n} sweeps of L={w.L} from the seed-{w.seed} hot start "
                         f"({dt:.1f} s), OpenMP over the sites of one colour"}

    launches = args.steps * (2 if persistent else
                             1 + ((w.sweeps + 1) // 2 if two else (1 if fused else 2) * w.sweeps))
    extra = None
    if not args.no_extra and world == 1:
        extra = {"batch": measure_batch(dev, 3, 1, args.sincos),
                 "differentiation": measure_differentiation(dev, args.sincos),
                 "precision": measure_precision(dev),
                 "table1_sizes": measure_table1_sizes(dev, args.sincos),
                 "hmc": measure_hmc(dev, args.sincos, issue_per_sm_clk=issue_clk,
                                    clk_mhz=clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0),
                 "quad": measure_quad(dev, args.sincos)}
        # the same issue-slot roofline as the main line, over a whole run of each
        # Metropolis workload (launch gaps included: a lower bound on the kernels')
        clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        for key in ("batch", "differentiation", "quad"):
            extra[key]["roofline"] = alu_roofline(extra[key]["value"], args.sincos, clk,
                                                  issue_clk)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "L": w.L, "beta": w.beta, "seed": w.seed,
                   "sweeps_per_step": w.sweeps, "sincos": args.sincos, "reduce": "exact",
                   "kernel": ("persistent fused (one cooperative launch per step)" if persistent
                              else "two sweeps per launch (temporal blocking)" if two
                              else "fused single-pass" if fused else "two-pass red/black"),
                   "ctas_per_sm": ctas or 3,
                   "plan": ("tuned" if tuned else "given") + f": {lat.algorithm}, "
                           f"{ctas or 3} CTAs per SM",
                   "plan_candidates_ms_per_sweep": tuned["ms_per_sweep"] if tuned else None,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "peaks": peaks, "other_workloads": extra,
    }
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batch_line(args, dev, world, rank):
    """Main line for --workload batch (replicas of the whole batch with N > 1)."""
    import torch
    sampler = ClockSampler(str(dev.index or 0))
    barrier(world)
    sampler.start()
    r = measure_batch(dev, args.steps, max(3, args.warmup), args.sincos)
    clocks = sampler.stop()
    total_ms = max_over_ranks(r["ms_per_step"] * args.steps, world, dev)
    value = r["sites"] * r["sweeps_per_step"] * args.steps * world / (total_ms * 1e-3)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": r["workload"], "sincos": args.sincos,
                                            "l2": "flushed before every timed step (256 MiB write)",
                                            "parallelism": f"replicas x{world}"},
            "batch": r, "gpu_launches": r["launches_per_step"] * args.steps, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_quad_line(args, dev, world, rank, sweeps_per_step=200):
    """Main line for --workload quad: four replicas per site (Sec. 3.2's RGBA
    packing) at L = 4096, betas 1.00, 1.06, 1.12, 1.18 (replicas with N > 1)."""
    import torch
    from paper_0811_2111_gb300.lattice import Quad

    L = 4096
    issue_clk = measure_peaks(dev, kinds=["issue"])["kinds"]["issue"]["per_sm_per_clock"]
    sampler = ClockSampler(str(dev.index or 0))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with Quad(L, [1.0, 1.06, 1.12, 1.18], 7, sincos=args.sincos, lattice_id=4 * rank,
              device=dev) as q:
        algo = q.algorithm
        for _ in range(max(3, args.warmup)):
            q.sweep(sweeps_per_step)
        q.synchronize()
        barrier(world)
        sampler.start()
        ms = []
        for k in range(args.steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(q.stream)
            q.sweep(sweeps_per_step)
            e1.record(q.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        clocks = sampler.stop()
    total_ms = max_over_ranks(sum(ms), world, dev)
    updates = 4 * L * L * sweeps_per_step * args.steps * world
    value = updates / (total_ms * 1e-3)
    per_sweep = 1 if algo == "fused" else 2
    clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "xy_quad_L4096_4replicas_beta1.00-1.18",
                       "sweeps_per_step": sweeps_per_step, "sincos": args.sincos,
                       "kernel": "fused single-pass" if algo == "fused" else "two-pass red/black",
                       "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": alu_roofline(value / world, args.sincos, clk, issue_clk),
            "gpu_launches": per_sweep * sweeps_per_step * args.steps + args.steps,
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_hmc_line(args, dev, world, rank, trajectories_per_step=10):
    """Main line for --workload hmc: the paper's own algorithm (replicas with N > 1;
    lattice id = rank)."""
    import torch
    from paper_0811_2111_gb300 import workloads as WL
    from paper_0811_2111_gb300.hmc import HMC

    from paper_0811_2111_gb300.lattice import Lattice

    L, N = WL.HMC_L, WL.HMC_L * WL.HMC_L
    sampler = ClockSampler(str(dev.index or 0))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with Lattice(L, WL.HMC_BETA, WL.HMC_SEED, sincos=args.sincos, lattice_id=rank,
                 device=dev) as lat:
        lat.reserve(WL.HMC_METROPOLIS_THERM)
        lat.sweep(WL.HMC_METROPOLIS_THERM)
        therm_state, _ = lat.state()
    with HMC(L, WL.HMC_BETA, WL.HMC_SEED, WL.HMC_EPS, WL.HMC_NMD, sincos=args.sincos,
             lattice_id=rank, device=dev) as h:
        h.set_state(therm_state, None, 0)
        for _ in range(max(3, args.warmup)):
            h.run(trajectories_per_step)
        h.synchronize()
        barrier(world)
        sampler.start()
        ms = []
        for k in range(args.steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(h.stream)
            h.run(trajectories_per_step)
            e1.record(h.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        clocks = sampler.stop()
        acc = float(h.observables()["accepted"][-args.steps * trajectories_per_step:].mean())
    total_ms = max_over_ranks(sum(ms), world, dev)
    steps_md = N * WL.HMC_NMD * trajectories_per_step * args.steps * world
    line = {"metric": "HMC leap-frog site-steps/s", "value": steps_md / (total_ms * 1e-3),
            "unit": "site-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"xy_hmc_L{L}_beta{WL.HMC_BETA}_eps{WL.HMC_EPS}_nmd{WL.HMC_NMD}",
                       "trajectories_per_step": trajectories_per_step, "sincos": args.sincos,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "acceptance": acc,
            "gpu_launches": ((WL.HMC_NMD + 2) * trajectories_per_step + 2) * args.steps,
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
