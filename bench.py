#!/usr/bin/env python
"""Spin-flip throughput of population annealing on a 3D +-1 spin glass.

Workload (one "step" of this benchmark = one complete annealing run): 3D
Edwards-Anderson +-1 spin glass, L = 8 periodic (512 spins), couplings from
seed 1, R0 = 100000 replicas, 201 inverse temperatures linear in 0..5 (200
annealing steps), 10 checkerboard Metropolis sweeps per step; the plain
single-run form (one launch of each kernel per annealing step).  Attempted
spin flips are counted exactly as sum over steps of R~_k * N * theta.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--batched] [--no-cpu-baseline]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its
own independent replica of the workload ("replicas only": the runs share
nothing), and value is the sum of all ranks' flips over the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1006_0252_gb300 import inputs  # noqa: E402

METRIC = "spin flips/s at 3D L=8 R0=1e5"
UNIT = "flips/s"
# Algorithmic integer operations per attempted flip: a quarter of one
# Philox4x32-10 block (10 rounds x (2 wide multiplies + 2
# three-input XORs) / 4 sites = 10) + the threshold compare (1) + the flip
# decision (1).
OPS_PER_FLIP = 12
TIME_EVERY = 8  # sweep launches timed with CUDA events: every 8th
# DRAM bytes (read + write) per sweep launch from one ncu capture of this
# kernel source (dram__bytes_read.sum + dram__bytes_write.sum); reported only
# while the kernel source is the one that was captured.
SWEEP_TRAFFIC = {"sha256_16": "e6c85eeaf62e4f52", "bytes": 5563477}


def sweep_traffic():
    import hashlib
    h = hashlib.sha256()
    for f in ("pa_sweep3d.cuh", "pa_lattice3d.cuh"):
        with open(os.path.join(ROOT, "paper_1006_0252_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return SWEEP_TRAFFIC["bytes"] if h.hexdigest()[:16] == SWEEP_TRAFFIC["sha256_16"] else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # The metric's other two parts (batched vs per-run launch, p50/p99 run
    # latency) and the paper's own Gaussian run sets run by default on one GPU
    # (about two minutes in all, after the timed L=8 runs); --quick skips them.
    p.add_argument("--quick", action="store_true", help="only the timed L=8 runs (and the CPU baseline)")
    p.add_argument("--batched", action=argparse.BooleanOptionalAction, default=None,
                   help="time the batched executor against per-run launches (default: on for one GPU)")
    p.add_argument("--batched-realisations", type=int, default=16)
    p.add_argument("--serving", type=int, default=None, metavar="N_REQUESTS",
                   help="run the serving workload with this many requests (default: 2000 for one GPU)")
    p.add_argument("--gauss", action=argparse.BooleanOptionalAction, default=None,
                   help="time the paper's Gaussian run sets (Sec. 4: 3D L=8 and the periodic chain)")
    p.add_argument("--gauss-study", action="store_true",
                   help="with --gauss: also the Sec. 4 overlap study (Gamma, P(q), temperature-dependent R)")
    p.add_argument("--chain", action=argparse.BooleanOptionalAction, default=None,
                   help="time the open-chain workload and check it against the closed form")
    p.add_argument("--no-cpu-baseline", action="store_true")
    a = p.parse_args()
    solo = a.gpus == 1 and not a.quick
    if a.batched is None:
        a.batched = solo
    if a.serving is None:
        a.serving = 2000 if solo else 0
    if a.gauss is None:
        a.gauss = solo
    if a.chain is None:
        a.chain = solo
    return a


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def run_flips(traj: dict, N: int, theta: int) -> int:
    return int(np.sum(traj["R"][1:]) * N * theta)


def oracle_sample(spec, R0: int, n_steps: int = 200):
    """The oracle as it stands on a bounded sample of the workload: init plus
    the first n_steps annealing steps (default: the whole schedule, beta 0 ->
    5, where the cost per flip changes with temperature) at R0 replicas.
    Returns (flips, s)."""
    from oracle import oracle as orc
    J = spec.couplings()
    L = spec.L
    t0 = time.perf_counter()
    r = orc.Run(J, 3, L, L, L, 7, R0=R0, R_cap=inputs.default_capacity(R0), seed=spec.seed)
    flips = 0
    for k in range(1, n_steps + 1):
        r.step(float(spec.betas[k]), spec.theta, R0)
        flips += r.state().R * spec.N * spec.theta
    dt = time.perf_counter() - t0
    r.close()
    return flips, dt


def _oracle_worker(a):
    """One host core: oracle_sample for PA seed offset a[2] (process-pool worker)."""
    R0, n_steps, off = a
    spec = inputs.config_l8()
    spec.seed = spec.seed + off
    return oracle_sample(spec, R0, n_steps)


def oracle_sample_cores(R0: int, n_cores: int, n_steps: int = 200, repeats: int = 1):
    """oracle_sample on n_cores host cores at once (independent runs of the
    same workload, PA seeds 1, 2, ...; a spawned pool, so that no process is
    forked from one that has touched the GPU), `repeats` times.  Returns a list
    of (flips, wall s), one per repeat."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = []
    with ctx.Pool(n_cores) as pool:
        pool.map(_oracle_worker, [(64, 2, i) for i in range(n_cores)])  # start-up and library load
        for _ in range(repeats):
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, [(R0, n_steps, i) for i in range(n_cores)])
            out.append((sum(f for f, _ in res), time.perf_counter() - t0))
    return out


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


REF_R0 = 160     # replicas per host core in each step of the reference arm
BASE_R0 = 600   # replicas per host core in the cpu_baseline sample


def reference_arm(args, ws, rank):
    """The oracle timed on the host cores on this benchmark's workload: each
    benchmark step is one complete annealing run (init + the 200 steps, beta 0
    -> 5) per host core at a reduced population."""
    if rank != 0:
        return 0
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(inputs.config_l8(), 64, 5)
    res = oracle_sample_cores(REF_R0, cores, 200, repeats=args.steps)
    tot_f = sum(f for f, _ in res)
    tot_t = sum(t for _, t in res)
    value = tot_f / tot_t
    sample = (f"L=8 couplings seed 1, R0={REF_R0} (of 1e5) per host core: init + all 200 annealing steps "
              f"(beta 0 -> 5), theta=10, one independent run per host core ({cores}), per benchmark step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i8/f64",
            "data": "synthetic", "config": {"workload": spec_name(), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(flips, gpu_ms, e2e_flips, e2e_t, dist=None):
    """Whole-job figures over independent replicas (one per rank): flips are
    summed, times take the slowest rank."""
    if dist is None:
        return flips, gpu_ms, e2e_flips, e2e_t
    import torch
    res = torch.tensor([flips, gpu_ms, e2e_flips, e2e_t], dtype=torch.float64)
    tot = res.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    mx = res.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    return tot[0].item(), mx[1].item(), tot[2].item(), mx[3].item()


def spec_name() -> str:
    return ("3D EA +-1 spin glass, L=8 periodic, couplings seed 1, R0=100000, 201 betas linear 0..5, "
            "theta=10, one run (init + 200 steps) per benchmark step")


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return reference_arm(args, ws, rank)

    import torch

    from paper_1006_0252_gb300 import pa

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="gloo")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)

    spec = inputs.config_l8()
    J = spec.couplings()
    N, theta, betas = spec.N, spec.theta, spec.betas
    seed_base = 1 + 1000 * rank
    run = pa.Run(J, 8, 3, spec.R0, seed_base)

    # One benchmark step: a fresh beta = 0 population, then the 200 annealing
    # steps replayed as one CUDA graph (captured in the warm-up; the steps read
    # their beta from the device schedule).
    def one_run(seed):
        run.reset(seed)
        pa.pa_run_schedule(run._h, betas[1:], theta, None, use_graph=True)

    # every TIME_EVERY-th sweep launch is timed with events (a systematic
    # sample over the whole schedule): events around every launch would add
    # about 1 % to the timed region; timing is on during the warm-up as well,
    # so the graph is captured with its timing events before the timed runs
    pa.pa_kernel_time(run._h, True, TIME_EVERY)
    for w in range(max(args.warmup, 3)):
        one_run(seed_base + 100 + w)
        run.sync()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(local)
    barrier()
    wall0 = time.perf_counter()
    pa.pa_kernel_time(run._h, True, TIME_EVERY)  # zero the counters, keep the graph
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    flips = 0
    for i in range(args.steps):
        flush.fill_(i)  # evict L2 between timed runs
        ev[i][0].record(stream)
        one_run(seed_base + i)
        ev[i][1].record(stream)
        flips += run_flips(run.trajectory(len(betas)), N, theta)
    sweep_ms, n_sweep, n_launch = pa.pa_kernel_time(run._h, False)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    gpu_ms = sum(a.elapsed_time(b) for a, b in ev)

    # e2e through the public C ABI with host buffers (create -> steps -> trajectory -> destroy)
    Jp = torch.empty(J.size, dtype=torch.int8, pin_memory=True).numpy()
    Jp[:] = J.reshape(-1)
    e2e_flips, e2e_t = 0, 0.0
    h2d = Jp.nbytes + 8 * (len(betas) - 1)
    d2h = 0
    for i in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = pa.pa_create(Jp, 8, 3, spec.R0, seed_base + 50 + i, pa.torch_opts())
        for k in range(1, len(betas)):
            pa.pa_step(h, float(betas[k]), theta)
        tr = pa.pa_trajectory(h, len(betas))
        pa.pa_destroy(h)
        e2e_t += time.perf_counter() - t0
        e2e_flips += run_flips(tr, N, theta)
        d2h = sum(v.nbytes for v in tr.values())

    flips_all, gpu_ms_max, e2e_f_all, e2e_t_max = aggregate_ranks(flips, gpu_ms, e2e_flips, e2e_t, dist)
    if rank != 0:
        return 0

    value = flips_all / (gpu_ms_max / 1000.0)
    shape = pa.pa_sweep_shape(run._h)  # (threads per block, threads per replica)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * sm_max * 1e6 / 1e12  # int32 lane ops/s, TOP/s
    per_launch_ms = sweep_ms / max(n_sweep, 1)  # mean over the sampled launches
    n_sweep_all = args.steps * (len(betas) - 1)  # one sweep launch per annealing step
    flips_per_launch = flips / n_sweep_all
    achieved = flips_per_launch * OPS_PER_FLIP / (per_launch_ms / 1000.0) / 1e12
    mul_bound = 152 * 64 * sm_max * 1e6 / (3.75 * 2)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": gpu_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f64",
        "data": "synthetic",
        "config": {"workload": spec_name(), "L": 8, "R0": spec.R0, "n_betas": len(betas), "theta": theta,
                   "execution": "200 steps replayed as one CUDA graph per run",
                   "spins": "bit-packed, 32-bit words", "l2": "flushed between timed runs (256 MB write)",
                   "parallelism": "replicas only" if ws > 1 else "single GPU"},
        "wall_s": wall,
        "roofline": {"bound": "alu", "kernel": f"k_sweep3d<8,{shape[0]},{shape[1]}>", "achieved": achieved,
                     "peak": alu_peak,
                     "unit": "TOP/s", "frac": achieved / alu_peak, "traffic": sweep_traffic(),
                     "ops_per_flip": OPS_PER_FLIP, "launch_ms": per_launch_ms,
                     "flips_per_launch": flips_per_launch,
                     "timed_launches": f"{n_sweep} of {n_sweep_all} (every {TIME_EVERY}th, CUDA events)",
                     "peak_source": "152 SMs x 128 int32 lanes x max SM clock (derived from unit counts and clock)",
                     # the bound the generator's multiplies alone set: 3.75 32x32->64
                     # multiplies per flip (15 per call of 4 uniforms, the first rounds
                     # tabulated), each 2 issue slots of the multiply pipe, which
                     # retires 64 lanes per cycle and SM
                     "multiply_pipe": {"flips_per_s_bound": mul_bound, "frac": flips_per_launch /
                                       (per_launch_ms / 1000.0) / mul_bound}},
        "e2e": {"value": e2e_f_all / e2e_t_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(n_launch),
        "clocks": clk,
    }
    # the long payloads first, so that the end of the line (which a truncated
    # log keeps) holds the CPU baseline and the metric's other two parts
    if args.gauss:
        line["gaussian"] = bench_gauss(pa, torch, args.gauss_study)
    if args.chain:
        line["chain"] = bench_chain(pa, torch)
    if not args.no_cpu_baseline and ws == 1:  # the oracle baseline at N=1 only
        cores = host_cores()
        (f, t), = oracle_sample_cores(BASE_R0, cores, 200)
        line["cpu_baseline"] = {"value": f / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"same couplings, R0={BASE_R0} per host core: init + all 200 annealing "
                                          f"steps (beta 0 -> 5), theta=10, one independent run per host core; "
                                          f"{t:.1f} s wall"}
    if args.batched:
        line["batched"] = bench_batched(pa, torch, args.batched_realisations)
    if args.serving:
        line["serving"] = bench_serving(pa, args.serving, value)
    print(json.dumps(line), flush=True)
    return 0


def bench_batched(pa, torch, n_real: int = 16, runs_per_real: int = 64):
    """Batched executor (all runs of all realisations through shared launches,
    the whole schedule captured in one CUDA graph, block size autotuned)
    against the plain form (each run alone, one launch per kernel per step),
    on the same runs; weighted averages per realisation (Eqs. (6)-(7))."""
    specs = inputs.config_batched(n_real, runs_per_real)
    betas = specs[0].betas
    n = len(specs)
    b = pa.Batch(specs, max_steps=len(betas))
    tuned = b.autotune(10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(betas[1:], thetas=10, use_graph=True)
    errs = b.sync()
    t_batch = time.perf_counter() - t0
    tr = b.trajectory(len(betas))
    res = b.results()
    flips_b = sum(int(np.sum(tr["R"][r, 1:])) * specs[r].N * 10 for r in range(n))
    b.close()
    # weighted averages over the runs of each realisation, R-weighted (Sec. 3)
    wav = []
    for d in range(n_real):
        sl = slice(d * runs_per_real, (d + 1) * runs_per_real)
        E = res["sumE"][sl] / res["R"][sl]
        m, f = pa.pa_weighted_average(res["minus_beta_F"][sl], E, np.array([s.R0 for s in specs[sl]], float))
        wav.append({"L": specs[d * runs_per_real].L, "E_bar": m, "minus_beta_F_bar": f,
                    "var_minus_beta_F": float(np.var(res["minus_beta_F"][sl], ddof=1))})
    # plain form: the same runs one at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    flips_p = 0
    for s in specs:
        r = pa.Run(s.couplings(), s.L, 3, s.R0, s.seed)
        for k in range(1, len(betas)):
            pa.pa_step(r._h, float(betas[k]), 10)
        flips_p += int(np.sum(r.trajectory(len(betas))["R"][1:])) * s.N * 10
        r.close()
    t_plain = time.perf_counter() - t0
    return {"workload": f"{n_real} realisations x {runs_per_real} runs, L = (6, 8, 10)[d mod 3], R0 uniform "
                        "in [2e4, 8e4], 101 betas 0..5, theta=10",
            "batched_flips_per_s": flips_b / t_batch, "batched_s": t_batch, "batched_errors": int(np.sum(errs != 0)),
            "plain_flips_per_s": flips_p / t_plain, "plain_s": t_plain,
            "speedup": (flips_b / t_batch) / (flips_p / t_plain), "autotuned": tuned,
            "weighted_averages_first_realisations": wav[:3]}


def chain_exact(J: np.ndarray, beta: float):
    """ln Z and <E> of the periodic chain, E = sum J_i s_i s_(i+1) with J =
    J_q 2^-15, by 2x2 transfer matrices renormalised at every bond (ln Z) and
    a central difference in beta (<E>)."""
    def lnZ(b):
        a = J.astype(np.float64) * 2.0 ** -15 * b
        M = np.eye(2)
        acc = 0.0
        for x in a:
            M = M @ np.array([[np.exp(-x), np.exp(x)], [np.exp(x), np.exp(-x)]])
            s = np.abs(M).max()
            M /= s
            acc += np.log(s)
        return acc + np.log(np.trace(M))
    h = 1e-6
    return lnZ(beta), -(lnZ(beta + h) - lnZ(beta - h)) / (2 * h)


def bench_gauss(pa, torch, study: bool = False):
    """The paper's Gaussian run sets (Sec. 4) through the batched executor,
    whole schedules in one graph launch each: 3D L=8, R=2000, theta=100, 25
    realisations x 50 runs; periodic chain N=256, R=1000, theta=50, 18 x 200.
    Weighted averages per realisation at the lowest temperature (Eqs. (6)-(7)),
    and for the chain the exact transfer-matrix values."""
    out = {}
    for name, specs, n_real in (("3d_L8", inputs.config_gauss_3d(), 25), ("1d_N256", inputs.config_gauss_1d(), 18)):
        betas = specs[0].betas
        theta = specs[0].theta
        per = len(specs) // n_real
        b = pa.Batch(specs, max_steps=len(betas))
        tuned = b.autotune(theta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(betas[1:], thetas=theta, use_graph=True)
        errs = b.sync()
        t = time.perf_counter() - t0
        tr = b.trajectory(len(betas))
        en = b.energy(len(betas))
        t1 = time.perf_counter()
        diag = b.diagnostics(per, len(betas))  # Sec. 3 estimators on the device, every realisation and beta
        boot = b.bootstrap(per, len(betas), B=100, seed=0)  # and their bootstrap errors
        t_diag = time.perf_counter() - t1
        extra = {}
        if specs[0].dim == 3 and study:
            extra = gauss_overlap_study(pa, b, specs, n_real, per, tr, diag)
        b.close()
        flips = int(np.sum(tr["R"][:, 1:])) * specs[0].N * theta
        rows = []
        for d in range(1):
            sl = slice(d * per, (d + 1) * per)
            row = {"realisation": d, "E_bar": float(diag["E_bar"][d, -1]),
                   "sd_E_bar": float(boot["sd_E_bar"][d, -1]),
                   "minus_beta_F_bar": float(diag["minus_beta_F_bar"][d, -1]),
                   "sd_minus_beta_F_bar": float(boot["sd_minus_beta_F_bar"][d, -1]),
                   "var_minus_beta_F": float(diag["var_minus_beta_F"][d, -1]),
                   "E_unweighted": float(np.mean(en["E_mean"][sl, -1]))}
            if specs[0].dim == 1:
                lz, ee = chain_exact(specs[d * per].couplings(), float(betas[-1]))
                row.update({"exact_minus_beta_F": lz, "exact_E": ee})
            rows.append(row)
        out[name] = {"workload": f"{n_real} x {per} runs, N={specs[0].N}, R={specs[0].R0}, theta={theta}, "
                                 f"{len(betas)} betas (the paper's schedule), one graph launch",
                     "flips_per_s": flips / t, "seconds": t, "errors": int(np.sum(errs != 0)),
                     "autotuned": tuned, "diagnostics_s": t_diag,
                     "max_var_minus_beta_F": float(diag["var_minus_beta_F"][:, -1].max()),
                     "lowest_temperature": rows, **extra}
    return out


def bench_chain(pa, torch):
    """C4: the open +-1 chain N = 4096, R0 = 2e5, 401 betas 0..4, theta = 5,
    8 runs (seeds 1..8, one realisation each) in one graph launch; the
    weighted -beta F and E over the 8 runs (Sec. 3) against the closed form
    ln Z = N ln 2 + (N - 1) ln cosh(beta), <E> = -(N - 1) tanh(beta), which
    every realisation of the open +-1 chain shares."""
    specs = inputs.config_chain()
    betas = specs[0].betas
    N = specs[0].N
    b = pa.Batch(specs, max_steps=len(betas))
    tuned = b.autotune(specs[0].theta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.run(betas[1:], thetas=specs[0].theta, use_graph=True)
    errs = b.sync()
    t = time.perf_counter() - t0
    tr = b.trajectory(len(betas))
    diag = b.diagnostics(len(specs), len(betas))
    boot = b.bootstrap(len(specs), len(betas), B=100, seed=0)
    b.close()
    flips = int(np.sum(tr["R"][:, 1:])) * N * specs[0].theta
    rows = []
    for beta in (1.0, 2.0, 4.0):
        k = int(round(beta / 4.0 * (len(betas) - 1)))
        lnz = N * math.log(2.0) + (N - 1) * math.log(math.cosh(betas[k]))
        fbar, sdf = float(diag["minus_beta_F_bar"][0, k]), float(boot["sd_minus_beta_F_bar"][0, k])
        ebar, sde = float(diag["E_bar"][0, k]), float(boot["sd_E_bar"][0, k])
        ex_e = -(N - 1) * math.tanh(betas[k])
        var = float(diag["var_minus_beta_F"][0, k])
        # |delta|/sigma against the closed form; the paper's criterion for a
        # trustworthy weighted average is Var(-beta F~) below about 0.5 (Sec. 3)
        rows.append({"beta": float(betas[k]), "minus_beta_F_bar": fbar, "sd_minus_beta_F_bar": sdf,
                     "exact_lnZ": lnz, "z_minus_beta_F": abs(fbar - lnz) / sdf if sdf > 0 else None,
                     "E_bar": ebar, "sd_E_bar": sde, "exact_E": ex_e,
                     "z_E": abs(ebar - ex_e) / sde if sde > 0 else None, "var_minus_beta_F": var,
                     "equilibrated": bool(var < 0.5)})
    return {"workload": "open +-1 chain N=4096, R0=2e5, 401 betas 0..4, theta=5, seeds 1..8, one graph launch",
            "flips_per_s": flips / t, "seconds": t, "errors": int(np.sum(errs != 0)), "autotuned": tuned,
            "closed_form": rows}


def gauss_overlap_study(pa, b, specs, n_real, per, tr, diag):
    """Sec. 4, 3D: Gamma = Prob(|q| < 0.2) from pairs of independent runs
    (runs 2i and 2i+1 of a realisation), their weighted average Gamma_bar
    (Eqs. (10)-(11)) per realisation, and its correlation with
    Var(-beta F~) over the realisations; then, for the realisation with the
    largest variance, the paper's temperature-dependent population (R = 1000
    below beta = 0.9, 3000 above) against the fixed R, same number of runs."""
    ra = [d * per + 2 * i for d in range(n_real) for i in range(per // 2)]
    rb = [r + 1 for r in ra]
    gamma, _ = b.overlap(ra, rb, 0.2)
    mbF = tr["minus_beta_F"][:, -1]
    half = per // 2
    gbar = []
    for d in range(n_real):
        sl = slice(d * half, (d + 1) * half)
        gbar.append(pa.pair_weighted_average(mbF[ra[sl.start:sl.stop]], mbF[rb[sl.start:sl.stop]], gamma[sl]))
    # the weighted P(q) (Eqs. (10)-(11)) of the realisation with the
    # largest Gamma_bar, from the per-pair histograms, on 16 bins of q
    top = int(np.argmax(gbar))
    pairs = slice(top * half, (top + 1) * half)
    hist = b.overlap_hist(ra[pairs], rb[pairs]).astype(np.float64)
    N = specs[0].N
    qv = (2.0 * np.arange(N + 1) - N) / N
    edges = np.linspace(-1.0, 1.0, 17)
    coarse = np.stack([hist[:, (qv >= lo) & ((qv < hi) | (hi == 1.0) & (qv <= hi))].sum(axis=1)
                       for lo, hi in zip(edges[:-1], edges[1:])], axis=1)
    coarse /= coarse.sum(axis=1, keepdims=True)
    pq = [pa.pair_weighted_average(mbF[ra[pairs]], mbF[rb[pairs]], coarse[:, i]) for i in range(16)]
    var = diag["var_minus_beta_F"][:, -1]
    worst = int(np.argmax(var))
    betas = specs[0].betas
    Rt = np.where(betas[1:] < 0.9, 1000, 3000)
    sp = [inputs.RunSpec(3, 8, worst, (worst << 8) | (128 + r), 1000, betas, specs[0].theta, gaussian=True,
                         R_cap=3800) for r in range(per)]
    bv = pa.Batch(sp, max_steps=len(betas))
    t0 = time.perf_counter()
    bv.run(betas[1:], thetas=specs[0].theta, R_targets=Rt)
    bv.sync()
    t_var = time.perf_counter() - t0
    dv = bv.diagnostics(per, len(betas))
    bv.close()
    return {"overlap_qcut": 0.2,
            "gamma_bar_per_realisation": [float(g) for g in gbar],
            "var_minus_beta_F_per_realisation": [float(v) for v in var],
            "corr_var_gamma_bar": float(np.corrcoef(var, gbar)[0, 1]),
            "P_q_weighted": {"realisation": top, "q_bin_edges": [float(x) for x in edges],
                             "P": [float(x) for x in pq]},
            "temperature_dependent_R": {"realisation": worst, "R_fixed_2000_var": float(var[worst]),
                                        "R_1000_3000_var": float(dv["var_minus_beta_F"][0, -1]),
                                        "runs": per, "seconds": t_var}}


def bench_serving(pa, n_req: int, capacity_flips_per_s: float, load: float = 0.8):
    """Poisson stream of annealing requests (L in {4..12}, R0 in [1e4, 2e5],
    51-201 betas, theta=10) at `load` times the measured throughput, served
    by continuous batching; p50/p99 latency from submission to result."""
    probe = inputs.serving_requests(n_req, rate_per_s=1.0)
    mean_flips = float(np.mean([q.spec.flips for q in probe]))
    rate = load * capacity_flips_per_s / mean_flips
    reqs = inputs.serving_requests(n_req, rate_per_s=rate)
    srv = pa.Server(max_runs=1024)
    ids = []
    i = 0
    done = 0
    t0 = time.perf_counter()
    max_active = 0
    while done < n_req:
        now = time.perf_counter() - t0
        while i < n_req and reqs[i].arrival_s <= now:
            q = reqs[i].spec
            ids.append(srv.submit(3, q.L, q.couplings(), q.R0, q.seed, q.betas[1:], q.theta))
            i += 1
        a, qd, f = srv.tick(2)
        done += f
        max_active = max(max_active, a + f)
        if a == 0 and qd == 0 and i < n_req:
            time.sleep(max(0.0, reqs[i].arrival_s - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    res = [srv.result(r) for r in ids]
    srv.close()
    lat = np.array([r["done_s"] - r["submit_s"] for r in res])
    flips = sum(r["flips"] for r in res)
    span = max(r["done_s"] for r in res) - min(r["submit_s"] for r in res)
    return {"workload": f"{n_req} requests, Poisson arrivals (seed 5) at {rate:.3f}/s = {load} x measured "
                        "capacity, L in {4,6,8,10,12}, R0 in [1e4, 2e5], 51-201 betas 0..5, theta=10",
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "flips_per_s": flips / span, "wall_s": wall, "failed": int(sum(r["status"] != 2 for r in res)),
            "max_concurrent_runs": max_active}


if __name__ == "__main__":
    sys.exit(main())
