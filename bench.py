"""Benchmark of the GB300 LMM PF-SMC sampler (particle-LMM-steps/s).

One step = one epoch of Algorithm 1 (Steps 2-6: shrink, propagate, first-stage
weights, systematic resampling, proliferation, repropagation with the
local-error innovation, reweighting, moments) over the Robertson workload:
N = 131072 particles, d = 3, p = 3, 50 geometric BDF2 substeps per interval,
K = 2 Newton iterations, FP64.  One particle-LMM-step is one implicit substep
(with its Newton iterations) of one particle; an epoch is 2 * S * N of them.

value     device-resident inputs (the whole observation series uploaded once),
          CUDA-event time of each step on the filter's stream, L2 flushed
          (256 MiB write) before every step, summed over K steps; the filter
          records its own events around stage 2 only.
e2e       the same metric through the C ABI with host buffers: pf_assimilate
          (host y_k, parameter upload) + pf_estimates (host read-back), wall
          time per step.
roofline  the dominant kernel (stage 2) against the FP64 ALU peak.
cpu_baseline / --impl reference: the CPU oracle on the host cores.
The default run adds the batched workload (256 filters of 2^10..2^17
particles, and 256 of 2^10..2^11) against per-filter launches, and the
serving trace's latency with a sweep of loads below capacity.

Multi-GPU (torchrun): independent replicas (one filter per rank, different
seeds); value = all ranks' particle-steps / the slowest rank's time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1411_1702_gb300.workloads import ADVDIFF as W_ADVDIFF  # noqa: E402
from paper_1411_1702_gb300.workloads import LMM_NAMES as W_LMM_NAMES  # noqa: E402

METRIC = "particle-LMM-steps/s"
UNIT = "particle-steps/s"
# FP64 ALU peak of one GB300: 2 FP64 FMA lanes per clock per SM (the
# sustained peak ncu reports for sm__sass_thread_inst_executed_op_dfma_pred_on
# on this part) x 152 SMs x 2070 MHz maximum SM clock x 2 flops per FMA
# = 1.259 TFLOP/s, the nominal GB300 FP64 rate.
FP64_PEAK_TFLOPS = 2.0 * 152 * 2.070e9 * 2 / 1e12

# Algorithmic FP64 flops (FMA = 2, a reciprocal = 1) of one substep of one
# particle in the stage-2 kernel: predictor 5d, history combination 3d, Milne
# estimate 4d, per-substep constants, and K Newton iterations.
def _advdiff_inverse_flops(nt, H):
    """One inverse transform of the half spectrum organised by twiddle
    symmetry: pair sums and differences 4 per unit (H^2 units), columns
    8 (H-1) + 4 per unit, Hermitian rows 4 (H-1) + 6 per (row, pair) unit."""
    units = H * H
    return 4 * units + units * (8 * (H - 1) + 4) + nt * H * (4 * (H - 1) + 6)


def _advdiff_flops(K, d):
    """M2 (2D advection-diffusion), stage 2 per substep, with nt = sqrt(d) and
    H = (nt+1)/2: per mode (nt H of them) the history combination,
    predictor, division by 1 - gamma lambda and Milne estimate (26 flops);
    the inverse transform of the local error; the squared-error sums 2d."""
    nt = int(round(math.sqrt(d)))
    H = (nt + 1) // 2
    return 26 * nt * H + _advdiff_inverse_flops(nt, H) + 2 * d


def _advdiff_flops_interval(K, d):
    """M2, stage 2 once per interval: three forward transforms of the history
    (rows of both members of a row pair, 8 nt per unit, and their sums and
    differences 4; columns 8 (H-1) + 4 per unit), the symbol of both modes of
    a unit (40) and its inverse factor (20), three inverse transforms of the
    final states with their 1/d scaling, and the innovation (5d)."""
    nt = int(round(math.sqrt(d)))
    H = (nt + 1) // 2
    units = H * H
    forward = units * (8 * nt + 4) + units * (8 * (H - 1) + 4)
    return (3 * forward + 60 * units + 3 * (_advdiff_inverse_flops(nt, H) + 4 * units)
            + 5 * d)


def _michaelis_flops(lmm):
    """M1 (Sec. 2.1), d = 3: one Newton iteration (two flux reciprocals, the
    fluxes as g V - (g V k) q, the residual by additions, the lower-triangular
    substitution with two pivot reciprocals) is 30 flops, one evaluation of f
    17.  Per substep, by family: BDF1/BDF2 predictor 15, history 9, input 2,
    pivot, flux and residual constants 14, Milne 12; BDF3 adds the slope
    f(t_n, x_n) and its term (81 in all); Adams-Moulton: AB predictor 18, AM
    history 12, input 2, constants 14, f(x_{n+1}) 17, Milne 12;
    Adams-Bashforth: predictor 18, history 12, f 17, Milne against AM 18 (no
    Newton)."""
    fam = lmm // 10
    if fam == 2:
        return lambda K, d: 65
    if fam == 1:
        return lambda K, d: 75 + 30 * K
    if lmm == 3:
        return lambda K, d: 81 + 30 * K
    return lambda K, d: 52 + 30 * K


# Exact FP64 operations of one steady-state particle-substep of the oracle's
# propagation with Step 4's Milne sums (additions, multiplications, divisions,
# square roots; a multiply-add is 2), from the op-counting build of the oracle:
# written by `python oracle/count_flops.py` (tests/test_opcount.py checks this
# copy against it).  For the problems of d <= 3, whose Newton system the
# oracle solves as the method states it (dense LU of I - gamma J), this is the
# algorithmic work the roofline divides by time; the kernels' own counts below
# (their specialised eliminations do less) are reported beside it.
ORACLE_SUBSTEP_FLOPS = {
    "linear2": {"K": 1, "flops": 49},
    "michaelis": {"K": 4, "flops": 364},
    "michaelisAB1": {"K": 4, "flops": 56},
    "michaelisAB2": {"K": 4, "flops": 85},
    "michaelisAB3": {"K": 4, "flops": 115},
    "michaelisAM1": {"K": 4, "flops": 378},
    "michaelisAM2": {"K": 4, "flops": 407},
    "michaelisAM3": {"K": 4, "flops": 437},
    "michaelisBDF1": {"K": 4, "flops": 371},
    "michaelisBDF2": {"K": 4, "flops": 364},
    "michaelisBDF3": {"K": 4, "flops": 392},
    "robertson": {"K": 2, "flops": 192},
}

STAGE2_FLOPS_PER_SUBSTEP = {
    # per Newton iteration: Robertson 41 (the first residual row one FMA on
    # its pivot 1 + g k1), linear2 12 (both rows on their pivots)
    "robertson": lambda K, d: 15 + 9 + 12 + 8 + 41 * K,
    "linear2": lambda K, d: 10 + 6 + 8 + 20 + 12 * K,
    # 32 grid points x 67 flops per Newton iteration (residual 16, 2x2 block,
    # Thomas forward and backward), predictor 5d, history 3d (+ the u rows'
    # g A, 1 each), Milne 4d, constants
    "brusselator": lambda K, d: 320 + 224 + 256 + 15 + 2144 * K,
    "advdiff20": _advdiff_flops,
    "advdiff40": _advdiff_flops,
}
for _name, _lmm in W_LMM_NAMES.items():
    STAGE2_FLOPS_PER_SUBSTEP["michaelis" + _name] = _michaelis_flops(_lmm)
STAGE2_FLOPS_PER_SUBSTEP["michaelis"] = _michaelis_flops(2)
# Stage-2 flops spent once per interval rather than per substep
STAGE2_FLOPS_PER_INTERVAL = {"advdiff20": _advdiff_flops_interval,
                             "advdiff40": _advdiff_flops_interval}
STAGE2_KERNEL = {"robertson": "k_stage2<Robertson>", "linear2": "k_stage2<Linear2>",
                 "brusselator": "k_bstage2", "advdiff20": "k_adstage<2, 1, 2>",
                 "advdiff40": "k_adstage<2, 1, 1>"}
_FAMILY_ID = {0: 0, 1: 2, 2: 3}
for _name, _lmm in W_LMM_NAMES.items():
    _fam = 1 if _lmm == 3 else _FAMILY_ID[_lmm // 10]
    STAGE2_KERNEL["michaelis" + _name] = f"k_stage2<Michaelis, {_fam}>"
STAGE2_KERNEL["michaelis"] = "k_stage2<Michaelis, 0>"
# DRAM bytes (read + write) of one stage-2 launch from an ncu capture of the
# same command on a GB300 (profiles/ names each capture); None where no capture
# of the kernel as it stands exists.
STAGE2_TRAFFIC = {"robertson": 11549184 + 0,
                  "brusselator": 11237054976 + 10729370624,
                  "advdiff20": 3076608 + 756736,
                  "advdiff40": 177258240 + 138143744,
                  "michaelisBDF2": 4355584 + 0,
                  "michaelisAM3": 4590336 + 0,
                  "michaelisAB3": 4454144 + 0}
# The paper's own number for the same workload, where it has one: Table 3's
# 2D advection-diffusion runs (BDF2, h = 0.1, N = 5000, 30 unit intervals,
# 8 MATLAB workers on an i7-3820), converted to particle-LMM-steps/s at 600
# steps per particle per run.
PAPER_BASELINE = {"advdiff20": 3.0e6 / 7.20e3, "advdiff40": 3.0e6 / 3.39e4}
# The ensemble size each traffic capture was taken at (traffic is reported only
# for that size).
TRAFFIC_N = {"robertson": 131072, "brusselator": 65536, "advdiff20": 5000, "advdiff40": 5000,
             "michaelisBDF2": 50000, "michaelisAM3": 50000, "michaelisAB3": 50000}
# the N range of the default run's second batched comparison (small filters)
SMALL_BATCH_LOG2N = (10.0, 11.0)
# epochs of the per-kernel breakdown pass that follows the timed region
BREAKDOWN_EPOCHS = 60
# Algorithmic DRAM bytes per particle of the scan and resampling launches:
# the tile scan reads log g and writes the tile-local c, resampling reads c
# (applying the tile offsets) and writes the int32 index.
SUPPORT_BYTES = {"scan_tile": 16, "resample": 12}


def hbm_peak():
    """The measured copy bandwidth of the GB300s (GB/s), else the
    profiling recipe's fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"
# Particles of the timed CPU-oracle sample, where the workload's own N would
# take minutes per epoch on the host cores.
CPU_SAMPLE_N = {"advdiff20": 512, "advdiff40": 48}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    backend = "nccl" if os.environ.get("PF_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
    dist.init_process_group(backend)
    return dist, dist.get_rank(), dist.get_world_size()


def reduce_times(dist, total_ms, steps_done, device=None):
    """Max of the per-rank times and sum of the per-rank particle-steps."""
    if dist is None:
        return total_ms, steps_done
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    s = torch.tensor([float(steps_done)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def fp64_fma_rate(ms, stream):
    """TFLOP/s of the benchmark's FP64 FMA probe (libpf_fp64_probe.so, built
    beside the library; not part of its C ABI), or None if it fails."""
    import ctypes as C
    from paper_1411_1702_gb300 import build as B
    lib = C.CDLL(B.PROBE_LIB)
    lib.fp64_fma_rate.restype = C.c_int
    lib.fp64_fma_rate.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_double)]
    out = C.c_double()
    rc = lib.fp64_fma_rate(C.c_void_p(stream) if stream else None, float(ms), C.byref(out))
    return out.value if rc == 0 else None


def device_sms():
    """SM count of GPU 0 (152 on a GB300), or 152 without a GPU."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(0).multi_processor_count)
    except Exception:  # noqa: BLE001 - no device: the GB300's count
        pass
    return 152


def epoch_launches(w, sms=None):
    """Kernels of one single-filter epoch: stage 1, scan tile, resampling
    (which applies the tile offsets as it reads c), stage 2, moments; plus the
    state mean of the 2D system and the corner pass of a resampling above one
    wave of merge tiles (the library's rs_two_phase: more than 4 tiles of 1024
    items for each of the device's SMs)."""
    sms = device_sms() if sms is None else sms
    n = 5 + (1 if w.ode == W_ADVDIFF else 0)
    return n + (1 if (2 * w.N + 1023) // 1024 > 4 * sms else 0)


def support_roofline(ktimes, N):
    """Achieved bandwidth of the scan and resampling phases (algorithmic bytes
    over their mean device time) against the HBM peak."""
    peak, src = hbm_peak()
    out = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": src, "kernels": {}}
    for name, bpp in SUPPORT_BYTES.items():
        ms, n = ktimes.get(name, (0.0, 0))
        if n and ms > 0.0:
            us = ms / n * 1e3
            gbs = bpp * N / (us * 1e-6) / 1e9
            out["kernels"][name] = {"us": us, "bytes": bpp * N, "achieved": gbs, "frac": gbs / peak}
    return out


def cpu_oracle_rate(w, seconds=12.0, max_epochs=None, N=None):
    """The oracle as it stands on the host cores: epochs of the same workload
    until `seconds` of work; returns (steps/s, cores, sample text)."""
    import oracle
    oracle.build()
    o = oracle.Filter(w, N=N)
    o.init()
    n = o.N
    steps, spent, k, passes, done = 0, 0.0, 0, 1, 0
    limit = max_epochs or w.T
    while spent < seconds or done < 2:
        if k == limit:
            if max_epochs:
                break
            # the whole series took less than the budget: run it again from Step 1
            # (not timed), as bench.py's GPU leg does
            o.init()
            k, passes = 0, passes + 1
        t0 = time.perf_counter()
        rc = o.epoch(w.t_obs[k], w.y_obs[k])
        spent += time.perf_counter() - t0
        if rc != oracle.OK:
            break
        steps += 2 * w.substeps_per_interval(k) * n
        k, done = k + 1, done + 1
    what = (f"first {k} epochs" if passes == 1 else
            f"{done} epochs ({passes} passes over the {limit}-epoch series)")
    return steps / spent, oracle.threads(), f"{what} of the workload at N={n} ({spent:.1f} s)"


def run_reference(args, w):
    dist, rank, world = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_ref = min(w.N, args.ref_particles or w.N, CPU_SAMPLE_N.get(w.name, w.N))
    o = oracle.Filter(w, N=n_ref)
    o.init()
    k = 0
    for _ in range(args.warmup):
        o.epoch(w.t_obs[k], w.y_obs[k])
        k += 1
    total, steps = 0.0, 0
    for _ in range(args.steps):
        if k >= w.T:
            o.init()
            k = 0
        t0 = time.perf_counter()
        rc = o.epoch(w.t_obs[k], w.y_obs[k])
        total += time.perf_counter() - t0
        if rc != oracle.OK:
            raise RuntimeError(f"oracle epoch failed: {rc}")
        steps += 2 * w.substeps_per_interval(k) * n_ref
        k += 1
    value = steps / total
    sample = (f"one epoch per step of the workload at its N={n_ref}" if n_ref == w.N else
              f"one epoch per step at N={n_ref} (the workload's N={w.N} would take minutes)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w.with_(N=n_ref)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(w):
    lmm = next((k for k, v in W_LMM_NAMES.items() if v == w.lmm), str(w.lmm))
    return {"workload": f"{w.name}: N={w.N} d={w.d} p={w.p} m={w.m} S={w.substeps_per_interval(1)} "
                        f"{'geometric' if w.spacing else 'uniform'} substeps, T={w.T}, {lmm}, "
                        f"K={w.newton_iters} Newton, FP64",
            "N": w.N, "substeps": w.substeps_per_interval(1), "newton_iters": w.newton_iters,
            "epochs_per_step": 1, "l2": "flushed before every step (256 MiB write)",
            "parallelism": "replicas"}


def run_ours(args, w):
    import torch
    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1411_1702_gb300 import build as B
    B.build()
    from paper_1411_1702_gb300 import pf
    # a dedicated stream: the library's kernels, the L2 flush and the timing
    # events are all ordered on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.profile:
        return run_profile(args, w, pf, stream)
    # timing events around stage 2 only (the dominant kernel the roofline
    # times): the other kernel boundaries keep their programmatic launch
    # overlap, which events between kernels would remove
    g = pf.Filter.from_workload(w, stream=stream.cuda_stream, seed=w.seed + rank, filter_id=rank,
                                timing=2)
    g.pf_load_observations(w.t_obs, w.y_obs)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    k = 0

    def next_epoch():
        nonlocal k
        if k >= w.T:
            g.pf_reset()
            k = 0
        g.pf_run(k, k + 1)
        k += 1
        return k - 1

    for _ in range(args.warmup):
        next_epoch()
    g.pf_synchronize()
    g.pf_kernel_times()  # drop the warm-up timings
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    steps_done = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for s in range(args.steps):
            if k >= w.T:
                g.pf_reset()
                k = 0
            flush.zero_()
            starts[s].record(stream)
            kk = next_epoch()
            ends[s].record(stream)
            steps_done += w.particle_steps(kk)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    g.pf_synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    ktimes = g.pf_kernel_times()
    total_max, steps_all = reduce_times(dist, total_ms, steps_done, device="cuda")
    value = steps_all / (total_max * 1e-3)
    # the per-kernel breakdown, after the timed region: a pass with events
    # around every kernel (each epoch after an L2 flush, as above)
    kb = min(args.steps, BREAKDOWN_EPOCHS)
    gb = pf.Filter.from_workload(w, stream=stream.cuda_stream, seed=w.seed + rank, filter_id=rank,
                                 timing=True)
    gb.pf_load_observations(w.t_obs, w.y_obs)
    kq = 0
    for i in range(args.warmup + kb):
        if i == args.warmup:
            gb.pf_synchronize()
            gb.pf_kernel_times()  # drop the warm-up timings
        if kq >= w.T:
            gb.pf_reset()
            kq = 0
        flush.zero_()
        gb.pf_run(kq, kq + 1)
        kq += 1
    kall = gb.pf_kernel_times()
    gb.close()

    # e2e through the C ABI with host buffers, on a filter as a user creates
    # it (no per-kernel timing events)
    e2e_steps = min(args.steps, args.e2e_steps)
    ge = pf.Filter.from_workload(w, stream=stream.cuda_stream, seed=w.seed + rank, filter_id=rank)
    ke, wall, e2e_done = 0, 0.0, 0
    st0 = ge.pf_stats()
    for _ in range(e2e_steps):
        if ke >= w.T:
            ge.pf_reset()
            ke = 0
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ge.pf_assimilate(w.t_obs[ke], w.y_obs[ke])
        ge.pf_estimates()
        wall += time.perf_counter() - t0
        e2e_done += w.particle_steps(ke)
        ke += 1
    st1 = ge.pf_stats()
    ge.close()
    wall_max, e2e_all = reduce_times(dist, wall * 1e3, e2e_done, device="cuda")
    # the FP64 FMA rate this GPU sustains (after the timed regions): checks
    # that the nominal FP64 peak used as the roofline denominator is reached
    fma_measured = fp64_fma_rate(200.0, stream.cuda_stream)
    e2e_value = e2e_all / (wall_max * 1e-3)
    # only the data of the steps themselves (the resets in between are not steps)
    h2d = (st1["h2d_bytes"] - st0["h2d_bytes"]) / e2e_steps
    d2h = (st1["d2h_bytes"] - st0["d2h_bytes"]) / e2e_steps

    if rank != 0:
        g.close()
        return 0
    base = PAPER_BASELINE.get(w.name)
    vs_base = value / base if base else None
    # roofline of the dominant kernel: stage 2 (repropagation)
    ms2, n2 = ktimes["stage2"]
    S = w.substeps_per_interval(1)
    kflops = STAGE2_FLOPS_PER_SUBSTEP[w.name](w.newton_iters, w.d) * S * w.N
    if w.name in STAGE2_FLOPS_PER_INTERVAL:
        kflops += STAGE2_FLOPS_PER_INTERVAL[w.name](w.newton_iters, w.d) * w.N
    oc = ORACLE_SUBSTEP_FLOPS.get(w.name)
    counted = oc is not None and oc["K"] == w.newton_iters
    flops = oc["flops"] * S * w.N if counted else kflops
    per_s = (ms2 / n2 * 1e-3) if n2 else None
    achieved = flops / per_s / 1e12 if per_s else None
    k_achieved = kflops / per_s / 1e12 if per_s else None
    shares = {name: round(ms / max(1e-12, sum(v[0] for v in kall.values())), 4)
              for name, (ms, _) in kall.items()}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": vs_base, "dtype": "f64", "data": "synthetic",
        "config": config_of(w), "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(round(h2d)),
                "d2h_bytes_per_step": int(round(d2h))},
        # the library's kernels in the timed region (epoch_launches)
        "gpu_launches": epoch_launches(w) * args.steps,
        "roofline": {"bound": "alu", "kernel": STAGE2_KERNEL[w.name], "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                     "count": ("the oracle's exact operation count of a substep (dense Newton), "
                               f"{oc['flops']} flops" if counted else
                               "the kernel's own count of its algorithm"),
                     "kernel_count_achieved": k_achieved,
                     "frac_kernel_count": (k_achieved / FP64_PEAK_TFLOPS) if k_achieved else None,
                     "traffic": (STAGE2_TRAFFIC.get(w.name)
                                 if TRAFFIC_N.get(w.name) == w.N else None),
                     "peak_source": "2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz (nominal GB300 FP64)",
                     "fp64_fma_measured": fma_measured,
                     "frac_of_measured_fma": (achieved / fma_measured) if achieved and fma_measured else None},
        "kernel_share": shares,
        "kernel_ms_per_step": {k2: v[0] / max(1, v[1]) for k2, v in kall.items()},
        "kernel_breakdown": (f"events around every kernel, a separate pass of {kb} epochs after "
                             "the timed region (which has events around stage 2 only)"),
        "support_roofline": support_roofline(kall, w.N),
    }
    if not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(w, seconds=args.cpu_seconds,
                                              N=CPU_SAMPLE_N.get(w.name))
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample}
        # and on one core, a shorter sample
        import oracle
        oracle.set_threads(1)
        rate1, _, sample1 = cpu_oracle_rate(w, seconds=args.cpu_seconds / 3.0,
                                            N=CPU_SAMPLE_N.get(w.name))
        oracle.set_threads(cores)
        line["cpu_baseline"]["single_thread"] = {"value": rate1, "sample": sample1}
    g.close()
    if world == 1 and args.patterns and args.workload == "robertson":
        # the metric's other halves on the same GPU: the batched workload
        # against per-filter launches, and serving latency
        b = batched_result(args)
        keys = ("value", "unit", "ms_per_step", "steps", "config", "clocks", "e2e",
                "per_filter_sync", "per_filter_streams", "speedup_vs_per_filter_sync",
                "speedup_vs_per_filter_streams", "autotune")
        line["batched"] = {k: b[k] for k in keys}
        # the same comparison where one filter's launches underfill the GPU:
        # 256 filters of 2^10 to 2^11 particles
        small = argparse.Namespace(**dict(vars(args), batch_log2n=list(SMALL_BATCH_LOG2N)))
        bs = batched_result(small)
        line["batched_small_filters"] = {k: bs[k] for k in keys}
        sv = serving_result(args)
        line["serving"] = {k: sv[k] for k in ("value", "unit", "config", "clocks", "server",
                                              "server_one_lane", "serial_per_filter",
                                              "throughput_vs_serial", "p99_vs_serial")}
        if "load_sweep" in sv:
            line["serving"]["load_sweep"] = sv["load_sweep"]
    print(json.dumps(line), flush=True)
    return 0


def run_profile(args, w, pf, stream):
    """Plain launcher for profilers: Step 1, then warmup + steps epochs of the
    loaded series on one stream, no timing, no CPU work.  Launch order: k_init,
    k_moments, then per epoch k_stage1, k_scan_tile, (k_rs_corners above one
    wave of merge tiles,) k_resample, k_stage2, k_moments (and k_xbar for the
    2D system)."""
    g = pf.Filter.from_workload(w, stream=stream.cuda_stream)
    g.pf_load_observations(w.t_obs, w.y_obs)
    n = min(args.warmup + args.steps, w.T)
    for k in range(n):
        g.pf_run(k, k + 1)
    g.pf_synchronize()
    g.close()
    print(json.dumps({"profile_run": w.name, "N": w.N, "epochs": n}), flush=True)
    return 0


def shard_by_work(work, world):
    """Independent filters over ranks: largest first, each to the rank with
    the least work so far (ties to the lower rank).  Returns one list of
    filter indices per rank; deterministic, disjoint, covering."""
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(work)), key=lambda j: (-work[j], j)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += work[i]
    return [sorted(o) for o in out]


def run_batched(args):
    line = batched_result(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


def batched_result(args):
    """Batched pattern: 256 independent filters of uneven N (2^10..2^17) and
    mixed problems advanced round by round (a round = every filter that still
    has an observation assimilates its next one).  The same rounds run three
    ways: one pf_batch (tile-scheduled launches in a CUDA graph), per-filter
    synchronous pf_assimilate calls, and per-filter asynchronous launches
    with each filter on its own stream."""
    import torch
    from paper_1411_1702_gb300 import workloads as W
    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    lo2, hi2 = args.batch_log2n
    ws_all = W.batched(args.batch_filters, n_min_log2=lo2, n_max_log2=hi2)
    # with several ranks, the filters are sharded (no collective on the data
    # path); each keeps its global filter id, so its results do not change
    # (work: the stage-2 flops of the whole series, as the roofline counts them)
    mine = shard_by_work([STAGE2_FLOPS_PER_SUBSTEP[w.name](w.newton_iters, w.d) * w.N *
                          sum(w.substeps_per_interval(k) for k in range(w.T)) for w in ws_all],
                         world)[rank]
    ws = [ws_all[i] for i in mine]
    ids = list(mine)
    torch.cuda.set_device(local)
    from paper_1411_1702_gb300 import build as B
    B.build()
    from paper_1411_1702_gb300 import pf
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n = len(ws_all)
    R = max(w.T for w in ws_all)

    def inputs(r):
        return ([w.t_obs[r] if r < w.T else 0.0 for w in ws],
                [w.y_obs[r] if r < w.T else None for w in ws])

    def steps(r):
        return sum(w.particle_steps(r) for w in ws if r < w.T)

    K = min(args.steps, R - args.warmup)
    timed = range(args.warmup, args.warmup + K)
    my_steps = sum(steps(r) for r in timed)

    def sync_ranks():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # 1. the batch
    fb = [pf.Filter.from_workload(w, stream=stream.cuda_stream, filter_id=i) for i, w in zip(ids, ws)]
    batch = pf.Batch(fb, stream=stream.cuda_stream)
    if args.profile:
        # plain launcher for profilers: warmup + steps rounds, no timing
        for r in range(min(args.warmup + args.steps, R)):
            batch.pf_batch_assimilate(*inputs(r))
        torch.cuda.synchronize()
        batch.close()
        return None
    for r in range(args.warmup):
        batch.pf_batch_assimilate(*inputs(r))
    dev_ms, wall = 0.0, 0.0
    sync_ranks()
    with ClockSampler(local) as clocks:
        for r in timed:
            t0 = time.perf_counter()
            st = batch.pf_batch_assimilate(*inputs(r))
            wall += time.perf_counter() - t0
            dev_ms += batch.pf_batch_stats()["last_device_ms"]
            assert all(s == pf.PF_OK for s in st), st
    bstats = batch.pf_batch_stats()
    batch.close()
    for f in fb:
        f.close()
    torch.cuda.synchronize()
    # 2. per-filter synchronous calls
    fs = [pf.Filter.from_workload(w, filter_id=i) for i, w in zip(ids, ws)]
    for r in range(args.warmup):
        t, y = inputs(r)
        for i, f in enumerate(fs):
            if y[i] is not None:
                f.pf_assimilate(t[i], y[i])
    wall_sync = 0.0
    sync_ranks()
    for r in timed:
        t, y = inputs(r)
        t0 = time.perf_counter()
        for i, f in enumerate(fs):
            if y[i] is not None:
                f.pf_assimilate(t[i], y[i])
        wall_sync += time.perf_counter() - t0
    for f in fs:
        f.close()
    # 3. per-filter asynchronous launches, one stream per filter
    fa = [pf.Filter.from_workload(w, filter_id=i) for i, w in zip(ids, ws)]
    for f, w in zip(fa, ws):
        f.pf_load_observations(w.t_obs, w.y_obs)
    for r in range(args.warmup):
        for f, w in zip(fa, ws):
            if r < w.T:
                f.pf_run(r, r + 1)
        for f in fa:
            f.pf_synchronize()
    wall_async = 0.0
    sync_ranks()
    for r in timed:
        t0 = time.perf_counter()
        for f, w in zip(fa, ws):
            if r < w.T:
                f.pf_run(r, r + 1)
        for f in fa:
            f.pf_synchronize()
        wall_async += time.perf_counter() - t0
    for f in fa:
        f.close()
    # the slowest rank's times, every rank's particle-steps
    dev_ms, total_steps = reduce_times(dist, dev_ms, my_steps, device="cuda")
    wall, _ = reduce_times(dist, wall * 1e3, 0, device="cuda")
    wall_sync, _ = reduce_times(dist, wall_sync * 1e3, 0, device="cuda")
    wall_async, _ = reduce_times(dist, wall_async * 1e3, 0, device="cuda")
    wall, wall_sync, wall_async = wall * 1e-3, wall_sync * 1e-3, wall_async * 1e-3
    if rank != 0:
        return None
    value = total_steps / (dev_ms * 1e-3)
    line = {
        "metric": METRIC, "mode": "batched", "value": value, "unit": UNIT, "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": dev_ms / K, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batched: {n} filters, N = round(2^U[{lo2:g},{hi2:g}]) "
                               f"(total {sum(w.N for w in ws_all)}), linear2/robertson 50/50, "
                               "one round per step", "filters": n,
                   "robertson_filters": sum(w.ode == W.ROBERTSON for w in ws_all),
                   "particles": sum(w.N for w in ws_all),
                   "l2": "working set ~2 GB > L2, no flush",
                   "parallelism": ("one GPU" if world == 1 else
                                   f"filters sharded over {world} ranks by work, no collective")},
        "clocks": clocks.summary(),
        "e2e": {"value": total_steps / wall, "unit": UNIT},
        "per_filter_sync": {"value": total_steps / wall_sync, "unit": UNIT,
                            "how": "pf_assimilate per filter, one after another"},
        "per_filter_streams": {"value": total_steps / wall_async, "unit": UNIT,
                               "how": "pf_run per filter, each on its own stream, then sync"},
        "speedup_vs_per_filter_sync": (total_steps / wall) / (total_steps / wall_sync),
        "speedup_vs_per_filter_streams": (total_steps / wall) / (total_steps / wall_async),
        "autotune": {"tile_order": bstats["tile_order"],
                     "concurrent_models": bstats["concurrent_models"],
                     "candidate_ms": bstats["tune_ms"]},
        "graph_captures": bstats["graph_captures"],
    }
    return line


def run_serving(args):
    print(json.dumps(serving_result(args)), flush=True)
    return 0


def serving_result(args):
    """Serving pattern: a trace of filter sessions arriving as a Poisson
    process, each with observations arriving at exponential intervals, served
    in real time three ways: the server (memory-budget admission, continuous
    batching over lanes), the server with a single lane, and serial
    per-filter calls (each observation assimilated with pf_assimilate, in
    arrival order, the filter created when its session opens).  Latency is
    arrival -> device completion of the assimilation."""
    import torch
    from paper_1411_1702_gb300 import workloads as W
    trace = W.serving(n_sessions=args.serve_sessions, obs_per_session=args.serve_obs)
    torch.cuda.set_device(0)
    from paper_1411_1702_gb300 import build as B
    B.build()
    from paper_1411_1702_gb300 import pf

    # warm-up: a short trace through both paths (kernels loaded, pools primed)
    warm = W.serving(n_sessions=6, obs_per_session=3, seed=99)
    srv = pf.Server(budget_bytes=8 << 30)
    for s, ss in enumerate(warm):
        sid = srv.pf_server_open(ss.w, filter_id=s)
        for k in range(3):
            srv.pf_server_submit(sid, ss.w.t_obs[k], ss.w.y_obs[k])
    srv.pf_server_drain()
    srv.close()
    torch.cuda.synchronize()
    budget = int(args.serve_budget_gb * (1 << 30))
    with ClockSampler(0) as clocks:
        ours = serve_trace(pf, trace, 0, budget)
    one_lane = serve_trace(pf, trace, 1, budget)
    base = serial_trace(pf, trace)
    n_obs = sum(len(ss.obs_s) for ss in trace)
    span = trace_span(trace)
    capacity = ours["particle_steps_per_s"]   # the server saturated: the GPU's rate on this mix
    line = {
        "metric": METRIC, "mode": "serving", "value": ours["particle_steps_per_s"], "unit": UNIT,
        "n_gpus": 1, "higher_is_better": True, "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"serving: {len(trace)} sessions, Poisson {200.0:g}/s, "
                               f"N = 2^U{{12..18}}, linear2/robertson/brusselator 1/3 each, "
                               + (f"{args.serve_obs} observations per session"
                                  if args.serve_obs else "the problem's T observations per session")
                               + f" at Exp(5 ms) gaps, {args.serve_budget_gb:g} GB budget",
                   "sessions": len(trace), "observations": n_obs,
                   "particles": sum(ss.w.N for ss in trace),
                   "brusselator_sessions": sum(ss.w.ode == W.BRUSSELATOR for ss in trace),
                   "offered_load": trace_steps(trace) / span / capacity},
        "clocks": clocks.summary(),
        "server": {k: ours[k] for k in ("p50_ms", "p99_ms", "mean_ms", "max_ms", "epochs",
                                        "mean_sessions_per_epoch", "admitted", "rejected",
                                        "submit_lag_p99_ms", "step_calls", "step_ms_mean",
                                        "step_ms_max", "collect_ms_max", "admit_ms_max",
                                        "launch_ms_max")},
        "server_one_lane": {k: one_lane[k] for k in ("particle_steps_per_s", "p50_ms", "p99_ms",
                                                     "mean_ms", "max_ms", "epochs",
                                                     "mean_sessions_per_epoch")},
        "serial_per_filter": base,
        "throughput_vs_serial": ours["particle_steps_per_s"] / base["particle_steps_per_s"],
        "p99_vs_serial": ours["p99_ms"] / base["p99_ms"],
    }
    if args.serve_sweep:
        line["load_sweep"] = serving_sweep(args, pf, capacity, budget)
    return line


def trace_span(trace):
    """Seconds from the first session's arrival to the last observation's."""
    return max(float(ss.obs_s[-1]) for ss in trace) - min(ss.open_s for ss in trace)


def trace_steps(trace):
    return sum(ss.w.particle_steps(k) for ss in trace for k in range(len(ss.obs_s)))


def _events(trace):
    events = []
    for s, ss in enumerate(trace):
        events.append((ss.open_s, 0, s, -1))
        for k, ta in enumerate(ss.obs_s):
            events.append((float(ta), 1, s, k))
    events.sort()
    return events


def _pct(lat, q):
    lat = sorted(lat)
    return lat[min(len(lat) - 1, max(0, int(math.ceil(q * len(lat))) - 1))]


def serve_trace(pf, trace, lanes, budget):
    """Replay the trace in real time through a server (admission by budget,
    continuous batching over `lanes` lanes, 0 = one per class)."""
    events = _events(trace)
    n_obs = sum(len(ss.obs_s) for ss in trace)
    srv = pf.Server(budget_bytes=budget, lanes=lanes)
    sid = {}
    lags = []
    t_start = time.perf_counter()
    i = 0
    while i < len(events):
        now = time.perf_counter() - t_start
        while i < len(events) and events[i][0] <= now:
            te, kind, s, k = events[i]
            ss = trace[s]
            if kind == 0:
                sid[s] = srv.pf_server_open(ss.w, filter_id=s)
            else:
                srv.pf_server_submit(sid[s], ss.w.t_obs[k], ss.w.y_obs[k])
                lags.append(time.perf_counter() - t_start - te)
                if k == len(ss.obs_s) - 1:
                    srv.pf_server_close(sid[s])
            i += 1
        srv.pf_server_step()
    srv.pf_server_drain()
    st = srv.pf_server_stats()
    srv.close()
    assert st["assimilations"] == n_obs, st
    st["submit_lag_p99_ms"] = 1e3 * _pct(lags, 0.99)
    return st


def serial_trace(pf, trace):
    """Replay the trace in real time with serial per-filter calls: each
    observation assimilated by pf_assimilate in arrival order, the filter
    created when its session opens."""
    def wait_until(t_start, te):
        while True:
            dt = te - (time.perf_counter() - t_start)
            if dt <= 0:
                return
            if dt > 2e-3:
                time.sleep(dt - 1e-3)

    fil = {}
    lat = []
    t_start = time.perf_counter()
    first = last = None
    for te, kind, s, k in _events(trace):
        wait_until(t_start, te)
        ss = trace[s]
        if kind == 0:
            fil[s] = pf.Filter.from_workload(ss.w, filter_id=s)
            continue
        fil[s].pf_assimilate(ss.w.t_obs[k], ss.w.y_obs[k])
        done = time.perf_counter() - t_start
        lat.append(1e3 * (done - te))
        first = te if first is None else first
        last = done
        if k == len(ss.obs_s) - 1:
            fil[s].close()
    return {"particle_steps_per_s": trace_steps(trace) / (last - first), "p50_ms": _pct(lat, 0.5),
            "p99_ms": _pct(lat, 0.99), "mean_ms": sum(lat) / len(lat), "max_ms": max(lat)}


def epoch_seconds(pf, w):
    """Wall time of one synchronous epoch of workload w alone (its second
    epoch, after a warm one)."""
    f = pf.Filter.from_workload(w)
    f.pf_assimilate(w.t_obs[0], w.y_obs[0])
    t0 = time.perf_counter()
    f.pf_assimilate(w.t_obs[1], w.y_obs[1])
    dt = time.perf_counter() - t0
    f.close()
    return dt


def serving_sweep(args, pf, capacity, budget):
    """The same kind of trace at loads below the GPU's capacity, so that the
    latency measures assimilation rather than queueing: a smaller trace
    (args.sweep_sessions sessions of args.sweep_obs observations) with every
    arrival time dilated by D, i.e. sessions at 200/D per second and
    observation gaps of mean 5 D ms.  A session's observations are
    assimilated one after another, so D is set per target load rho from the
    slowest session: its epoch time alone (measured here) over its mean gap
    is rho.  offered_load is the whole trace's work over its span against
    the capacity the saturated server measured on the full trace."""
    from paper_1411_1702_gb300 import workloads as W
    base = W.serving(n_sessions=args.sweep_sessions, obs_per_session=args.sweep_obs, seed=1)
    span0, work = trace_span(base), trace_steps(base)
    slowest = {}
    for ss in base:
        key = (ss.w.ode, ss.w.N)
        if key not in slowest:
            slowest[key] = epoch_seconds(pf, ss.w)
    t_epoch = max(slowest.values())
    out = []
    for rho in args.sweep_loads:
        D = max(1.0, t_epoch / (5e-3 * rho))
        trace = W.serving(n_sessions=args.sweep_sessions, obs_per_session=args.sweep_obs, seed=1,
                          rate_hz=200.0 / D, mean_gap_ms=5.0 * D)
        ours = serve_trace(pf, trace, 0, budget)
        ser = serial_trace(pf, trace)
        out.append({"session_load": rho, "slowest_epoch_ms": 1e3 * t_epoch,
                    "offered_load": work / (capacity * trace_span(trace)),
                    "session_rate_per_s": 200.0 / D, "mean_obs_gap_ms": 5.0 * D,
                    "sessions": len(trace), "observations": sum(len(ss.obs_s) for ss in trace),
                    "server": {k: ours[k] for k in ("particle_steps_per_s", "p50_ms", "p99_ms",
                                                    "mean_ms", "max_ms", "epochs",
                                                    "mean_sessions_per_epoch")},
                    "serial_per_filter": ser,
                    "p50_vs_serial": ours["p50_ms"] / ser["p50_ms"],
                    "p99_vs_serial": ours["p99_ms"] / ser["p99_ms"]})
    return out


def run_sharded(args):
    """One filter of the workload's N particles split into shards
    (paper_1411_1702_gb300/shard.py): one shard per rank under torchrun,
    exchanging over NCCL, or --shards G shards driven by threads on one GPU.
    A step is one epoch of the whole filter; value = its particle-LMM-steps
    over the slowest rank's time."""
    import torch
    from paper_1411_1702_gb300 import workloads as W
    from paper_1411_1702_gb300 import shard as SH
    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1411_1702_gb300 import build as B
    B.build()
    from paper_1411_1702_gb300 import pf
    w = W.get(args.workload)
    G = world if dist is not None else max(1, args.shards)
    tile = pf.pf_shard_tile(w.N)
    bounds = SH.shard_bounds(w.N, G, tile)
    mine = [rank] if dist is not None else list(range(G))
    engines = {q: SH.LibraryShard(pf, w, w.N, bounds[q], bounds[q + 1] - bounds[q]) for q in mine}
    torch.cuda.synchronize()
    if dist is not None:
        comms = {rank: SH.TorchComm(device=torch.device("cuda", local))}
    else:
        hub = SH.ThreadComm(G, timeout=600.0)
        comms = {q: hub.view(q) for q in mine}
    filters = {}

    def each(fn):
        """fn(q) for every shard of this process, side by side."""
        if len(mine) == 1:
            fn(mine[0])
            return
        errs = []

        def body(q):
            try:
                fn(q)
            except BaseException as ex:   # noqa: BLE001 - re-raised below
                errs.append(ex)
                hub.abort()
        th = [threading.Thread(target=body, args=(q,)) for q in mine]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]

    each(lambda q: filters.__setitem__(q, SH.ShardedFilter(engines[q], comms[q], bounds, tile)))
    k = 0

    def step():
        nonlocal k
        kk = k
        each(lambda q: filters[q].assimilate(w.t_obs[kk], w.y_obs[kk]))
        k += 1
        return kk

    for _ in range(args.warmup):
        step()
    K = min(args.steps, w.T - args.warmup)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    steps_done = 0
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for _ in range(K):
            steps_done += w.particle_steps(step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    total_ms, _ = reduce_times(dist, wall * 1e3, 0, device="cuda")
    for e in engines.values():
        e.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "mode": "sharded", "value": steps_done / (total_ms * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": total_ms / K,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(config_of(w), parallelism=(f"{G} shards over {world} ranks (NCCL)" if dist
                                                  else f"{G} shards on one GPU (threads)"),
                       shards=G, shard_tile=tile, bounds=bounds[:3] + ["..."] if G > 3 else bounds),
        "clocks": clocks.summary(),
        "timing": "wall time of whole epochs, all exchanges included",
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="robertson",
                    choices=["robertson", "robertson22", "linear2", "brusselator", "advdiff20",
                             "advdiff40", "michaelis"] + ["michaelis" + n for n in W_LMM_NAMES] + [
                             "batched", "serving"])
    ap.add_argument("--batch-filters", type=int, default=256)
    ap.add_argument("--batch-log2n", type=float, nargs=2, default=[10.0, 17.0],
                    help="the batched filters' N = round(2^U[lo, hi])")
    ap.add_argument("--serve-sessions", type=int, default=64)
    ap.add_argument("--serve-obs", type=int, default=0,
                    help="observations per session (0: the problem's T)")
    ap.add_argument("--serve-sweep", type=int, default=1,
                    help="also serve a smaller trace at loads below capacity")
    ap.add_argument("--sweep-sessions", type=int, default=16)
    ap.add_argument("--sweep-obs", type=int, default=10)
    ap.add_argument("--sweep-loads", type=float, nargs="+", default=[0.5, 0.25])
    ap.add_argument("--patterns", type=int, default=1,
                    help="default run: add the batched and serving objects (one GPU)")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--e2e-steps", type=int, default=80)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-particles", type=int, default=0,
                    help="particles of the reference arm's oracle (0: the workload's N)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sharded", action="store_true",
                    help="one filter split into shards: one per rank, or --shards on one GPU")
    ap.add_argument("--shards", type=int, default=1)
    ap.add_argument("--profile", action="store_true",
                    help="only launch the epochs (for ncu); prints no measurement")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    from paper_1411_1702_gb300 import workloads as W
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.sharded and args.impl != "reference":
        return run_sharded(args)
    w = W.get(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
