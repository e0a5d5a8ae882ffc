"""Benchmark: time-to-RMSE 1e-3 of the MLMC estimate of E[AB] on one GB300.

Workload ("mlmc_256x65536x256"): A 256 x 65536, B 65536 x 256, A = M + S o Z, B = M' + S' o Z'
with M ~ U[-1,1], S ~ U[0.1,1] (A from seed 0, B from seed 1), c_l = 64 * 2^l for l = 0..8,
N_l from the variance-optimal allocation (Remark 3.6) of 256 pilot samples per level for an
absolute Frobenius tolerance eps = 1e-3 * ||E[AB]||_F = 1e-3 * ||M M'||_F.

A full run at that tolerance evaluates about 5e13 sampled outer products (hours on one GPU),
so the benchmark measures the exact work mix instead: after the pilot and the allocation
(untimed setup), every step evaluates B_l = ceil(f * N_l) fresh samples of every level l
(f fixed, sample ids continue across steps) through ``mlmc_level_stats``, the per-level
statistics included, followed by the telescoping sum.  Samples are independent and the
estimator has no bias for f = identity, so the time of the full run is
    T(1e-3) = sum_l N_l * t_l / B_l
with t_l the measured device time of level l's batches (CUDA events on the plan's stream).
``value`` is that projected time in seconds (lower is better).

Measured end to end as well (default legs): the headline workload at rel. RMSE 3e-2 through
mlmc_estimate (``ladder``: extrapolated to 1e-3 by eps^-2 and set beside the projection), and
the 64 x 1024 x 64 workload at 1e-3 (BF16) and 3e-3 (BF16, FP32, E4M3) (``ttr_64x1024x64``).

e2e: the same metric through the C ABI from pinned host buffers: each e2e step copies the
four parameter matrices host->device, builds a plan (layout copy), runs the step's batches
and reads the estimate back; T_e2e = (e2e step time - its sampling time) + sum_l N_l t_l / B_l.

--impl reference: the FP64 CPU oracle (test infrastructure) timed on the host cores on one
sample per level per step, projected the same way.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="mlmc_256x65536x256", m=256, n=65536, p=256, c0=64, R=2, L=8, pilot=256, rel_rmse=1e-3)
FRACTION = {"fp32": 2.0**-20, "fp64": 2.0**-26, "bf16": 2.0**-18, "fp8": 2.0**-18}
# ALU peaks (TFLOP/s), replaced at run time by mlmc_measure_peaks (FP32 / FP64 fused multiply-add
# chains at full occupancy on this GPU); the unit-count figure below is the fallback only
ALU_PEAKS = {"fp32": 152 * 128 * 2 * 2.070e9 / 1e12, "fp64": None,
             "source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived; not measured in this run)"}


def measure_alu_peaks(stream):
    """Measure the FP32 / FP64 peaks on this GPU (mlmc_measure_peaks) and keep them for the
    rooflines of the CUDA-core kernels; returns the full measurement."""
    from paper_1904_00429_gb300 import binding
    pk = binding.measure_peaks(stream)
    ALU_PEAKS.update({"fp32": pk["fp32_flops"] / 1e12, "fp64": pk["fp64_flops"] / 1e12,
                      "source": "mlmc_measure_peaks in this run (FMA chains at full occupancy)"})
    return pk
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel from one ncu capture
# (profiles/); None once the kernel changed after the capture
TRAFFIC = {
    # DRAM bytes per sampled outer product of the 128 x 64 tile kernel (level-0 capture of 262144
    # outer products), used for every level
    "fp32": {"dram_bytes_per_outer_product": {0: (745842432 + 13862912) / 262144, 8: (745842432 + 13862912) / 262144},
             "source": "profiles/level_cuda_core_f32_mlmc_256x65536x256.md"},
    # DRAM bytes (read + write) per sampled outer product of the CTA-pair kernel (tile 3256) at
    # levels 0 and 8, each from one ncu pass over one launch of the bench's profile case
    # (16384 level-0 samples, 2432 level-8 samples of this workload); levels between are
    # interpolated, and bench.py scales them by the outer products of its own launches
    "bf16": {"dram_bytes_per_outer_product": {0: (2901958400 + 62803200) / 1048576,
                                              8: (108988471808 + 78316800) / 39845888},
             # levels with c_l >= 4096 run on the single-CTA 256 x 256 tile: its level-8 capture
             "wide": {"from_c": 4096, "dram_bytes_per_outer_product": (109698142208 + 624583168) / 39845888},
             "source": "profiles/level_tc_bf16_mlmc_256x65536x256.md"},
    "fp8": {"dram_bytes_per_outer_product": {0: (2902601984 + 62838272) / 1048576,
                                             8: (109010083328 + 77853952) / 39845888},
            "source": "profiles/level_tc_bf16_mlmc_256x65536x256.md"},
}


def dram_per_outer(prec, level, c=None):
    w = TRAFFIC[prec].get("wide")
    if w is not None and c is not None and c >= w["from_c"]:
        return w["dram_bytes_per_outer_product"]   # levels on the single-CTA 256 x 256 tile
    t = TRAFFIC[prec]["dram_bytes_per_outer_product"]
    if level in t:
        return t[level]
    f = min(max(level / 8.0, 0.0), 1.0)   # levels without a measurement: linear between 0 and 8
    return t[0] + (t[8] - t[0]) * f


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def batch_sizes(Nl, frac):
    return [max(8, int(math.ceil(frac * n))) for n in Nl]


def run_reference(args):
    """The oracle (test infrastructure) on all host cores: one round (every worker process one
    sample of every level) per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1904_00429_gb300.inputs import make_params
    W = WORKLOAD
    pp = make_params(W["m"], W["n"], W["p"], seed_A=0, seed_B=1, dtype=np.float32)
    levels = list(range(W["L"] + 1))
    # allocation from the closed-form level variances of this law would need no sampling, but the
    # reference arm reuses the device arm's quantity: N_l for eps from per-level variances of the
    # oracle's own pilot is out of reach on a CPU, so N_l comes from the closed form of V_l.
    Nl = closed_form_allocation(pp, W)
    del pp
    pool = OraclePool(W)
    per_level = {l: [] for l in levels}
    step_times = []
    for it in range(args.warmup + args.steps):
        t_l, wall = pool.round((1 << 43) + it * (W["L"] + 1) * pool.cores)
        if it >= args.warmup:
            for l in levels:
                per_level[l].append(t_l[l])
            step_times.append(wall)
    pool.close()
    t_l = [statistics.mean(per_level[l]) for l in levels]
    T = sum(n * t for n, t in zip(Nl, t_l))
    line = {"impl": "reference", "metric": "time-to-RMSE 1e-3 for E[AB] (projected from the measured per-level "
            "sample rate)", "value": T, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(step_times), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "m": W["m"], "n": W["n"], "p": W["p"], "c0": W["c0"], "L": W["L"],
                       "N_l": Nl, "sample": f"one oracle sample per level per worker process per step "
                                            f"({pool.cores} processes)"},
            "cpu_baseline": {"value": T, "unit": "s", "cores": pool.cores, "kind": "oracle",
                             "sample": f"one FP64 oracle sample per level 0..8 per step on each of {pool.cores} "
                                       "worker processes"},
            "e2e": {"value": T, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def closed_form_allocation(pp, W):
    """N_l for eps from the closed-form single-sample variances of the Gaussian law (used only
    to size the CPU reference arm; the device arm allocates from its own pilot)."""
    M, S, Mp, Sp = pp.f64()
    n = W["n"]
    Q = (M**2 + S**2) @ (Mp**2 + Sp**2)
    Rr = (M**2) @ (Mp**2)
    mu = M @ Mp
    K = float((n * Q - Q + Rr - mu**2).sum())
    c = [W["c0"] * W["R"]**l for l in range(W["L"] + 1)]
    V = [float((((n * Q - Q + Rr - mu**2) / c[0]) + Q - Rr).sum())] + \
        [(1.0 / c[l - 1] - 1.0 / c[l]) * K for l in range(1, W["L"] + 1)]
    C = [c[0]] + [c[l] + c[l - 1] for l in range(1, W["L"] + 1)]
    eps = W["rel_rmse"] * float(np.linalg.norm(mu))
    root = sum(math.sqrt(v * cc) for v, cc in zip(V, C))
    return [max(W["pilot"], int(math.ceil(2.0 / eps**2 * math.sqrt(v / cc) * root))) for v, cc in zip(V, C)]


def cpu_baseline_sample(W, budget_s=20.0):
    """The oracle timed on a bounded sample (one sample per level, levels 0..8) on one host core."""
    import oracle
    from paper_1904_00429_gb300.inputs import make_params
    pp = make_params(W["m"], W["n"], W["p"], seed_A=0, seed_B=1, dtype=np.float32)
    orc = oracle.Problem(*pp.f64())
    lv = oracle.Levels(W["c0"], W["R"], W["L"])
    t_l = []
    start = time.perf_counter()
    for l in range(W["L"] + 1):
        t0 = time.perf_counter()
        oracle.sample(orc, lv, l, 1 << 40)
        t_l.append(time.perf_counter() - t0)
        if time.perf_counter() - start > budget_s:
            # extrapolate the remaining levels by the per-slot cost of the last one
            per_slot = t_l[-1] / lv.cl(l)
            t_l += [per_slot * lv.cl(k) for k in range(l + 1, W["L"] + 1)]
            break
    return t_l, pp


_ORACLE = {}


def _oracle_pool_init(W):
    """Worker set-up of the all-cores oracle timing: the workload's parameters, once per process."""
    import oracle
    from paper_1904_00429_gb300.inputs import make_params
    pp = make_params(W["m"], W["n"], W["p"], seed_A=0, seed_B=1, dtype=np.float32)
    _ORACLE["orc"] = oracle.Problem(*pp.f64())
    _ORACLE["lv"] = oracle.Levels(W["c0"], W["R"], W["L"])


def _oracle_pool_task(task):
    import oracle
    level, sample = task
    if level < 0:   # start-up probe: the worker is initialised
        time.sleep(0.5)
        return level, 0.0
    t0 = time.perf_counter()
    oracle.sample(_ORACLE["orc"], _ORACLE["lv"], level, sample)
    return level, time.perf_counter() - t0


class OraclePool:
    """The FP64 oracle on every host core: `cores` spawned worker processes (spawned, so no CUDA
    state is inherited), each computing whole samples; a round gives every worker one sample of
    every level, longest levels first, and the throughput of a level is its mean sample time
    divided by the parallelism the round achieved (busy time / wall time)."""

    def __init__(self, W):
        import multiprocessing as mp
        self.W = W
        self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_pool_init, initargs=(W,))
        self.pool.map(_oracle_pool_task, [(-1, 0)] * self.cores, chunksize=1)

    def round(self, sample_base):
        levels = range(self.W["L"], -1, -1)
        tasks = [(l, sample_base + l * self.cores + i) for l in levels for i in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_pool_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
        busy = sum(d for _, d in res)
        per_level = [statistics.mean([d for lv, d in res if lv == l]) for l in range(self.W["L"] + 1)]
        # seconds per sample of each level at the throughput of all cores
        return [t * wall / busy for t in per_level], wall

    def close(self):
        self.pool.close()
        self.pool.join()


def _measure(args, prec, W, host, dev, rank, stream, world, with_e2e):
    """Pilot + allocation (untimed), then warm-up and exactly ``args.steps`` timed steps of the
    allocation's work mix for one precision.  Returns a dict of measurements."""
    import torch

    from paper_1904_00429_gb300 import binding

    def make_plan(tensors):
        spec = binding.ProblemSpec(*tensors, seed_A=0, seed_B=1, seed_idx=2, problem_id=rank)
        return binding.Plan([spec], c0=W["c0"], L=W["L"], ratio=W["R"], precision=prec, pilot_n=W["pilot"],
                            tile_override=args.tile if prec in ("bf16", "fp8") else
                            args.fp32_tile if prec == "fp32" else 0, stream=stream)

    pdtype = torch.float64 if prec == "fp64" else torch.float32
    dev_params = [h.to(dev, pdtype, non_blocking=True) for h in host]
    torch.cuda.synchronize()
    plan = make_plan(dev_params)
    levels = list(range(W["L"] + 1))
    for l in levels:
        plan.level_stats(0, l, 0, W["pilot"])
    Nl = plan.allocate([W["eps"]])[0]
    B = batch_sizes(Nl, FRACTION[prec])
    next_id = [W["pilot"]] * len(levels)

    def step(p, timing):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(levels) + 1)]
        ev[0].record(stream)
        for i, l in enumerate(levels):
            p.level_stats(0, l, next_id[l], B[l])
            next_id[l] += B[l]
            ev[i + 1].record(stream)
        p.telescoping_sum()
        timing.append(ev)

    for _ in range(args.warmup):
        step(plan, [])
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = plan.launch_count()
    timings = []
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        torch.cuda.synchronize()
        t_start.record(stream)
        for _ in range(args.steps):
            step(plan, timings)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    plan.synchronize()   # surfaces any device-side error of the timed launches
    launches = plan.launch_count() - launches0
    total_ms = t_start.elapsed_time(t_end)
    lvl_ms = [sum(ev[i].elapsed_time(ev[i + 1]) for ev in timings) for i in range(len(levels))]
    t_l = [ms / 1e3 / (args.steps * B[l]) for l, ms in zip(levels, lvl_ms)]   # seconds per sample
    T_proj = sum(n * t for n, t in zip(Nl, t_l))
    outer = sum(args.steps * B[l] * plan.cl(l) for l in levels)
    res = {"prec": prec, "Nl": Nl, "B": B, "t_l": t_l, "T": T_proj, "total_ms": total_ms,
           "sample_s": sum(lvl_ms) / 1e3, "outer": outer, "launches": launches, "clocks": clocks.summary(),
           "steps": args.steps}
    plan.close()
    del dev_params

    if with_e2e:
        # end to end through the C ABI with host buffers: mlmc_plan_host copies the four pinned
        # parameter matrices to the device inside the call, the step's batches run, and
        # mlmc_telescoping_sum_host writes the estimate back to host memory (synchronising);
        # timed on the host around the whole step
        e2e_s, e2e_sample_ms = [], []
        m, p = W["m"], W["p"]
        out_host = torch.empty(m * p, dtype=torch.float64).pin_memory()
        host_p = [h if h.dtype == pdtype else h.to(pdtype).pin_memory() for h in host]
        for it in range(args.warmup + max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            spec = binding.ProblemSpec(*host_p, seed_A=0, seed_B=1, seed_idx=2, problem_id=rank)
            p2 = binding.Plan([spec], c0=W["c0"], L=W["L"], ratio=W["R"], precision=prec, pilot_n=W["pilot"],
                              tile_override=args.tile if prec in ("bf16", "fp8") else 0, stream=stream, host=True)
            tm = []
            step(p2, tm)
            p2.telescoping_sum_host(out_host)
            t1 = time.perf_counter()
            p2.close()
            if it >= args.warmup:
                e2e_s.append(t1 - t0)
                e2e_sample_ms.append(sum(tm[0][i].elapsed_time(tm[0][i + 1]) for i in range(len(levels))))
        res["e2e_overhead_s"] = statistics.mean(e2e_s) - statistics.mean(e2e_sample_ms) / 1e3
        res["h2d"] = sum(h.numel() * h.element_size() for h in host_p)
        res["d2h"] = m * p * 8
        res["e2e_api"] = "mlmc_plan_host + mlmc_level_stats + mlmc_telescoping_sum_host (host buffers)"
    return res


def _roofline(res, W, peaks, peak_kind, gen_rate=None):
    m, p = W["m"], W["p"]
    prec = res["prec"]
    flops = 2.0 * m * p * res["outer"]
    elem = 8 if prec == "fp64" else 4
    bytes_alg = 2.0 * (m + p) * elem * res["outer"]
    t = res["sample_s"]
    traffic = TRAFFIC.get(prec)
    if traffic is not None:
        # estimated DRAM bytes per level-kernel launch, averaged over the timed launches
        # (each level_stats call is one level-kernel launch and two merges; one telescoping sum per step)
        level_launches = max(1, (res["launches"] - res["steps"]) // 3)
        dram = sum(res["steps"] * b * (W["c0"] * W["R"]**l) * dram_per_outer(prec, l, W["c0"] * W["R"]**l)
                   for l, b in enumerate(res["B"]))
        traffic = {"value": dram / level_launches, "unit": "bytes per launch", "launches": level_launches,
                   "algorithmic_bytes_per_launch": bytes_alg / level_launches, "source": TRAFFIC[prec]["source"]}
    if prec in ("fp32", "fp64"):
        peak = ALU_PEAKS[prec]
        achieved = flops / t / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": traffic, "peak_source": ALU_PEAKS["source"],
                "hbm_achieved_gbs": bytes_alg / t / 1e9, "hbm_peak_gbs": peaks["hbm_gbs"],
                "kernel": f"level_cuda_core_kernel<{prec}>"}
    # tensor-core path: the slower of gathered bytes at HBM bandwidth and FLOPs at the tensor peak
    hbm = bytes_alg / t / 1e9
    tflops = flops / t / 1e12
    # the E4M3 form runs its dequantised operands through the same bf16 MMA
    tpeak = peaks["bf16_tflops_sustained"]
    t_hbm = bytes_alg / (peaks["hbm_gbs"] * 1e9)
    t_tc = flops / (tpeak * 1e12)
    # third bound: every sampled outer product needs m + p freshly generated entries
    gen = None
    t_gen = 0.0
    if gen_rate:
        entries = float(m + p) * res["outer"]
        t_gen = entries / gen_rate
        gen = {"bound": "alu", "achieved": entries / t, "peak": gen_rate, "unit": "entries/s",
               "frac": entries / t / gen_rate,
               "peak_source": "mlmc_measure_generation_rate in this run (Philox4x32-10 + special-function "
                              "Box-Muller + M + S z + bf16, full occupancy)"}
    if t_gen > max(t_hbm, t_tc):
        return {"bound": "alu", "achieved": gen["achieved"], "peak": gen_rate, "unit": "entries/s",
                "frac": gen["frac"], "traffic": traffic, "peak_source": gen["peak_source"],
                "hbm_achieved_gbs": hbm, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_frac": hbm / peaks["hbm_gbs"],
                "tensor_achieved_tflops": tflops, "tensor_peak_tflops": tpeak, "tensor_frac": tflops / tpeak,
                "kernel": f"level_tc_{prec}_kernel"}
    if t_hbm >= t_tc:
        out = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": hbm / peaks["hbm_gbs"], "traffic": traffic,
               "peak_source": f"hbm_gbs ({peak_kind})", "tensor_achieved_tflops": tflops,
               "tensor_peak_tflops": tpeak, "tensor_frac": tflops / tpeak,
               "kernel": f"level_tc_{prec}_kernel"}
    else:
        out = {"bound": "tensor", "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s", "frac": tflops / tpeak,
               "traffic": traffic, "peak_source": f"bf16_tflops_sustained ({peak_kind})",
               "hbm_achieved_gbs": hbm, "kernel": f"level_tc_{prec}_kernel"}
    if gen is not None:
        out["generation"] = gen
    return out


ADJOINT = dict(name="adjoint_256x65536x256", m=256, n=65536, p=256, c0=64, R=2, L=8, N=256, precision="bf16")


def _measure_adjoint(args, host, dev, stream, peaks, peak_kind, gen_rate=None):
    """Backward of the loss ||Yhat - T||_F^2 through mlmc_backward: A 256 x 65536, B 65536 x 256,
    c_l = 64 * 2^l for l = 0..8, N_l = 256 samples per level, BF16 forward (straight-through
    adjoint).  Times exactly ``args.steps`` backward calls after ``args.warmup`` untimed ones."""
    import torch

    from paper_1904_00429_gb300 import binding
    from paper_1904_00429_gb300.inputs import make_target

    A = ADJOINT
    tensors = [h.to(dev, torch.float32, non_blocking=True) for h in host]
    spec = binding.ProblemSpec(*tensors, seed_A=0, seed_B=1, seed_idx=2, problem_id=0)
    plan = binding.Plan([spec], c0=A["c0"], L=A["L"], ratio=A["R"], precision=A["precision"], stream=stream)
    for l in range(A["L"] + 1):
        plan.level_stats(0, l, 0, A["N"])
    (Y,) = plan.telescoping_sum()
    T = torch.from_numpy(make_target(A["m"], A["p"])).to(dev)
    G = (2.0 * (Y - T)).contiguous()
    grads = [tuple(torch.empty_like(t) for t in tensors)]
    for _ in range(args.warmup):
        plan.backward([G], grads)
    torch.cuda.synchronize()
    launches0 = plan.launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        plan.backward([G], grads)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    plan.synchronize()
    launches = plan.launch_count() - launches0
    ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    records = A["N"] * sum(A["c0"] * A["R"]**l for l in range(A["L"] + 1))
    # two contractions (G b and G^T a) of m x p FMAs per sampled product
    flops = 2.0 * 2.0 * A["m"] * A["p"] * records
    # normals the replay needs at least: per record and side, the contracted vector and the
    # output-side normals (m + p), twice
    normals = 2.0 * (A["m"] + A["p"]) * records
    t = statistics.mean(ms) / 1e3
    plan.close()
    achieved = flops / t / 1e12
    peak, src = peaks["bf16_tflops_sustained"], f"bf16_tflops_sustained ({peak_kind})"
    return {"workload": A["name"], "metric": "backward time (mlmc_backward, all four gradients)",
            "value": t, "unit": "s", "ms_per_backward": [round(x, 4) for x in ms], "records": records,
            "N_l": [A["N"]] * (A["L"] + 1), "precision": A["precision"], "gpu_launches": launches,
            "normals_per_s": normals / t,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "flops": "useful: 4 m p per record (the hi/lo split of G issues twice that)",
                         "kernel": "segment_tc_kernel",
                         # the bound that binds: regenerating the replayed vectors, 2 (m + p) normals
                         # per record against the measured generation rate (the same arithmetic)
                         "generation": None if not gen_rate else
                         {"bound": "alu", "achieved": normals / t, "peak": gen_rate, "unit": "entries/s",
                          "frac": normals / t / gen_rate,
                          "peak_source": "mlmc_measure_generation_rate in this run"}}}


def _measure_ladder(args, rels, W, host, exact, dev, stream, projected):
    """Alg. 2 end to end through mlmc_estimate at looser targets: for each relative RMSE a fresh
    plan runs the pilot, the allocation and the top-up (timed on the host around the call, which
    returns after the estimate is on the device).  The estimator has no bias, so its cost scales
    as eps^-2 up to the fixed pilot; the time at 1e-3 is extrapolated by (rel / 1e-3)^2 and set
    beside the projection of the headline."""
    import torch

    from paper_1904_00429_gb300 import binding

    tensors = [h.to(dev, torch.float32, non_blocking=True) for h in host]
    norm = float(np.linalg.norm(exact))
    rungs = []
    for rel in rels:
        eps = rel * norm
        spec = binding.ProblemSpec(*tensors, seed_A=10, seed_B=11, seed_idx=12, problem_id=0)
        with binding.Plan([spec], c0=W["c0"], L=W["L"], ratio=W["R"], precision=args.precision,
                          pilot_n=W["pilot"], stream=stream) as plan:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (Y,), (rep,) = plan.estimate([eps])
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            err = float(np.linalg.norm(Y.cpu().numpy() - exact))
        rungs.append({"rel_rmse": rel, "eps_abs": eps, "seconds": t, "N_l": rep["N"],
                      "outer_products": rep["outer_products"], "rmse_pred": rep["rmse_pred"],
                      "error": err, "error_over_eps": err / eps,
                      "extrapolated_1e-3_s": t * (rel / 1e-3) ** 2})
    return {"metric": "time-to-RMSE measured at looser targets through mlmc_estimate",
            "unit": "s", "rungs": rungs, "projected_1e-3_s": projected}


TTR = dict(name="mlmc_64x1024x64", m=64, n=1024, p=64, c0=16, R=2, L=5, pilot=256)


def _measure_ttr(args, rels, precs, dev, stream):
    """Time-to-RMSE measured end to end on the 64 x 1024 x 64 workload (M ~ U[-1,1], S ~ U[0.1,1],
    A from seed 0, B from seed 1, c_l = 16 * 2^l for l = 0..5): for every precision and relative
    target a fresh plan runs Alg. 2 through mlmc_estimate (pilot of 256 samples per level, the
    allocation of Remark 3.6 for eps = rel * ||M M'||_F, the top-up), timed on the host around the
    call (which returns with the estimate on the device).  The achieved error ||Yhat - M M'||_F is
    set against eps: the allocation aims at eps / sqrt(2)."""
    import torch

    from paper_1904_00429_gb300 import binding
    from paper_1904_00429_gb300.inputs import make_params

    T = TTR
    pp = make_params(T["m"], T["n"], T["p"], seed_A=0, seed_B=1, dtype=np.float32)
    exact = pp.exact_mean()
    norm = float(np.linalg.norm(exact))
    out = {"workload": T["name"], "metric": "time-to-RMSE measured end to end through mlmc_estimate",
           "unit": "s", "m": T["m"], "n": T["n"], "p": T["p"], "c0": T["c0"], "ratio": T["R"], "L": T["L"],
           "pilot": T["pilot"], "runs": []}
    for prec in precs:
        pdt = torch.float64 if prec == "fp64" else torch.float32
        ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev, pdt) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
        for rel in rels:
            eps = rel * norm
            spec = binding.ProblemSpec(*ts, seed_A=0, seed_B=1, seed_idx=2, problem_id=0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with binding.Plan([spec], c0=T["c0"], L=T["L"], ratio=T["R"], precision=prec, pilot_n=T["pilot"],
                              stream=stream) as plan:
                launches0 = plan.launch_count()
                (Y,), (rep,) = plan.estimate([eps])
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                launches = plan.launch_count() - launches0
            err = float(np.linalg.norm(Y.cpu().numpy() - exact))
            out["runs"].append({"precision": prec, "rel_rmse": rel, "eps_abs": eps, "seconds": t,
                                "error": err, "error_over_eps": err / eps, "rmse_pred": rep["rmse_pred"],
                                "N_l": rep["N"], "V_l": rep["V"], "outer_products": rep["outer_products"],
                                "outer_products_per_s": rep["outer_products"] / t, "gpu_launches": launches})
        del ts
    by = {(r["precision"], r["rel_rmse"]): r["seconds"] for r in out["runs"]}
    out["fp32_over"] = {f"{p}@{rel:g}": by[("fp32", rel)] / by[(p, rel)]
                        for p in precs for rel in rels if p != "fp32" and ("fp32", rel) in by}
    return out


def _measure_dedupe_bound(args, head, W, dev, stream):
    """Index dedupe (merging the repeated draws of one sample, the note after Alg. 1) would save
    at most the repeated slots' share of each level's work.  Measured on the draws themselves:
    the fraction of a sample's c_l slots whose index already appeared earlier in the sample,
    over 16 samples per level drawn by the library (mlmc_debug_indices), for the headline
    workload and the 64 x 1024 x 64 workload; weighted by each level's measured share of the
    headline's time (N_l t_l), and by the cost split C_l of the 64 x 1024 x 64 allocation."""
    import torch

    from paper_1904_00429_gb300 import binding
    from paper_1904_00429_gb300.inputs import make_params

    out = {}
    for name, (m, n, p, c0, L) in {"mlmc_256x65536x256": (W["m"], W["n"], W["p"], W["c0"], W["L"]),
                                   "mlmc_64x1024x64": (64, 1024, 64, 16, 5)}.items():
        # the index draws depend only on n, the level and the sample: a one-row stand-in keeps the plan small
        pp = make_params(1, n, 1, seed_A=0, seed_B=1, dtype=np.float32)
        ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
        with binding.Plan([binding.ProblemSpec(*ts, seed_A=0, seed_B=1, seed_idx=2)], c0=c0, L=L,
                          precision="fp32", stream=stream) as plan:
            frac = []
            for l in range(L + 1):
                c = c0 * 2 ** l
                rep = 0
                for smp in range(16):
                    idx = plan.debug_indices(0, l, 10_000 + smp, 0, c).cpu().numpy()
                    rep += c - len(np.unique(idx))
                frac.append(rep / (16.0 * c))
        if name == W["name"] and head is not None:
            share = [nl * t for nl, t in zip(head["Nl"], head["t_l"])]
        else:
            share = [1.0] * (L + 1)   # equal cost per level (the allocation's sqrt(V_l C_l) is about level-free)
        tot = sum(share)
        bound = sum(f * sh for f, sh in zip(frac, share)) / tot
        out[name] = {"repeated_slot_fraction_per_level": frac, "expected_c2_over_2n": [min(1.0, (c0 * 2**l) / (2.0 * n))
                                                                                    for l in range(L + 1)],
                     "time_saving_upper_bound": bound,
                     "weights": "measured N_l t_l of the headline" if name == W["name"] else "equal per level"}
    return out


NONLINEAR = dict(name="abs_step_64x1024x64", m=64, n=1024, p=64, c0=16, R=2, Lmax=12, pilot=256, eps_entry=0.01,
                 precision="fp32")


def _nonlinear_params():
    """The E[f(AB)] workload's parameters: the precision workload's laws (M ~ U[-1,1], S ~ U[0.1,1],
    seeds 0 and 1) with A scaled by 2 / sqrt(n) and shifted by 2 / n, so that the entries of AB
    are O(1) and straddle the jump of f at 2."""
    from paper_1904_00429_gb300.inputs import make_params
    Nw = NONLINEAR
    pp = make_params(Nw["m"], Nw["n"], Nw["p"], seed_A=0, seed_B=1, dtype=np.float64)
    k = 2.0 / math.sqrt(Nw["n"])
    return [x.astype(np.float32) for x in (pp.M * k + 2.0 / Nw["n"], pp.S * k, pp.Mp, pp.Sp)]


def _mc_at_finest(spec, Nw, c, eps, sampling, stream, precision=None):
    """Standard MC at one level of c draws (Eq. Phigh) under the sampling law `sampling`: pilot,
    allocation for the variance target eps^2 / 2, then a bounded timed batch projected to the
    allocated N (seconds, N, seconds per sample)."""
    import torch

    from paper_1904_00429_gb300 import binding

    with binding.Plan([spec], c0=c, L=0, ratio=2, precision=precision or Nw["precision"], f="abs_step",
                      sampling=sampling,
                      pilot_n=Nw["pilot"], stream=stream) as mc:
        mc.level_stats(0, 0, 0, Nw["pilot"])
        N_mc = int(mc.allocate([eps])[0][0])
        batch = max(64, min(N_mc, int(2e8 // c)))
        mc.level_stats(0, 0, Nw["pilot"], 64)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mc.level_stats(0, 0, Nw["pilot"] + 64, batch)
        torch.cuda.synchronize()
        per_sample = (time.perf_counter() - t0) / batch
    return N_mc * per_sample, N_mc, per_sample, batch


def _measure_nonlinear(args, dev, stream):
    """E[f(AB)] with f(x) = |x| H(2 - x) (the paper's matrix example) on the CUDA cores (FP32):
    Alg. 2 with the adaptive choice of L, end to end through mlmc_estimate, against standard MC
    at the finest level MLMC chose (Eq. Phigh: one level of c_L draws, the same variance target
    eps^2 / 2) under the uniform law and under xi** (Thm 3.1, the comparator of the paper's
    Table 2), each timed on a bounded batch and projected to its allocated N; for level ratios
    R = 2, 4 and 10 (the paper's experiments use 10)."""
    import torch

    from paper_1904_00429_gb300 import binding

    Nw = NONLINEAR
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in _nonlinear_params()]
    eps = Nw["eps_entry"] * math.sqrt(Nw["m"] * Nw["p"])
    spec = binding.ProblemSpec(*ts, seed_A=7, seed_B=8, seed_idx=9, problem_id=0)
    sweep = []
    for R in (2, 4, 10):
        Lmax = Nw["Lmax"]
        while Nw["c0"] * R ** Lmax > (1 << 26):
            Lmax -= 1
        with binding.Plan([spec], c0=Nw["c0"], L=Lmax, ratio=R, precision=Nw["precision"], f="abs_step",
                          adaptive_L=True, pilot_n=Nw["pilot"], stream=stream) as plan:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            (Y,), (rep,) = plan.estimate([eps])
            torch.cuda.synchronize()
            t_mlmc = time.perf_counter() - t0
        if R == 2:
            Y_r2 = Y.cpu().numpy()
        L = rep["L"]
        cL = Nw["c0"] * R ** L
        t_u, N_u, _, batch_u = _mc_at_finest(spec, Nw, cL, eps, "uniform", stream)
        t_x, N_x, _, batch_x = _mc_at_finest(spec, Nw, cL, eps, "optimal", stream)
        sweep.append({"ratio": R, "L_max": Lmax,
                      "mlmc": {"value": t_mlmc, "L": L, "bias_unmet": rep["bias_unmet"], "N_l": rep["N"],
                               "outer_products": rep["outer_products"], "rmse_pred": rep["rmse_pred"],
                               "level_mean_norms": rep["mean_norm"], "timing": "end to end through mlmc_estimate"},
                      "mc_uniform": {"value": t_u, "c": cL, "N": N_u, "outer_products": float(N_u) * cL,
                                     "timing": f"{batch_u} samples timed, projected to N"},
                      "mc_xi_optimal": {"value": t_x, "c": cL, "N": N_x, "outer_products": float(N_x) * cL,
                                        "timing": f"{batch_x} samples timed, projected to N"},
                      "mc_uniform_over_mlmc": t_u / t_mlmc, "mc_xi_optimal_over_mlmc": t_x / t_mlmc})
    # the tensor-core form of the targeted function (BF16 operands, ratio 2 only): the same
    # problem and target, end to end, and MC at its finest level in BF16
    bf16_spec = binding.ProblemSpec(*ts, seed_A=7, seed_B=8, seed_idx=9, problem_id=0)
    with binding.Plan([bf16_spec], c0=Nw["c0"], L=Nw["Lmax"], ratio=2, precision="bf16", f="abs_step",
                      adaptive_L=True, pilot_n=Nw["pilot"], stream=stream) as plan:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (Yb,), (repb,) = plan.estimate([eps])
        torch.cuda.synchronize()
        t_bf16 = time.perf_counter() - t0
    cLb = Nw["c0"] * 2 ** repb["L"]
    t_ub, N_ub, _, batch_ub = _mc_at_finest(bf16_spec, Nw, cLb, eps, "uniform", stream, precision="bf16")
    bf16 = {"mlmc": {"value": t_bf16, "L": repb["L"], "bias_unmet": repb["bias_unmet"], "N_l": repb["N"],
                     "outer_products": repb["outer_products"], "rmse_pred": repb["rmse_pred"],
                     "timing": "end to end through mlmc_estimate"},
            "mc_uniform": {"value": t_ub, "c": cLb, "N": N_ub, "outer_products": float(N_ub) * cLb,
                           "timing": f"{batch_ub} samples timed, projected to N"},
            "mc_uniform_over_mlmc": t_ub / t_bf16,
            "fp32_mlmc_over_bf16_mlmc": sweep[0]["mlmc"]["value"] / t_bf16,
            "diff_to_fp32_estimate_over_eps": float(np.linalg.norm(Yb.cpu().numpy() - Y_r2)) / eps,
            "kernel": "level_tc_bf16_kernel<F = |x| H(2 - x)>: fine and coarse sums in two TMEM accumulators"}
    head = sweep[0]
    # FMAs of the fine contraction (2 m p per outer product; the coarse slots add their own
    # contraction on top) over the end-to-end time, host rounds included
    achieved = 2.0 * Nw["m"] * Nw["p"] * head["mlmc"]["outer_products"] / head["mlmc"]["value"] / 1e12
    return {"workload": Nw["name"], "metric": "time to RMSE eps for E[f(AB)], f(x) = |x| H(2 - x)", "unit": "s",
            "eps_abs": eps, "precision": Nw["precision"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAKS["fp32"], "unit": "TFLOP/s",
                         "frac": achieved / ALU_PEAKS["fp32"], "traffic": None,
                         "peak_source": ALU_PEAKS["source"],
                         "kernel": "level_cuda_core_kernel<float, F = |x| H(2 - x)>",
                         "note": "end to end (pilot and allocation rounds of Alg. 2 included), ratio 2"},
            "mlmc": head["mlmc"], "mc_finest_level": head["mc_uniform"],
            "mc_over_mlmc": head["mc_uniform_over_mlmc"], "sweep": sweep, "bf16": bf16}


XI = dict(name="sparse_rows_64x4096x64", m=64, n=4096, p=64, c0=16, R=2, L=5, pilot=256, rel_rmse=1e-2,
          precision="fp32", row_density=0.2)


def _xi_params():
    """The structure of the paper's matrix example (Sec. 5.2: entries of A growing with the
    column index, B with Bernoulli(0.2) support) in this model's laws: the precision workload's
    M ~ U[-1,1], S ~ U[0.1,1] (seeds 0 and 1), column k of M and S scaled by 4 (k + 1) / n, and
    each row of M' and S' kept with probability 0.2 (Philox-seeded draw, seed 2), else zero."""
    from paper_1904_00429_gb300.inputs import make_params
    X = XI
    pp = make_params(X["m"], X["n"], X["p"], seed_A=0, seed_B=1, dtype=np.float64)
    col = 4.0 * (np.arange(X["n"]) + 1.0) / X["n"]
    keep = (np.random.Generator(np.random.Philox(1002)).uniform(size=X["n"]) < X["row_density"])[:, None]
    return [x.astype(np.float32) for x in (pp.M * col, pp.S * col, pp.Mp * keep, pp.Sp * keep)]


def _measure_xi(args, dev, stream):
    """MLMC of E[AB] under the uniform law xi^u and the variance-optimal xi** (Thm 3.1) on the
    same problem and target, each end to end through mlmc_estimate (pilot, allocation, top-up)."""
    import torch

    from paper_1904_00429_gb300 import binding

    X = XI
    params = _xi_params()
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in params]
    mu = params[0].astype(np.float64) @ params[2].astype(np.float64)
    eps = X["rel_rmse"] * float(np.linalg.norm(mu))
    out = {}
    # FP32 (CUDA cores) under both laws, then BF16 (tensor cores, the slot weights folded into B)
    for key, law, prec in (("uniform", "uniform", X["precision"]), ("optimal", "optimal", X["precision"]),
                           ("bf16_uniform", "uniform", "bf16"), ("bf16_optimal", "optimal", "bf16")):
        spec = binding.ProblemSpec(*ts, seed_A=3, seed_B=4, seed_idx=5, problem_id=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with binding.Plan([spec], c0=X["c0"], L=X["L"], ratio=X["R"], precision=prec, pilot_n=X["pilot"],
                          sampling=law, stream=stream) as plan:
            (Y,), (rep,) = plan.estimate([eps])
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        err = float(np.linalg.norm(Y.cpu().numpy() - mu))
        out[key] = {"value": t, "N_l": rep["N"], "V_l": rep["V"], "outer_products": rep["outer_products"],
                    "rmse_pred": rep["rmse_pred"], "error": err, "precision": prec,
                    "timing": "end to end through mlmc_estimate, plan creation included"}
    # FMAs of the contraction (2 m p per sampled outer product) over the end-to-end time of xi**
    achieved = 2.0 * X["m"] * X["p"] * out["optimal"]["outer_products"] / out["optimal"]["value"] / 1e12
    return {"workload": X["name"], "metric": "time to rel. RMSE 1e-2 for E[AB] under xi^u and xi**", "unit": "s",
            "eps_abs": eps, "precision": X["precision"], "uniform": out["uniform"], "optimal": out["optimal"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAKS["fp32"], "unit": "TFLOP/s",
                         "frac": achieved / ALU_PEAKS["fp32"], "traffic": None,
                         "peak_source": ALU_PEAKS["source"],
                         "kernel": "level_cuda_core_kernel<float, XI>",
                         "note": "xi** run end to end (plan creation, pilot and allocation included)"},
            "uniform_over_optimal": out["uniform"]["value"] / out["optimal"]["value"],
            "V0_uniform_over_optimal": out["uniform"]["V_l"][0] / out["optimal"]["V_l"][0],
            "bf16": {"uniform": out["bf16_uniform"], "optimal": out["bf16_optimal"],
                     "uniform_over_optimal": out["bf16_uniform"]["value"] / out["bf16_optimal"]["value"],
                     "fp32_optimal_over_bf16_optimal": out["optimal"]["value"] / out["bf16_optimal"]["value"],
                     "kernel": "level_tc_bf16_kernel (xi** weights folded into B before rounding)"}}


BATCHED = dict(name="batched_64_problems", count=64, shape_seed=7, c0=32, R=2, pilot=256, rel_rmse=1e-3,
               step_outer=4.0e8, precision="bf16")


_BATCHED_INPUTS = {}

# DRAM bytes (read + write) per algorithmic gathered byte of the batched kernel, by tile, from one
# ncu pass over one launch of a profile case: 1128 on the workload's first 8 problems (29.995 GB
# algorithmic), the CTA pair 3256 on its first 8 problems of more than 128 rows and columns
# (21.937 GB), which carry most of the gathered bytes
BATCHED_TRAFFIC = {1128: {"dram_over_algorithmic": (36247647744 + 71866112) / 29995171840,
                          "captured_on": "batched_8_problems",
                          "source": "profiles/level_tc_bf16_batched_64_problems.md"},
                   3256: {"dram_over_algorithmic": (22977974784 + 119399936) / 21936668672,
                          "captured_on": "batched_8_large_problems",
                          "source": "profiles/level_tc_bf16_batched_64_problems.md"}}


def _measure_batched(args, dev, stream, peaks, peak_kind, precision="bf16", step_target=None, steps=None, warmup=None):
    """64 problems (m, p log-uniform on [32, 512], n log-uniform on [4096, 262144], L+1 uniform on
    3..9; M ~ N(0,1), S ~ U[0.05, 2]; c_l = 32 * 2^l; BF16) through mlmc_level_stats_batch: one
    persistent launch per wave, graph-replayed.  After the pilot (256 samples per level, which
    also runs the tile autotuner) and each problem's own allocation for eps_q = 1e-3 ||M_q M'_q||_F,
    every step evaluates B = max(8, ceil(f N)) fresh samples of every (problem, level) in one
    batched call; the full run's time is projected by the ratio of sampled outer products."""
    import torch

    from paper_1904_00429_gb300 import binding
    from paper_1904_00429_gb300.inputs import batched_shapes, make_params

    Bc = BATCHED
    shapes = batched_shapes(Bc["count"], Bc["shape_seed"])
    key = (str(dev), Bc["count"], Bc["shape_seed"])
    if key not in _BATCHED_INPUTS:
        # drawn once per process: the BF16 run and its FP32 comparator use the same problems
        specs, eps, mpq = [], [], []
        t0 = time.perf_counter()
        for q, (m, n, p, L) in enumerate(shapes):
            pp = make_params(m, n, p, law="gauss", seed_A=2 * q, seed_B=2 * q + 1, seed_idx=2, problem_id=q,
                             dtype=np.float32)
            ts = [torch.from_numpy(x).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
            specs.append(binding.ProblemSpec(*ts, seed_A=2 * q, seed_B=2 * q + 1, seed_idx=2, problem_id=q, L=L))
            eps.append(Bc["rel_rmse"] * float(np.linalg.norm(pp.exact_mean())))
            mpq.append((m, p))
            del pp
        _BATCHED_INPUTS[key] = (specs, eps, mpq, time.perf_counter() - t0)
    specs, eps, mpq, gen_s = _BATCHED_INPUTS[key]
    Lmax = max(L for *_, L in shapes)
    plan = binding.Plan(specs, c0=Bc["c0"], L=Lmax, ratio=Bc["R"], precision=precision, pilot_n=Bc["pilot"],
                        stream=stream)
    step_target = Bc["step_outer"] if step_target is None else step_target
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    levels = [L for *_, L in shapes]
    ranges = [(q, l) for q in range(len(shapes)) for l in range(levels[q] + 1)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.level_stats_batch([(q, l, 0, Bc["pilot"]) for q, l in ranges])
    plan.synchronize()
    pilot_s = time.perf_counter() - t0
    tile, tune = plan.batch_tile()
    Nl = plan.allocate(eps)
    cl = [Bc["c0"] * Bc["R"]**l for l in range(Lmax + 1)]
    full_outer = sum(Nl[q][l] * cl[l] for q, l in ranges)
    f = step_target / full_outer
    B = {(q, l): max(8, int(math.ceil(f * Nl[q][l]))) for q, l in ranges}
    step_outer = sum(B[r] * cl[r[1]] for r in ranges)
    next_id = {r: max(Bc["pilot"], 0) for r in ranges}

    def step():
        plan.level_stats_batch([(q, l, next_id[(q, l)], B[(q, l)]) for q, l in ranges])
        for r in ranges:
            next_id[r] += B[r]

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches0 = plan.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    plan.synchronize()
    launches = plan.launch_count() - launches0
    t = e0.elapsed_time(e1) / 1e3 / steps
    T = t * full_outer / step_outer
    flops = sum(2.0 * mpq[q][0] * mpq[q][1] * B[(q, l)] * cl[l] for q, l in ranges)
    bytes_alg = sum(2.0 * (mpq[q][0] + mpq[q][1]) * 4 * B[(q, l)] * cl[l] for q, l in ranges)
    plan.close()
    hbm = bytes_alg / t / 1e9
    tpeak = peaks["bf16_tflops_sustained"]
    tfl = flops / t / 1e12
    bound_hbm = bytes_alg / (peaks["hbm_gbs"] * 1e9) >= flops / (tpeak * 1e12)
    if precision in ("fp32", "fp64"):
        # CUDA cores, one launch sequence per range: bound by FMA issue
        peak = ALU_PEAKS[precision]
        roof = {"bound": "alu", "achieved": tfl, "peak": peak, "unit": "TFLOP/s",
                "frac": tfl / peak if peak else None, "traffic": None, "peak_source": ALU_PEAKS["source"],
                "hbm_achieved_gbs": hbm, "kernel": f"level_cuda_core_kernel<{precision}> (one range at a time)"}
        return {"workload": Bc["name"], "precision": precision,
                "metric": "time-to-RMSE 1e-3 for every problem's E[A_q B_q] (projected)",
                "value": T, "unit": "s", "ms_per_step": 1e3 * t, "step_fraction": f,
                "outer_products_per_s": step_outer / t, "full_run_outer_products": full_outer,
                "gpu_launches": launches, "pilot_s": pilot_s, "problems": len(shapes), "levels": len(ranges),
                "roofline": roof, "clocks": clocks.summary()}
    roof = ({"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm / peaks["hbm_gbs"],
             "tensor_achieved_tflops": tfl, "tensor_frac": tfl / tpeak}
            if bound_hbm else
            {"bound": "tensor", "achieved": tfl, "peak": tpeak, "unit": "TFLOP/s", "frac": tfl / tpeak,
             "hbm_achieved_gbs": hbm})
    # DRAM traffic per level launch: the DRAM bytes per algorithmic byte of one captured launch of
    # the batched kernel on this tile times this step's algorithmic bytes per launch; null for a
    # tile without a capture
    waves = max(1, launches // (3 * steps))
    bt = BATCHED_TRAFFIC.get(tile)
    traffic = None if bt is None else {
        "value": bt["dram_over_algorithmic"] * bytes_alg / waves, "unit": "bytes per launch", "launches": waves * steps,
        "algorithmic_bytes_per_launch": bytes_alg / waves, "captured_on": bt["captured_on"], "source": bt["source"]}
    roof.update({"traffic": traffic,
                 "peak_source": f"{'hbm_gbs' if bound_hbm else 'bf16_tflops_sustained'} ({peak_kind})",
                 "kernel": "level_tc_bf16_kernel<batched>"})
    return {"workload": Bc["name"], "metric": "time-to-RMSE 1e-3 for every problem's E[A_q B_q] (projected)",
            "value": T, "unit": "s", "ms_per_step": 1e3 * t, "step_fraction": f,
            "outer_products_per_s": step_outer / t, "full_run_outer_products": full_outer,
            "gpu_launches": launches, "tile": tile, "autotune_ms": tune, "pilot_s": pilot_s,
            "input_generation_s": gen_s, "problems": len(shapes), "levels": len(ranges),
            "roofline": roof, "clocks": clocks.summary()}


def run_ours(args):
    import torch

    from paper_1904_00429_gb300.inputs import make_params

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = dict(WORKLOAD)
    pp = make_params(W["m"], W["n"], W["p"], seed_A=0, seed_B=1, dtype=np.float32)
    host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    mu = pp.exact_mean()
    W["eps"] = W["rel_rmse"] * float(np.linalg.norm(mu))
    stream = torch.cuda.current_stream(dev)

    peaks_alu = measure_alu_peaks(stream) if rank == 0 else None
    head = _measure(args, args.precision, W, host, dev, rank, stream, world, with_e2e=True)
    others = []
    if not args.no_compare:
        for prec in ("fp32", "fp8"):
            if prec != args.precision:
                others.append(_measure(args, prec, W, host, dev, rank, stream, world, with_e2e=False))
    T = head["T"]
    if world > 1:
        tt = torch.tensor([T, head["total_ms"]] + [o["T"] for o in others], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        # every rank evaluates its own sample ranges: the N_l are split across the ranks
        T, head["total_ms"] = float(tt[0]) / world, float(tt[1])
        for i, o in enumerate(others):
            o["T"] = float(tt[2 + i]) / world
    if rank != 0:
        return
    peaks, peak_kind = read_peaks()
    from paper_1904_00429_gb300 import binding as _binding
    gen_rate = _binding.generation_rate(stream)   # the generation bound, measured on this GPU now
    m, n, p = W["m"], W["n"], W["p"]
    prec = head["prec"]
    line = {
        "metric": "time-to-RMSE 1e-3 for E[AB] (projected from the measured per-level sample rate)",
        "value": T, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head["total_ms"] / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16", "fp8": "e4m3"}[prec],
        "data": "synthetic",
        "config": {"workload": W["name"], "m": m, "n": n, "p": p, "c0": W["c0"], "ratio": W["R"], "L": W["L"],
                   "pilot": W["pilot"], "eps_abs": W["eps"], "N_l": head["Nl"], "batch_per_step": head["B"],
                   "inputs": "parameters 256 MiB > L2 (random row gathers), no flush", "precision": prec},
        "outer_products_per_s": head["outer"] / head["sample_s"],
        "per_level_us_per_sample": [1e6 * t for t in head["t_l"]],
        "gpu_launches": head["launches"],
        "roofline": _roofline(head, W, peaks, peak_kind, gen_rate),
        "peaks_measured": {"fp32_tflops": peaks_alu["fp32_flops"] / 1e12, "fp64_tflops": peaks_alu["fp64_flops"] / 1e12,
                           "int32_imad_per_s": peaks_alu["int32_imad_per_s"], "mufu_sin_per_s": peaks_alu["mufu_sin_per_s"],
                           "generation_entries_per_s": gen_rate,
                           "how": "mlmc_measure_peaks / mlmc_measure_generation_rate in this run"},
        "clocks": head["clocks"],
        "e2e": {"value": head["e2e_overhead_s"] + T, "unit": "s", "h2d_bytes_per_step": head["h2d"],
                "d2h_bytes_per_step": head["d2h"], "overhead_s": head["e2e_overhead_s"], "api": head["e2e_api"]},
    }
    if others:
        line["compare"] = {o["prec"]: {"value": o["T"], "unit": "s",
                                       "outer_products_per_s": o["outer"] / o["sample_s"],
                                       "speedup_of_headline": o["T"] / T,
                                       "roofline": _roofline(o, W, peaks, peak_kind, gen_rate),
                                       "clocks": o["clocks"]}
                           for o in others}
    if not args.no_adjoint and world == 1:
        line["adjoint"] = _measure_adjoint(args, host, dev, stream, peaks, peak_kind, gen_rate)
    if not args.no_batched and world == 1:
        line["batched"] = _measure_batched(args, dev, stream, peaks, peak_kind)
        if not args.no_compare:
            # the plain FP32 comparator of the same 64 problems (CUDA cores, the ranges in turn), on
            # steps of the same size (one timed step)
            fp32b = _measure_batched(args, dev, stream, peaks, peak_kind, precision="fp32",
                                     step_target=BATCHED["step_outer"], steps=1, warmup=1)
            line["batched"]["compare"] = {"fp32": fp32b, "fp32_over_bf16": fp32b["value"] / line["batched"]["value"]}
    if not args.no_nonlinear and world == 1:
        line["nonlinear"] = _measure_nonlinear(args, dev, stream)
    if not args.no_xi and world == 1:
        line["xi"] = _measure_xi(args, dev, stream)
    if not args.no_dedupe and world == 1:
        line["dedupe_bound"] = _measure_dedupe_bound(args, head, W, dev, stream)
    def _floats(text):
        return [float(x) for x in text.split(",") if x.strip("'\" ")]

    def _words(text):
        return [x for x in text.split(",") if x.strip("'\" ")]

    ttr_sets = [(_floats(args.ttr), _words(args.ttr_precisions)),
                (_floats(args.ttr_side), _words(args.ttr_side_precisions))]
    ttr_sets = [(r, p) for r, p in ttr_sets if r and p]
    if ttr_sets and world == 1:
        out = None
        for rels, precs in ttr_sets:
            o = _measure_ttr(args, rels, precs, dev, stream)
            if out is None:
                out = o
            else:
                out["runs"] += o["runs"]
        by = {(r["precision"], r["rel_rmse"]): r["seconds"] for r in out["runs"]}
        out["fp32_over"] = {f"{p}@{rel:g}": by[("fp32", rel)] / t for (p, rel), t in by.items()
                            if p != "fp32" and ("fp32", rel) in by}
        line["ttr_64x1024x64"] = out
    if args.ladder and world == 1:
        rels = [float(x) for x in args.ladder.split(",")]
        line["ladder"] = _measure_ladder(args, rels, W, host, mu, dev, stream, T)
    if not args.no_cpu_baseline and world == 1:
        t_cpu, _ = cpu_baseline_sample(W)
        T_one = sum(nl * t for nl, t in zip(head["Nl"], t_cpu))
        pool = OraclePool(W)
        t_all, wall = pool.round(1 << 42)
        pool.close()
        T_cpu = sum(nl * t for nl, t in zip(head["Nl"], t_all))
        line["cpu_baseline"] = {"value": T_cpu, "unit": "s", "cores": pool.cores, "kind": "oracle",
                                "sample": f"one FP64 oracle sample per level 0..8 on each of {pool.cores} worker "
                                          f"processes ({wall:.1f} s wall), projected with the same N_l",
                                "single_core": {"value": T_one, "unit": "s", "cores": 1,
                                                "sample": "one FP64 oracle sample per level 0..8, one process"}}
    print(json.dumps(line), flush=True)


PROFILE_CASES = {
    # name: (precision, level, samples) on the 256x65536x256 workload (parameters 256 MiB > L2)
    "tc_bf16_level0": ("bf16", 0, 16384),
    "tc_bf16_level8": ("bf16", 8, 2432),
    "tc_bf16_pair_level8": ("bf16", 8, 2432),
    "tc_e4m3_level0": ("fp8", 0, 16384),
    "tc_e4m3_level8": ("fp8", 8, 2432),
    "cuda_core_f32_level0": ("fp32", 0, 4096),
}


SMALL_PROFILE_CASES = {
    # name: (precision, level, samples per launch) on the 64x1024x64 workload (one launch each)
    "small_bf16_level0": ("bf16", 0, 262144),
    "small_bf16_level5": ("bf16", 5, 8192),
    "small_f32_level0": ("fp32", 0, 262144),
    "small_f32_level5": ("fp32", 5, 8192),
}


def run_profile_case(args):
    """One small invocation of one kernel for ncu (no bench line): two warm-up launches, then the
    launch to capture (the third launch of the level kernel in the process), or, for "adjoint",
    two backward calls of the 256x65536x256 adjoint workload (N_l = 256 per level, BF16)."""
    import torch

    from paper_1904_00429_gb300 import binding
    from paper_1904_00429_gb300.inputs import make_params, make_target

    dev = torch.device("cuda:0")
    if args.profile_case in ("batched_8_problems", "batched_8_large_problems"):
        # the first 8 problems of the batched workload on the 128 x 128 tile, or the first 8 of more
        # than 128 rows and columns on the CTA pair; 256 samples per level
        from paper_1904_00429_gb300.inputs import batched_shapes
        large = args.profile_case == "batched_8_large_problems"
        all_shapes = list(enumerate(batched_shapes(BATCHED["count"], BATCHED["shape_seed"])))
        picked = [(q0, sh) for q0, sh in all_shapes if not large or (sh[0] > 128 and sh[2] > 128)][:8]
        specs, ranges = [], []
        for q, (q0, (m, n, p, L)) in enumerate(picked):
            pq = make_params(m, n, p, law="gauss", seed_A=2 * q0, seed_B=2 * q0 + 1, seed_idx=2, problem_id=q0,
                             dtype=np.float32)
            specs.append(binding.ProblemSpec(*[torch.from_numpy(x).to(dev) for x in (pq.M, pq.S, pq.Mp, pq.Sp)],
                                             seed_A=2 * q0, seed_B=2 * q0 + 1, seed_idx=2, problem_id=q0, L=L))
            ranges += [(q, l) for l in range(L + 1)]
        plan = binding.Plan(specs, c0=BATCHED["c0"], L=8, precision="bf16", tile_override=3256 if large else 1128)
        waves = []
        for i in range(3):
            c0 = plan.launch_count()
            plan.level_stats_batch([(q, l, 256 * i, 256) for q, l in ranges])
            waves.append((plan.launch_count() - c0) // 3)   # a wave: the level kernel and two merges
        plan.synchronize()
        plan.close()
        shapes = [sh for _, sh in picked]
        alg = sum(256 * BATCHED["c0"] * BATCHED["R"]**l * 2 * (shapes[q][0] + shapes[q][2]) * 4 for q, l in ranges)
        print(json.dumps({"profile_case": args.profile_case, "status": "ok", "level_launches_per_call": waves,
                          "algorithmic_bytes_per_call": alg}), flush=True)
        return
    if args.profile_case == "cuda_core_f32_xi_level3":
        # the xi** variant of the CUDA-core kernel on the sparse-row workload, level 3 (c = 128)
        xt = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in _xi_params()]
        plan = binding.Plan([binding.ProblemSpec(*xt, seed_A=3, seed_B=4, seed_idx=5)], c0=XI["c0"], L=XI["L"],
                            precision="fp32", sampling="optimal")
        for i in range(3):
            plan.level_stats(0, 3, i * 19456, 19456)
        plan.synchronize()
        plan.close()
        print(json.dumps({"profile_case": args.profile_case, "status": "ok"}), flush=True)
        return
    if args.profile_case in SMALL_PROFILE_CASES:
        # one level of the 64 x 1024 x 64 workload (c_l = 16 * 2^l): three launches of one level kernel
        prec, level, count = SMALL_PROFILE_CASES[args.profile_case]
        ps = make_params(64, 1024, 64, seed_A=0, seed_B=1, dtype=np.float32)
        st = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (ps.M, ps.S, ps.Mp, ps.Sp)]
        plan = binding.Plan([binding.ProblemSpec(*st)], c0=16, L=5, precision=prec)
        for i in range(3):
            plan.level_stats(0, level, i * count, count)
        plan.synchronize()
        plan.close()
        print(json.dumps({"profile_case": args.profile_case, "status": "ok"}), flush=True)
        return
    pp = make_params(256, 65536, 256, seed_A=0, seed_B=1, dtype=np.float32)
    ts = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (pp.M, pp.S, pp.Mp, pp.Sp)]
    if args.profile_case == "adjoint":
        plan = binding.Plan([binding.ProblemSpec(*ts)], c0=64, L=8, precision="bf16")
        for l in range(9):
            plan.level_stats(0, l, 0, ADJOINT["N"])
        (Y,) = plan.telescoping_sum()
        G = 2.0 * (Y - torch.from_numpy(make_target(256, 256)).to(dev))
        plan.backward([G])
        plan.backward([G])
    else:
        prec, level, count = PROFILE_CASES[args.profile_case]
        plan = binding.Plan([binding.ProblemSpec(*ts)], c0=64, L=8, precision=prec,
                            tile_override=3256 if "pair" in args.profile_case else 0)
        for i in range(3):
            plan.level_stats(0, level, i * count, count)
    plan.synchronize()
    plan.close()
    print(json.dumps({"profile_case": args.profile_case, "status": "ok"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64", "bf16", "fp8"], default="bf16")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 and FP8 comparison measurements")
    ap.add_argument("--tile", type=int, default=0, help="tensor-core tile id of the headline workload (0: automatic)")
    ap.add_argument("--fp32-tile", type=int, default=0,
                    help="CUDA-core tile id of the FP32 comparator (0: automatic; 64064, 128064, 128128)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the backward measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-problem batched measurement")
    ap.add_argument("--no-nonlinear", action="store_true", help="skip the E[f(AB)] adaptive-L measurement")
    ap.add_argument("--no-xi", action="store_true", help="skip the xi^u / xi** comparison")
    ap.add_argument("--no-dedupe", action="store_true", help="skip the index-dedupe bound")
    ap.add_argument("--ladder", default="3e-2", help="comma-separated relative RMSE targets to run end to end "
                    "through mlmc_estimate on the headline workload (about a minute at 3e-2; '' to skip)")
    ap.add_argument("--ttr", default="1e-3", help="comma-separated relative RMSE targets of the end-to-end "
                    "time-to-RMSE runs on the 64x1024x64 workload ('' to skip)")
    ap.add_argument("--ttr-precisions", default="bf16", help="precisions of those runs (each about 3 minutes "
                    "at 1e-3)")
    ap.add_argument("--ttr-side", default="3e-3", help="relative targets of the shorter runs of every "
                    "precision in --ttr-side-precisions ('' to skip)")
    ap.add_argument("--ttr-side-precisions", default="bf16,fp32,fp8", help="precisions of the shorter runs")
    ap.add_argument("--profile-case", choices=sorted(list(PROFILE_CASES) + list(SMALL_PROFILE_CASES) +
                                                     ["adjoint", "batched_8_problems", "batched_8_large_problems",
                                                      "cuda_core_f32_xi_level3"]),
                    default=None,
                    help="run one small kernel invocation for ncu instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
