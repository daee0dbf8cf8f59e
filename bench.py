"""Throughput benchmark of the exact exponential field step (cell*mode*steps/s).

Default line: the uneven-instance batch - 64 seeded simulations (Nz from {512, 1024, 2048, 4096}, Nr in
[64, 512], M in {1, 2, 3}, order 8 or 16, m = 1 pulse with waist 10-40 dr, seeded smooth current on every
mode) advanced together by one captured CUDA graph per step (one persistent grouped projection launch, every
instance's spectral kernel on its own branch, one grouped back-projection launch), split-BF16 (BF16x6, FP32
accumulation), against the plain FP64 path on the same mix, with the per-field error of one step against
that FP64 step, the per-step latency percentiles, the stage roofline, the host-buffer end-to-end rate and
two single-instance legs (the 2048 x 256 two-mode and the 8192 x 512 three-mode workloads).  Inputs (8 GB
resident) are far larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16x3|bf16x6|fp32|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores, same mix
    python bench.py --mode step ...        # one instance (--workload), L2 flushed between steps
    python bench.py --mode serve ...       # Poisson request stream through the continuous-batching server

N > 1 (torchrun, one process per GPU) runs independent replicas: the step has no
data-path exchange, so each rank advances its own copy and `value` sums them.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell\u00b7mode\u00b7steps/s split-BF16 batched vs plain FP64 at \u22641e-6 rel err; p50/p99 latency"
STEP_METRIC = "cell*mode*steps/s (exact exponential field step, one real-space round trip per step)"
UNIT = "cell*mode*steps/s"
BATCH_WORKLOAD = "uneven_mix_64: 64 seeded instances, Nz in {512,1024,2048,4096}, Nr in [64,512], M in {1,2,3}, " \
                 "order 8/16, 100-step batches advanced one step per graph replay"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), float(p[4]), p[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        loaded = [r for r in rows if r[2] >= 30] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over the ranks of the process group (x itself without one): every timed region of a
    replica run is reported as its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, seconds, world):
    """Whole-job throughput of `world` independent replicas that each processed units_per_rank units, timed
    by the slowest rank (seconds = max over ranks)."""
    return units_per_rank * world / seconds


STAGE_SOURCE = {"projection": "k_tc.cu", "spectral": "k_spectral32.cu", "backprojection": "k_tc.cu"}


def recorded_traffic(stage, workload, prec):
    """DRAM bytes per launch of a stage's kernel from profiles/traffic.json (one ncu capture), or None
    when no capture exists for this workload/precision or the kernel source changed since (sha256)."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[f"{stage}/{workload}/{prec}"]
        src = os.path.join(ROOT, "paper_2605_12132_gb300", "csrc", STAGE_SOURCE[stage])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
            return None
        return rec["dram_bytes_per_launch"]
    except Exception:
        return None


def _rounded(pipeline):
    """Pipeline shares of the tensor-core kernels, rounded for the JSON line."""
    return {k: {a: (round(b, 4) if isinstance(b, float) else b) for a, b in v.items()} for k, v in pipeline.items()}


def gemm_flops(w, hasJ):
    """Algorithmic FLOPs of one step's radial transforms: each nonzero n x n block of the
    (3n)^2 projection / back-projection matrices times a complex column, per z row and mode."""
    n = w.Nr
    fwd = (15 if hasJ else 10)
    bwd = 10
    per_block = 4.0 * n * n * w.Nz   # real matrix x complex vector = 2 real MACs per entry
    return fwd * per_block * len(w.modes), bwd * per_block * len(w.modes)


def spectral_bytes(w, hasJ, elt):
    """Algorithmic bytes of the spectral stage: the coefficient arrays read once, written once."""
    return ((9 if hasJ else 6) + 6) * w.Nz * w.Nr * len(w.modes) * elt


def cpu_oracle_rate(w, F, J, kz_count, mode_index=None, seed=123):
    """The FP64 oracle (per-kz dense eigendecomposition evaluator) on a bounded sample of kz columns of one
    mode of workload w (an object with Nz, Nr, modes, order, dz, dr, dt)."""
    from oracle import maxwell as mx
    rng = np.random.default_rng(seed)
    qs = list(rng.choice(w.Nz, size=kz_count, replace=False))
    m_i = len(w.modes) - 1 if mode_index is None else mode_index
    t0 = time.perf_counter()
    mx.step_spectral(F[m_i], None if J is None else J[m_i], w.Nz, w.Nr, w.modes[m_i], w.order, w.dz, w.dr, w.dt,
                     nsteps=1, kz_subset=qs, method="eig")
    dt = time.perf_counter() - t0
    return kz_count * w.Nr / dt, dt


class _Inst:
    """One instance of the uneven mix seen as a workload (sizes and spacings)."""

    def __init__(self, c):
        self.Nz, self.Nr, self.order = c["Nz"], c["Nr"], c["order"]
        self.modes = list(range(c["M"] + 1))
        self.dz, self.dr, self.dt = 1 / 16, 1 / 4, 1 / 16
        self.name = f"mix instance Nz={self.Nz} Nr={self.Nr} M={c['M']} order={self.order}"


def _oracle_sample(cfgs):
    """The mix instance the CPU oracle samples: the one at the lower quartile of the radial sizes (a dense
    (6 Nr - 3)^2 eigendecomposition per kz column keeps a step of the oracle to a few seconds)."""
    from paper_2605_12132_gb300 import inputs
    c = sorted(cfgs, key=lambda c: c["Nr"])[len(cfgs) // 4]
    F, J = inputs.instance_inputs(c)
    return _Inst(c), F, J


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle as it stands, on the host cores (rank 0 only), on the default line's
    workload: per step one kz column of one mode of the lower-quartile-size instance of the uneven mix."""
    if rank != 0:
        return
    from paper_2605_12132_gb300 import inputs
    cfgs = inputs.uneven_instances(args.instances, seed=0)
    w, F, J = _oracle_sample(cfgs)
    for k in range(args.warmup):
        cpu_oracle_rate(w, F, J, 1, mode_index=1, seed=100 + k)
    tot, cells = 0.0, 0
    for k in range(args.steps):
        _, dt = cpu_oracle_rate(w, F, J, 1, mode_index=1, seed=200 + k)
        tot += dt
        cells += w.Nr
    value = cells / tot
    cores = os.cpu_count()
    sample = (f"one kz column ({w.Nr} cells) of mode 1 of the lower-quartile-size instance of the mix ({w.name}) per step, "
              "per-kz dense eigendecomposition evaluator, FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uneven instances: Gaussian pulse + smooth random current)",
            "config": {"workload": BATCH_WORKLOAD, "precision": "fp64-oracle", "l2": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def _field_error_stats(torch, got, ref):
    """Largest relative L2 error per field (floor 1e-12 of the mode's norm) over the modes of one instance,
    split into fields carrying at least 10% of their mode's state and the rest: (strong, weak), None where a
    class has no field."""
    d = got.to(torch.complex128) - ref
    num = torch.linalg.vector_norm(d, dim=(2, 3))
    den = torch.linalg.vector_norm(ref, dim=(2, 3))
    tot = torch.linalg.vector_norm(ref, dim=(1, 2, 3))[:, None]
    rel = num / torch.maximum(den, 1e-12 * tot)
    share = den / tot
    strong = rel[share >= 0.1]
    weak = rel[share < 0.1]
    return (float(strong.max()) if strong.numel() else None, float(weak.max()) if weak.numel() else None)


def _build_plans(fd, cfgs, prec):
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        return list(ex.map(lambda c: fd.fdetd_plan(c["Nz"], c["Nr"], c["M"], c["order"], 1 / 16, 1 / 4, 1 / 16,
                                                    precision=prec), cfgs))


def batch_gemm_flops(cfgs, hasJ=True):
    """Algorithmic FLOPs of one step's radial transforms over the mix (per cell and
    mode, 9 products of a real Nr x Nr matrix with a complex column forward including the current, 6 back,
    4 Nr flops each), and the dense-equivalent count the tensor-core kernels execute per bf16 product
    (15 / 10 nonzero Nr x Nr blocks of the folded projection / back-projection matrices)."""
    fa = ba = fe = be = 0.0
    for c in cfgs:
        cm = c["Nz"] * c["Nr"] * (c["M"] + 1)
        fa += (9 if hasJ else 6) * 4.0 * c["Nr"] * cm
        ba += 6 * 4.0 * c["Nr"] * cm
        fe += (15 if hasJ else 10) * 4.0 * c["Nr"] * cm
        be += 10 * 4.0 * c["Nr"] * cm
    return fa, ba, fe, be


def run_batch(args, rank, world, dist):
    """The default line: the uneven mix advanced by one captured graph per step."""
    import torch
    import paper_2605_12132_gb300 as fd
    from paper_2605_12132_gb300 import inputs

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    prec = args.precision or "bf16x6"
    cfgs = inputs.uneven_instances(args.instances, seed=0)
    t0 = time.perf_counter()
    plans = _build_plans(fd, cfgs, prec)
    plan_s = time.perf_counter() - t0
    host, dev = [], []
    cells = 0
    for c, p in zip(cfgs, plans):
        F, J = inputs.instance_inputs(c)
        host.append((F, J))
        dev.append((torch.from_numpy(F).to(p.complex_dtype).cuda(), torch.from_numpy(J).to(p.complex_dtype).cuda()))
        cells += c["Nz"] * c["Nr"] * (c["M"] + 1)
    batch = fd.FdetdBatch()
    for p, (f, j) in zip(plans, dev):
        batch.add(p, f, j)
    batch.set_profiling(True)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    batch.capture(1)
    capture_s = time.perf_counter() - t0
    groups = batch.groups()
    # one step from the initial state, kept for the accuracy check against the FP64 path
    batch.launch()
    torch.cuda.synchronize()
    one_step = [f.clone() for f, _ in dev]
    for _ in range(args.warmup - 1):
        batch.launch()
    barrier()
    # timed region: K graph replays, each bracketed by events on the launching stream
    clocks = ClockSampler()
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        evs[k][0].record(stream)
        batch.launch()
        evs[k][1].record(stream)
        torch.cuda.synchronize()
        batch.collect_stage_times()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    for p in plans:
        p.status()
    lat = np.array([a.elapsed_time(b) for a, b in evs])
    ms = max_over_ranks(float(lat.sum()), dist, "cuda")
    value = replica_rate(cells * args.steps, ms / 1e3, world)
    st = batch.stage_times()
    pipeline = _rounded(batch.pipeline_waits())

    # plain FP64 path on the same mix: its one-step result is the accuracy reference, its rate the baseline
    fp64_value = err = None
    if not args.no_fp64 and prec != "fp64":
        plans64 = _build_plans(fd, cfgs, "fp64")
        dev64 = [(torch.from_numpy(F).cuda(), torch.from_numpy(J).cuda()) for F, J in host]
        b64 = fd.FdetdBatch()
        for p, (f, j) in zip(plans64, dev64):
            b64.add(p, f, j)
        b64.capture(1)
        b64.launch()
        torch.cuda.synchronize()
        strong = weak = 0.0
        for g, (r, _) in zip(one_step, dev64):
            s_, w_ = _field_error_stats(torch, g, r)
            strong, weak = max(strong, s_ or 0.0), max(weak, w_ or 0.0)
        err = {"strong_fields_max": strong, "weak_fields_max": weak,
               "definition": "one step from the same state, per mode and field ||X - X_fp64|| / ||X_fp64|| (floor "
                             "1e-12 of the mode's norm), largest over the 64 instances; strong = fields with at least "
                             "10% of their mode's norm"}
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b64.launch()
        b.record(stream)
        torch.cuda.synchronize()
        for p in plans64:
            p.status()
        fp64_value = cells / (a.elapsed_time(b) / 1e3)
        b64.close()
        for p in plans64:
            p.close()
        del dev64, plans64
        torch.cuda.empty_cache()

    # end to end through the host-buffer form of the batch: every step copies every instance's fields and
    # current in from pinned host memory and the fields back out (the library's default: sixteen parts whose
    # copies overlap each other's compute; the serial form is timed beside it)
    hf = [torch.from_numpy(F).to(torch.complex64).pin_memory() for F, _ in host]
    hj = [torch.from_numpy(J).to(torch.complex64).pin_memory() for _, J in host]

    def time_host_steps():
        batch.step_host(hf, hj, 1)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            batch.step_host(hf, hj, 1)
        barrier()
        return max_over_ranks(time.perf_counter() - t0, dist, "cuda")

    batch.set_host_pipeline(1)
    e2e_serial = replica_rate(cells * args.e2e_steps, time_host_steps(), world)
    batch.set_host_pipeline(args.host_parts)
    e2e_s = time_host_steps()
    h2d = sum(t.numel() * t.element_size() for t in hf) + sum(t.numel() * t.element_size() for t in hj)
    d2h = sum(t.numel() * t.element_size() for t in hf)
    e2e_val = replica_rate(cells * args.e2e_steps, e2e_s, world)

    # roofline of the dominant stage, from the stage times recorded inside the timed graph replays
    peaks, src = _peaks()
    fa, ba, fe, be = batch_gemm_flops(cfgs)
    products = {"bf16x3": 3, "bf16x6": 6}.get(prec, 1)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in st.items()}
    dom = max(stage_ms, key=stage_ms.get)
    tsec = stage_ms[dom] / 1e3
    if dom == "spectral":
        algo = sum(15 * c["Nz"] * c["Nr"] * (c["M"] + 1) * 8 for c in cfgs)
        roof = {"bound": "hbm", "achieved": algo / tsec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        algo, execd = (fa, fe) if dom == "projection" else (ba, be)
        pk = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": algo * products / tsec / 1e12, "peak": pk, "unit": "TFLOP/s",
                "executed_tflops": execd * products / tsec / 1e12, "executed_frac": execd * products / tsec / 1e12 / pk,
                "note": f"achieved = the algorithmic flops (9 forward and 6 back Nr x Nr real products per cell and "
                        f"mode) x {products} bf16 products per FP32-accurate product; executed = the folded dense "
                        "blocks the kernel multiplies"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = recorded_traffic(dom, f"uneven_mix_{len(cfgs)}", prec)
    roof["algorithmic"] = algo
    roof["kernel"] = {"projection": "tcg_project_kernel (grouped, persistent)", "spectral": "spectral32_kernel",
                      "backprojection": "tcg_backproject_kernel (grouped, persistent)"}[dom]
    roof["peak_source"] = src
    roof["stage_ms_per_step"] = stage_ms
    roof["pipeline"] = pipeline

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        w, F, J = _oracle_sample(cfgs)
        rate, secs = cpu_oracle_rate(w, F, J, 2, mode_index=1)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"2 kz columns ({2 * w.Nr} cells) of mode 1 of the lower-quartile-size instance ({w.name}), one "
                         f"step, per-kz dense eigendecomposition evaluator, FP64 ({secs:.1f} s)"}

    legs = {}
    if not args.no_legs:
        for name in ("lwfa_m01_2048x256", "sweep_m012_8192x512"):
            legs[name] = run_step(args, inputs.workload(name), prec, leg=True)

    if rank == 0:
        launches_per_step = 2 * len(groups) + len(cfgs)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": prec + "-split/f32-accumulate" if prec.startswith("bf16") else prec,
                "data": "synthetic (seeded uneven instances: Gaussian pulse + smooth random current)",
                "config": {"workload": BATCH_WORKLOAD, "instances": len(cfgs), "cells_modes": cells,
                           "precision": prec, "parallelism": "replicas" if world > 1 else "single",
                           "l2": f"inputs larger than L2 ({sum(f.numel() * f.element_size() + j.numel() * j.element_size() for f, j in dev) / 1e9:.1f} GB resident)",
                           "fp64_value": fp64_value, "speedup_vs_fp64": value / world / fp64_value if fp64_value else None,
                           "rel_err_vs_fp64_1step": err, "plan_build_s": plan_s, "capture_s": capture_s,
                           "wall_s": t_wall,
                           "graph": "per step: one persistent grouped projection launch, every instance's spectral "
                                    "kernel on its own branch, one grouped back-projection launch",
                           "groups": [{k: g[k] for k in ("instances", "tn_proj", "tn_back", "sched_proj",
                                                         "sched_back", "proj_tiles", "back_tiles", "tuned_ms")}
                                      for g in groups],
                           "legs": legs},
                "latency": {"unit": "ms per step (one graph replay)", "p50": float(np.percentile(lat, 50)),
                            "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "pipeline_parts": args.host_parts, "serial_value": e2e_serial,
                        "api": "fdetd_batch_step_host"},
                "gpu_launches": launches_per_step * args.steps, "roofline": roof, "cpu_baseline": cpu,
                "clocks": clk}
        print(json.dumps(line), flush=True)


def run_taylor(args, w):
    """The paper's Taylor-polynomial stepper (banded stencils, FP32) on the same workload; its error after one
    step against the exact exponential step (FP64 path) is reported beside the throughput."""
    import torch
    import paper_2605_12132_gb300 as fd
    from paper_2605_12132_gb300 import inputs
    F, J = inputs.workload_inputs(w)
    plan = fd.fdetd_taylor_plan(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, args.taylor_order, args.substeps)
    f0 = torch.from_numpy(F).to(torch.complex64).cuda()
    Jd = torch.from_numpy(J).to(torch.complex64).cuda() if J is not None else None
    f = f0.clone()
    fd.fdetd_taylor_step(plan, f, Jd, 1)
    torch.cuda.synchronize()
    p64 = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision="fp64")
    x64 = torch.from_numpy(F).cuda()
    fd.fdetd_step(p64, x64, torch.from_numpy(J).cuda() if J is not None else None, 1)
    torch.cuda.synchronize()
    a, b = f.cpu().numpy().astype(np.complex128), x64.cpu().numpy()
    err = max(float(np.linalg.norm(a[i, c] - b[i, c]) / max(np.linalg.norm(b[i, c]), 0.1 * np.linalg.norm(b[i])))
              for i in range(len(w.modes)) for c in range(6))
    p64.close()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        fd.fdetd_taylor_step(plan, f, Jd, 1)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        fd.fdetd_taylor_step(plan, f, Jd, 1)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in evs)
    cells = w.Nz * w.Nr * len(w.modes)
    line = {"metric": METRIC + " [paper's Taylor stepper]", "value": cells * args.steps / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Gaussian pulse + seeded smooth random current)",
            "config": {"workload": w.name, "taylor_order": args.taylor_order, "substeps": args.substeps,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "error_vs_exact_step": err, "launches_per_step": plan.launches_per_step + 1}}
    # roofline of the term kernel: per term and cell*mode it reads the previous term and the running sum and
    # writes the new term and the sum, 6 complex64 fields each (192 B)
    algo = cells * 192 * plan.launches_per_step
    peaks, src = _peaks()
    roof = {"bound": "hbm", "achieved": algo / (ms / args.steps / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"traffic": None, "algorithmic": algo, "kernel": "taylor_term_kernel", "peak_source": src})
    line["roofline"] = roof
    print(json.dumps(line), flush=True)


def run_destagger(args, w):
    """Destagger of the workload's fields to the primary grids (HBM-bound: 12 complex values per cell*mode)."""
    import torch
    import paper_2605_12132_gb300 as fd
    from paper_2605_12132_gb300 import inputs
    prec = args.precision or "bf16x6"
    F, _ = inputs.workload_inputs(w)
    plan = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision=prec)
    f = torch.from_numpy(F).to(plan.complex_dtype).cuda()
    out = torch.empty_like(f)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        fd.fdetd_destagger(plan, f, out)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        fd.fdetd_destagger(plan, f, out)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in evs) / args.steps
    cells = w.Nz * w.Nr * len(w.modes)
    algo = cells * 12 * f.element_size()
    peaks, src = _peaks()
    roof = {"bound": "hbm", "achieved": algo / (ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"traffic": None, "algorithmic": algo, "kernel": "destagger", "peak_source": src})
    line = {"metric": "destaggered cell*mode/s (fields moved to the primary grids)", "value": cells / (ms / 1e3),
            "unit": "cell*mode/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic (seeded Gaussian pulse)",
            "config": {"workload": w.name, "precision": prec, "l2": "flushed between timed calls (256 MiB write)"},
            "roofline": roof}
    print(json.dumps(line), flush=True)


def _time_calls(fn, steps, warmup, flush=True):
    """Mean CUDA-event time (ms) of fn() over `steps` calls after `warmup`, L2 flushed before each."""
    import torch
    buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if flush else None
    stream = torch.cuda.current_stream()
    for _ in range(max(warmup, 3)):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if buf is not None:
            buf.zero_()
        evs[k][0].record(stream)
        fn()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(x.elapsed_time(y) for x, y in evs) / steps


def run_envelope(args):
    """The envelope propagator (second entry point) on the 4096x256 envelope workload: term by term, with every
    term in one launch, and with an absorbing layer over the last eighth of the box."""
    import torch
    import paper_2605_12132_gb300 as fd
    from paper_2605_12132_gb300 import inputs
    ew = inputs.envelope_workload("envelope_4096x256")
    a, at, chi = inputs.envelope_inputs(ew)
    plan = fd.envelope_plan(ew.Nz, ew.Nr, ew.order, ew.taylor_order, ew.dz, ew.dr, ew.dt)
    psi = torch.from_numpy(np.stack([a, at])).to(torch.complex64).cuda()
    c = torch.from_numpy(chi).to(torch.float32).cuda()
    z = np.arange(ew.Nz) / ew.Nz
    sig = np.repeat((8.0 * np.clip((z - 0.875) / 0.125, 0, None) ** 2)[:, None], ew.Nr, axis=1)
    sigma = torch.from_numpy(sig).to(torch.float32).cuda()
    ms_plain = _time_calls(lambda: fd.envelope_step(plan, psi, c, 1), args.steps, args.warmup)
    ms_fused = _time_calls(lambda: fd.envelope_step_fused(plan, psi, c, 1), args.steps, args.warmup)
    ms_abs = _time_calls(lambda: fd.envelope_step_absorbing(plan, psi, c, sigma, 1), args.steps, args.warmup)
    cells = ew.Nz * ew.Nr
    # algorithmic bytes of one step: the state (a, a~) and chi read once, the state written once (36 B per cell)
    algo = cells * 36
    peaks, src = _peaks()
    best = min(ms_plain, ms_fused)
    ach = algo / (best / 1e3) / 1e9
    line = {"metric": "envelope cell*steps/s (exponential laser-envelope propagator, Taylor-N)",
            "value": cells / (best / 1e3), "unit": "cell*steps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (Gaussian envelope, seeded smooth chi)",
            "config": {"workload": ew.name, "taylor_order": ew.taylor_order, "order": ew.order,
                       "term_by_term_ms_per_step": ms_plain, "fused_ms_per_step": ms_fused,
                       "absorbing_layer_ms_per_step": ms_abs, "l2": "flushed between timed calls (256 MiB write)"},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "traffic": None, "algorithmic": algo,
                         "kernel": "envelope_term_kernel" if ms_plain <= ms_fused else "envelope_fused_kernel",
                         "peak_source": src}}
    print(json.dumps(line), flush=True)


def run_current(args, w):
    """The current pipeline (stagger, planar divergence error, banded Poisson solve, correction; one fused
    launch) on the field workload's grid with seeded deposited currents and densities."""
    import torch
    import paper_2605_12132_gb300 as fd
    prec = args.precision or "bf16x6"
    rng = np.random.default_rng(3)
    nm = len(w.modes)
    plan = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision=prec)
    dt_c = plan.complex_dtype
    J = torch.from_numpy(rng.standard_normal((nm, 3, w.Nz, w.Nr)) + 0j).to(dt_c).cuda()
    rho = torch.from_numpy(rng.standard_normal((nm, w.Nz, w.Nr)) + 0j).to(dt_c).cuda()
    out = torch.empty_like(J)
    ms = _time_calls(lambda: fd.fdetd_current_correct(plan, J, rho, out), args.steps, args.warmup)
    cells = w.Nz * w.Nr * nm
    # algorithmic bytes: J (3 components) and rho_xy read, the corrected J written
    algo = cells * 7 * J.element_size()
    peaks, src = _peaks()
    roof = {"bound": "hbm", "achieved": algo / (ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"traffic": None, "algorithmic": algo, "kernel": "current_kernel", "peak_source": src,
                 "note": "latency-bound: the banded solve is a serial recurrence over Nr per (mode, z row)"})
    line = {"metric": "current-corrected cell*mode/s (stagger + planar current correction)",
            "value": cells / (ms / 1e3), "unit": "cell*mode/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32 data / double-float solve",
            "data": "synthetic (seeded random deposited current and density)",
            "config": {"workload": w.name, "precision": prec, "launches": 1,
                       "l2": "flushed between timed calls (256 MiB write)"},
            "roofline": roof}
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Poisson stream of field- and envelope-advance requests (50/50) through the library's continuous-batching
    server: field requests drawn from the uneven mix with 10-500 steps, envelope requests on the 4096x256 envelope
    workload with 10-500 steps.  Arrivals run for --duration seconds at --rate per second; completions are collected
    for --drain more seconds, then the requests still waiting for admission are cancelled and the admitted ones
    finish.  Reports the served throughput over the whole window, the latency percentiles of the completed
    requests, and how many were still waiting (queue growth when the stream is over capacity)."""
    import torch
    from paper_2605_12132_gb300 import inputs, serve
    prec = args.precision or "bf16x6"
    pool = inputs.uneven_instances(32, seed=5)
    pool_arrays = [inputs.instance_inputs(c) for c in pool]
    pool_arrays = [(F.astype(np.complex64), J.astype(np.complex64)) for F, J in pool_arrays]
    ew = inputs.envelope_workload("envelope_4096x256")
    ea, eat, echi = inputs.envelope_inputs(ew)
    env_state = np.stack([ea, eat]).astype(np.complex64)
    env_chi = echi.astype(np.float32)

    def field_request(k, steps):
        c = pool[k]
        F, J = pool_arrays[k]
        return serve.FieldRequest(c["Nz"], c["Nr"], list(range(c["M"] + 1)), c["order"], 1 / 16, 1 / 4, 1 / 16,
                                  steps, F, J, prec)

    def make(i, rng):
        if rng.random() < 0.5:
            k = int(rng.integers(len(pool)))
            return field_request(k, int(rng.integers(10, 501)))
        return serve.EnvelopeRequest(ew.Nz, ew.Nr, ew.order, ew.taylor_order, ew.dz, ew.dr, ew.dt,
                                     int(rng.integers(10, 501)), env_state, env_chi)

    free, total = torch.cuda.mem_get_info()
    budget = int(0.6 * free)
    srv = serve.Server(budget, chunk_steps=32, plan_workers=8)
    warm_s, warm_tables = None, 0
    if args.prewarm:
        # the radial tables of the pool's grids computed before the arrival window (a server that knows the
        # grids it serves); the plans themselves are still built per request
        tw = time.perf_counter()
        warm_tables = srv.prewarm([field_request(k, 1) for k in range(len(pool))], workers=16)
        warm_s = time.perf_counter() - tw
    t0 = time.perf_counter()
    tickets = serve.run_poisson(srv, make, args.rate, args.duration, seed=11, keep_result=False)
    arrive_end = time.perf_counter()
    deadline = arrive_end + args.drain
    while time.perf_counter() < deadline:
        s = srv.stats()
        if s["queued"] + s["building"] + s["running"] == 0:
            break
        time.sleep(0.05)
    window = time.perf_counter() - t0
    st_window = srv.stats()
    served_in_window = st_window["served_cell_steps"]
    waiting = srv.cancel_queued()
    srv.close()
    wall = time.perf_counter() - t0
    st = serve.latency_stats(tickets)
    done = [t for t in tickets if t.state == serve.DONE]
    line = {"metric": "served cell*mode*steps/s and request latency (continuous batching)",
            "value": served_in_window / window, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "latency": st, "requests": len(tickets), "completed": len(done), "cancelled_waiting": waiting,
            "rate_hz": args.rate, "duration_s": args.duration, "window_s": window, "wall_s": wall,
            "hbm_budget_bytes": budget, "peak_admitted_bytes": st_window["peak_bytes"],
            "recaptures": st_window["recaptures"], "prewarm": {"tables": warm_tables, "seconds": warm_s},
            "config": {"workload": "Poisson 50/50 mix of field requests (uneven sizes, 10-500 steps) and 4096x256 "
                                   "envelope requests (10-500 steps)", "precision": prec, "chunk_steps": 32}}
    print(json.dumps(line), flush=True)


def run_step(args, w, prec, leg=False, dist=None, rank=0, world=1):
    """One instance of workload w stepped through fdetd_step, L2 flushed between timed steps.  As a leg of
    the default line it returns a summary dict; with --mode step it prints the full line."""
    import torch
    import paper_2605_12132_gb300 as fd
    from paper_2605_12132_gb300 import inputs

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    F, J = inputs.workload_inputs(w)
    plan = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision=prec)
    cdt = plan.complex_dtype
    fields = torch.from_numpy(F).to(cdt).cuda()
    Jd = torch.from_numpy(J).to(cdt).cuda() if J is not None else None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    tiles = tuned = None
    if prec in ("bf16x3", "bf16x6"):
        tuned = plan.autotune(fields, Jd)       # tile shapes / schedules, timed on these arrays (read only)
        tiles = dict(zip(("tn_proj", "tn_back", "sched_proj", "sched_back"), plan.tile_config))
    # one step from the initial state for the accuracy check, then the warm-up steps
    fd.fdetd_step(plan, fields, Jd, 1)
    torch.cuda.synchronize()
    one_step = fields.clone()
    for _ in range(args.warmup - 1):
        fd.fdetd_step(plan, fields, Jd, 1)
    barrier()
    steps = args.steps if not leg else min(args.steps, 10)
    clocks = ClockSampler()
    if not leg:
        clocks.start()
    plan.set_profiling(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    t_wall = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        fd.fdetd_step(plan, fields, Jd, 1)
        evs[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = None if leg else clocks.stop()
    ktimes = plan.kernel_times()
    pipeline = _rounded(plan.pipeline_waits()) if prec in ("bf16x3", "bf16x6") else None
    plan.set_profiling(False)
    plan.status()
    lat = np.array([a.elapsed_time(b) for a, b in evs])
    ms = max_over_ranks(float(lat.sum()), dist, "cuda")
    cells = w.Nz * w.Nr * len(w.modes)
    value = replica_rate(cells * steps, ms / 1e3, world)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in ktimes.items()}

    # FP64 single-instance path on the same workload: its rate, the error of one step from the same state, and
    # (where FP64 steps take milliseconds, Nz <= 4096) the error after 100 steps, which shows the drift of the
    # per-step error
    fp64_value = err = err100 = None
    if not args.no_fp64 and prec != "fp64":
        p64 = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision="fp64")
        f64 = torch.from_numpy(F).cuda()
        J64 = torch.from_numpy(J).cuda() if J is not None else None
        fd.fdetd_step(p64, f64, J64, 1)
        barrier()
        strong, weak = _field_error_stats(torch, one_step, f64)
        err = {"strong_fields_max": strong, "weak_fields_max": weak}
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n64 = 2
        a.record(stream)
        fd.fdetd_step(p64, f64, J64, n64)
        b.record(stream)
        barrier()
        fp64_value = cells * n64 / (a.elapsed_time(b) / 1e3)
        if w.Nz <= 4096:
            n_long = 100
            fl = torch.from_numpy(F).to(cdt).cuda()
            fd.fdetd_step(plan, fl, Jd, n_long)
            f64 = torch.from_numpy(F).cuda()
            fd.fdetd_step(p64, f64, J64, n_long)
            barrier()
            plan.status()
            strong, weak = _field_error_stats(torch, fl, f64)
            err100 = {"steps": n_long, "strong_fields_max": strong, "weak_fields_max": weak}
            del fl
        p64.close()
        del f64, J64

    summary = {"workload": w.name, "Nz": w.Nz, "Nr": w.Nr, "modes": w.modes, "order": w.order, "precision": prec,
               "steps": steps, "ms_per_step": ms / steps, "value": value, "stage_ms_per_step": stage_ms,
               "fp64_value": fp64_value, "rel_err_vs_fp64_1step": err, "rel_err_vs_fp64_100steps": err100,
               "tiles": tiles, "pipeline": pipeline,
               "l2": "flushed between timed steps (256 MiB write)"}
    launches = plan.launches_per_step * steps
    plan.close()
    if leg:
        return summary

    # end-to-end through the host entry point: h2d of fields + J, the step, d2h of the fields
    plan = fd.fdetd_plan_modes(w.Nz, w.Nr, w.modes, w.order, w.dz, w.dr, w.dt, precision=prec)
    hf = torch.from_numpy(F).to(cdt).pin_memory()
    hJ = torch.from_numpy(J).to(cdt).pin_memory() if J is not None else None
    fd.fdetd_step_host(plan, hf, hJ, 1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        fd.fdetd_step_host(plan, hf, hJ, 1)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    elt = hf.element_size()
    h2d = hf.numel() * elt + (hJ.numel() * elt if hJ is not None else 0)
    d2h = hf.numel() * elt
    e2e_val = replica_rate(cells * args.e2e_steps, e2e_s, world)
    plan.close()

    peaks, src = _peaks()
    hasJ = J is not None
    fwd_flops, bwd_flops = gemm_flops(w, hasJ)
    elt_c = 16 if prec == "fp64" else 8
    dom = max(stage_ms, key=stage_ms.get)
    per_launch_s = stage_ms[dom] / 1e3
    products = {"bf16x3": 3, "bf16x6": 6}.get(prec, 1)
    if dom == "spectral":
        algo = spectral_bytes(w, hasJ, elt_c)
        roof = {"bound": "hbm", "achieved": algo / per_launch_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    else:
        algo = fwd_flops if dom == "projection" else bwd_flops
        if prec in ("bf16x3", "bf16x6"):
            roof = {"bound": "tensor", "achieved": algo * products / per_launch_s / 1e12,
                    "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s"}
        else:
            # CUDA-core FMA peak: 152 SMs x 128 FP32 lanes (FP64: nominal 1.25 TFLOP/s) x 2 flops x max clock
            pk = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12 if prec == "fp32" else 1.25
            roof = {"bound": "alu", "achieved": algo / per_launch_s / 1e12, "peak": pk, "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = recorded_traffic(dom, w.name, prec)
    roof["algorithmic"] = algo
    roof["kernel"] = dom
    roof["peak_source"] = src
    roof["stage_ms_per_step"] = stage_ms
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs = cpu_oracle_rate(w, F, J, 4)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"4 kz columns ({4 * w.Nr} cells) of mode {w.modes[-1]}, one step, per-kz dense "
                         f"eigendecomposition evaluator, FP64 ({secs:.1f} s)"}
    if rank == 0:
        summary.update({"parallelism": "replicas" if world > 1 else "single", "wall_s": t_wall, "autotune_ms": tuned})
        line = {"metric": STEP_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32"}.get(prec, prec + "-split/f32-accumulate"),
                "data": "synthetic (seeded Gaussian pulse + seeded smooth random current)", "config": summary,
                "latency": {"unit": "ms per step", "p50": float(np.percentile(lat, 50)),
                            "p99": float(np.percentile(lat, 99))},
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--workload", default="lwfa_m01_2048x256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-legs", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--mode", default="batch",
                    choices=["batch", "step", "serve", "taylor", "destagger", "envelope", "current"])
    ap.add_argument("--taylor-order", type=int, default=4)
    ap.add_argument("--substeps", type=int, default=1)
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--drain", type=float, default=30.0)
    ap.add_argument("--prewarm", action="store_true", help="serve mode: radial tables of the pool computed first")
    ap.add_argument("--host-parts", type=int, default=16, help="batch mode: parts of the host-buffer step")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2605_12132_gb300 import inputs
    w = inputs.workload(args.workload)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "taylor":
        return run_taylor(args, w)
    if args.mode == "destagger":
        return run_destagger(args, w)
    if args.mode == "envelope":
        return run_envelope(args)
    if args.mode == "current":
        return run_current(args, w)

    import torch
    import paper_2605_12132_gb300 as fd
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.precision is None:
        # the split-BF16 precision that stays within 1e-6 relative per step on the strong fields (BF16x3: ~1e-5)
        args.precision = "bf16x6"
        try:
            fd.fdetd_plan_modes(64, 16, [0], 4, 0.1, 0.1, 0.1, precision="bf16x6").close()
        except fd.FdetdError:
            args.precision = "fp32"
    if args.mode == "batch":
        run_batch(args, rank, world, dist)
    else:
        run_step(args, w, args.precision, dist=dist, rank=rank, world=world)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
