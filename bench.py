#!/usr/bin/env python
"""Throughput benchmark of guided walk on stars on GB300.

Workload (one "step" = one full solve, every hot-path stage included):
2D Poisson/Laplace with mixed boundary conditions -- a seeded star-shaped
polyline of 4096 segments (r = 1 + 0.3 sum of 5 Fourier modes), a contiguous
zero-flux Neumann arc on 40% of it, Dirichlet data x^2 - y^2 elsewhere; a
512 x 512 grid over the bounding box masked to the interior; 32 walks per
point in 32 batches of one walk per point; guided sampling from the hash-grid
+ MLP vMF mixture field with learnable MIS selection, trained after every
batch (fused tcgen05 backward + Adam); eps = 1e-3, at most 128 steps per walk.

Metric: walk-steps/s (loop iterations of all walks, terminal step included),
whole job over all ranks.  Timed with CUDA events on the launching stream;
the L2 cache is flushed (a 512 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica (own field and seed): the
walks partition without any data-path exchange ("scaling": "weak").
--impl reference times the CPU FP64 oracle (the test checker) on a bounded
sample of the same workload on the host cores.
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "walk-steps/s and equal-time relMSE: guided vs plain WoSt on one GB300"
UNIT = "walk-steps/s"
WORKLOAD = dict(workload="2D mixed Dirichlet/Neumann guided WoSt: star polyline 4096 segments, 40% zero-flux "
                         "Neumann arc, g = x^2 - y^2, 512x512 grid masked inside, 32 walks/point, online training "
                         "after every batch, 16-level 2^16-entry FP16 hash grid + 32-64-64-33 BF16 MLP, K = 8",
                nseg=4096, grid=512, spp=32, eps=1e-3, maxsteps=128, l2="flushed (512 MiB write) before each step")


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def make_workload(res=512):
    import wost_inputs as wi
    sc, pts = wi.config_star_guided(res=res)
    return sc, pts


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def combine_ranks(total_ms, steps_local, device=None):
    """Whole-job figures over all ranks: the slowest rank's timed span (MAX)
    and the walk-steps of all ranks (SUM).  Single process: unchanged."""
    try:
        import torch
        import torch.distributed as dist
    except ImportError:
        return float(total_ms), float(steps_local)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(steps_local)
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(steps_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t[0]), float(n[0])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_rate(sc, pts, field_params, seconds=12.0, seed=3, guided=True):
    """Walk-steps/s of the FP64 oracle on the host cores: guided walks (field
    frozen at the given parameters) over a seeded subsample of the points,
    repeated until about `seconds` of CPU time has been spent."""
    import oracle
    import wost_inputs as wi
    nth = os.cpu_count() or 1
    O = oracle.Scene(sc)
    OF = oracle.Field(oracle.FieldParams(**field_params)) if guided else None
    prm = oracle.make_params(eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"], guided=int(guided), seed=seed,
                             nthreads=nth)
    sample = wi.subsample(pts, 4 * nth * 16, seed=1)
    steps = 0
    walks = 0
    t0 = time.perf_counter()
    w = 0
    while time.perf_counter() - t0 < seconds:
        r = oracle.solve(O, prm, sample, w, 1, field=OF)
        steps += r["steps"]
        walks += len(sample)
        w += 1
    dt = time.perf_counter() - t0
    return steps / dt, dict(cores=nth, sample=f"{len(sample)} seeded grid points x {w} walks ({walks} walks, "
                                               f"{steps} walk-steps, {dt:.1f} s) of the same scene, guided with "
                                               f"the initial field frozen (no training step)")


def field_params_dict(F, lo, hi):
    import wost_inputs as wi
    p = F.get_params()
    d = F.desc
    return dict(dim=2, K=d.K, L=d.levels, log2T=d.log2_table, F=d.features, H=d.hidden, base_res=d.base_res,
                max_res=d.max_res, lo=np.asarray(lo, float), hi=np.asarray(hi, float),
                grid=wi.round_to_fp16(p["grid"]), W1=wi.round_to_bf16(p["W1"]), W2=wi.round_to_bf16(p["W2"]),
                W3=wi.round_to_bf16(p["W3"]), b3=p["b3"].astype(float))


# ---------------------------------------------------------------------------
# reference arm: the oracle, timed as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import wost_inputs as wi
    sc, pts = make_workload()
    # the field the oracle walks with: the library's default initialisation
    # is not available without a GPU, so use a seeded field of the same shape
    lo, hi = sc.padded_bbox()
    fp = wi.random_field_params(2, 1, lo, hi, grid_scale=1e-4, w_scale=1.0)
    per = []
    info = None
    for i in range(args.warmup + args.steps):
        rate, info = oracle_rate(sc, pts, fp, seconds=args.ref_seconds, seed=10 + i)
        if i >= args.warmup:
            per.append(rate)
    value = statistics.mean(per)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * args.ref_seconds, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, reference_sample=info["sample"]), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    from paper_2410_18944_gb300 import api, build
    if rank == 0:
        build.build()
    barrier()
    sc, pts_np = make_workload()
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(2, lo, hi, seed=1 + rank)
    init = F.get_params()
    pts = torch.tensor(pts_np, dtype=torch.float64, device=dev)
    npts = len(pts_np)
    stream = torch.cuda.current_stream()
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)   # 512 MiB > L2
    kw = dict(eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"], guided=True, field=F, train=1,
              train_until_wpp=256, stream=stream)

    def one_step(i, timed_events=None):
        F.set_params(init["grid"], init["W1"], init["W2"], init["W3"], init["b3"])   # fresh field every step
        flush.zero_()
        torch.cuda.synchronize()
        if timed_events is not None:
            timed_events[0].record(stream)
        m, v, st = api.solve(S, pts, WORKLOAD["spp"], seed=1000 * rank + i, **kw)
        if timed_events is not None:
            timed_events[1].record(stream)
        last_mean[0] = m
        return st

    last_mean = [None]

    for i in range(args.warmup):
        one_step(i)
    torch.cuda.synchronize()
    barrier()
    per_ms, stats = [], []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            st = one_step(args.warmup + i, ev)
            torch.cuda.synchronize()
            per_ms.append(ev[0].elapsed_time(ev[1]))
            stats.append(st)
    barrier()
    steps_local = sum(s["walk_steps"] for s in stats)
    total_ms, steps_all = combine_ranks(sum(per_ms), steps_local, dev)
    value = steps_all / (total_ms / 1000.0)

    # end to end through the C ABI with host buffers (pinned points and
    # outputs; H2D of the points and D2H of mean and variance inside)
    pts_host = torch.tensor(pts_np, dtype=torch.float64).pin_memory()
    e2e_steps, e2e_s = 0, 0.0
    for i in range(max(1, min(args.steps, 3))):
        F.set_params(init["grid"], init["W1"], init["W2"], init["W3"], init["b3"])
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m, v, st = api.solve(S, pts_host.numpy(), WORKLOAD["spp"], seed=7000 + i, eps=WORKLOAD["eps"],
                             maxsteps=WORKLOAD["maxsteps"], guided=True, field=F, train=1, train_until_wpp=256)
        e2e_s += time.perf_counter() - t0
        e2e_steps += st["walk_steps"]
    e2e_value = world * e2e_steps / e2e_s

    if rank != 0:
        return 0

    # plain WoSt on the same workload (same grid, spp), for context
    mp, vp, stp = api.solve(S, pts, WORKLOAD["spp"], seed=99, eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"],
                            stream=stream)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    flush.zero_()
    torch.cuda.synchronize()
    ev[0].record(stream)
    mp, vp, stp = api.solve(S, pts, WORKLOAD["spp"], seed=98, eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"],
                            stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    plain_rate = stp["walk_steps"] / (ev[0].elapsed_time(ev[1]) / 1000.0)

    # the tensor-core decode on its own: 4 Mi positions through
    # wost_field_decode (hash-grid encode + three tcgen05 BF16 MMAs per
    # 128-row tile), device buffers, CUDA events on the stream
    ndec = 1 << 22
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    lo_t = torch.tensor(lo, dtype=torch.float64, device=dev)
    hi_t = torch.tensor(hi, dtype=torch.float64, device=dev)
    dec_pts = lo_t + (hi_t - lo_t) * torch.rand((ndec, 2), dtype=torch.float64, device=dev, generator=g)
    dec_out = torch.empty((ndec, F.nout), dtype=torch.float32, device=dev)
    for _ in range(2):
        F.decode(dec_pts, out=dec_out, exec_=api.exec_defaults(stream=stream))
    flush.zero_()
    torch.cuda.synchronize()
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev[0].record(stream)
    F.decode(dec_pts, out=dec_out, exec_=api.exec_defaults(stream=stream))
    ev[1].record(stream)
    torch.cuda.synchronize()
    dec_s = ev[0].elapsed_time(ev[1]) / 1000.0
    flop_per = 2.0 * (32 * 64 + 64 * 64 + 64 * 48)       # padded output width 48
    bf16_peak = measured_peaks().get("bf16_tflops")
    dec_tflops = ndec * flop_per / dec_s / 1e12
    decode = {"points": ndec, "ms": dec_s * 1e3, "decodes_per_s": ndec / dec_s, "bound": "tensor",
              "achieved_tflops": dec_tflops, "peak_tflops": bf16_peak or 1900.0,
              "frac": dec_tflops / (bf16_peak or 1900.0),
              "peak_source": "measured" if bf16_peak else "fallback",
              "note": "per point 18.4 kFLOP of BF16 MMA against 64 hash-grid corner gathers (L2): "
                      "the encode gathers, not the tensor pipe, set the decode time"}

    # equal-time relMSE (guided with training vs plain), against a plain
    # reference at 16x the walks per point; relMSE = mean (u^ - u)^2 / (u^2 + 1e-2)
    relmse = None
    if not args.no_relmse:
        guided_mean = last_mean[0].cpu().numpy()
        spp_ref = 16 * WORKLOAD["spp"]
        ref, _, _ = api.solve(S, pts, spp_ref, seed=424242, eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"],
                              stream=stream)
        ref = ref.cpu().numpy()

        def rel(u):
            return float(np.mean((u - ref) ** 2 / (ref ** 2 + 1e-2)))
        t32 = stp["walk_steps"] / plain_rate          # seconds for 32 plain walks per point
        guided_s = total_ms / args.steps / 1000.0
        spp_eq = max(1, int(WORKLOAD["spp"] * guided_s / t32))
        mp_eq, _, _ = api.solve(S, pts, spp_eq, seed=515151, eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"],
                                stream=stream)
        r_g, r_pe, r_ps = rel(guided_mean), rel(mp_eq.cpu().numpy()), rel(mp.cpu().numpy())
        relmse = {"guided": r_g, "plain_equal_time": r_pe, "plain_equal_spp": r_ps, "plain_spp_at_equal_time": spp_eq,
                  "equal_time_ratio_plain_over_guided": r_pe / r_g, "reference": f"plain WoSt, {spp_ref} walks/point",
                  "guided_s_per_solve": guided_s}

    # roofline of the dominant kernel (the guided walk kernel): algorithmic
    # bytes per launch over its average launch time (library CUDA events on
    # the same stream, summed over the timed steps)
    walk_ms = sum(s["ms_walk"] for s in stats)
    train_ms = sum(s["ms_train"] for s in stats)
    walk_launches = sum(s["walk_launches"] for s in stats)
    alg = sum(s["alg_bytes"] for s in stats)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = (alg / walk_launches) / ((walk_ms / walk_launches) / 1000.0) / 1e9
    traffic = args.traffic
    if traffic is None:
        # DRAM bytes per walk-step of the walk kernel from its ncu capture,
        # scaled to this run's walk-steps per launch
        try:
            tr = json.load(open(os.path.join(ROOT, "profiles", "guided_walk_traffic.json")))
            traffic = tr["dram_bytes_per_walk_step"] * sum(s["walk_steps"] for s in stats) / walk_launches
        except (OSError, ValueError, KeyError):
            traffic = None
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": "guided_walk_kernel<2>", "peak_source": peak_src,
            "alg_bytes_per_walk_step": alg / sum(s["walk_steps"] for s in stats)}

    cpu_rate, cpu_info = (None, {})
    if not args.no_cpu_baseline:
        cpu_rate, cpu_info = oracle_rate(sc, pts_np, field_params_dict(F, lo, hi), seconds=args.cpu_seconds)

    launches = sum(s["kernel_launches"] for s in stats) // len(stats)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 geometry, bf16 MLP, f64 accumulators",
            "data": "synthetic", "config": dict(WORKLOAD, points=npts, parallelism=f"replicas x{world}"),
            "clocks": clk.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(npts * 2 * 8),
                    "d2h_bytes_per_step": int(npts * 2 * 8)},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": ({"value": cpu_rate, "unit": UNIT, "cores": cpu_info.get("cores"), "kind": "oracle",
                              "sample": cpu_info.get("sample")} if cpu_rate else None),
            "breakdown": {"walk_ms_per_step": walk_ms / len(stats), "train_ms_per_step": train_ms / len(stats),
                          "walk_steps_per_step": steps_local / len(stats),
                          "records_per_step": sum(s["records"] for s in stats) / len(stats)},
            "plain_walk_steps_per_s": plain_rate,
            "decode": decode,
            "relmse": relmse}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = {
    "sphere3d": dict(workload="3D mixed Dirichlet/Neumann Poisson guided WoSt: icosphere 81,920 triangles displaced "
                              "by 0.15 Perlin noise, 30% Neumann cap, f = 4 Gaussians (sigma 0.1), g = 1/|x - c|, "
                              "256x256 slice z = 0 masked inside, 64 walks/point, online training after every batch "
                              "in minibatches of 2^18 records, 16-level 2^19-entry FP16 hash grid + 32-64-64-41 BF16 "
                              "MLP, K = 8",
                     grid=256, spp=64, eps=1e-3, maxsteps=128, train_samples=1 << 18,
                     l2="flushed (512 MiB write) before each step"),
    "genus3": dict(workload="3D mixed Dirichlet/Neumann Laplace guided WoSt with learned MIS selection: genus-3 "
                            "solid (sphere displaced by 0.15 Perlin noise minus three smoothly rimmed tunnels, "
                            "993,640 triangles by surface nets), 30% Neumann cap, g = 1/|x - c|, 1024x1024 slice "
                            "z = 0 masked inside, 128 walks/point, online training after every batch in minibatches "
                            "of 2^18 records, 16-level 2^19-entry FP16 hash grid + 32-64-64-41 BF16 MLP, K = 8",
                   grid=1024, spp=128, eps=1e-3, maxsteps=128, train_samples=1 << 18,
                   l2="inputs larger than L2 (the BVHs and 1 M-walk batches); no flush"),
    "batch64": dict(workload="64 independent 2D star scenes (256-16384 segments log-uniform, Neumann fraction "
                             "U(0.2, 0.5), 1k-256k points and 8-128 walks per point log-uniform), one persistent "
                             "launch per training round under a CUDA graph, guided with online training per scene "
                             "(and the plain batch for comparison)",
                    scenes=64, eps=1e-3, maxsteps=128, l2="flushed (512 MiB write) before each step"),
}


def run_workload_3d(args, W, api, wi, torch, dev, flush, stream):
    """A 3D workload line: guided solves with online training (fresh field
    each), the plain solve of the same size, and equal-time relMSE on a
    seeded 4096-point subset against a plain reference at 64x the walks per
    point (the oracle's brute-force geometry cannot reach a low-variance
    reference on these meshes)."""
    if args.workload == "sphere3d":
        sc, pts_np = wi.config_3d_guided(res=W["grid"])
    else:
        sc, pts_np = wi.config_genus3(res=W["grid"])
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(3, lo, hi, seed=1)
    init = F.get_params()
    pts = torch.tensor(pts_np, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(7)
    sub = np.sort(rng.choice(len(pts_np), min(4096, len(pts_np)), replace=False))
    sub_t = torch.tensor(sub, device=dev)
    psub = pts[sub_t].contiguous()
    common = dict(eps=W["eps"], maxsteps=W["maxsteps"], stream=stream)

    def timed(fn):
        flush.zero_()
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        out = fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), out

    def guided(p, spp, seed):
        F.set_params(init["grid"], init["W1"], init["W2"], init["W3"], init["b3"])
        return api.solve(S, p, spp, seed=seed, guided=True, field=F, train=1, train_until_wpp=256,
                         train_samples=W.get("train_samples", 0), **common)

    big = W["spp"] * len(pts_np) > 20_000_000
    steps = 1 if big else args.steps
    # warm-up: full solves for the small workload, a 16k-point subset of the large one
    wp = pts[:16384].contiguous() if big else pts
    for i in range(args.warmup):
        guided(wp, 2 if big else W["spp"], i)
        api.solve(S, wp, 2 if big else W["spp"], seed=50 + i, **common)
    ms_g, nsteps, stats = 0.0, 0, []
    for i in range(steps):
        t, (mg, _, st) = timed(lambda: guided(pts, W["spp"], 100 + i))
        ms_g += t
        nsteps += st["walk_steps"]
        stats.append(st)
    ms_p, (mp, _, stp) = timed(lambda: api.solve(S, pts, W["spp"], seed=999, **common))
    guided_s = ms_g / steps / 1000.0
    plain_s = ms_p / 1000.0
    spp_ref = 64 * W["spp"]
    ref = api.solve(S, psub, spp_ref, seed=424242, **common)[0].cpu().numpy()
    spp_eq = max(1, int(W["spp"] * guided_s / plain_s))
    mpe = api.solve(S, psub, spp_eq, seed=515151, **common)[0].cpu().numpy()

    def rel(u):
        return float(np.mean((u - ref) ** 2 / (ref ** 2 + 1e-2)))
    r_g = rel(mg[sub_t].cpu().numpy())
    r_ps = rel(mp[sub_t].cpu().numpy())
    r_pe = rel(mpe)
    line = {"metric": METRIC, "value": nsteps / (ms_g / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms_g / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 geometry, bf16 MLP, f64 accumulators", "data": "synthetic",
            "config": dict(W, points=len(pts_np), warmup_points=len(wp)),
            "plain_walk_steps_per_s": stp["walk_steps"] / plain_s,
            "breakdown": {"walk_ms": sum(s["ms_walk"] for s in stats) / steps,
                          "train_ms": sum(s["ms_train"] for s in stats) / steps,
                          "train_steps": stats[-1]["train_steps"], "records_last_batch": stats[-1]["records"]},
            "relmse": {"guided": r_g, "plain_equal_spp": r_ps, "plain_equal_time": r_pe,
                       "plain_spp_at_equal_time": spp_eq, "equal_time_ratio_plain_over_guided": r_pe / r_g,
                       "subset_points": len(sub), "reference": f"plain WoSt, {spp_ref} walks/point on the subset",
                       "guided_s_per_solve": guided_s, "plain_s_per_solve": plain_s}}
    print(json.dumps(line), flush=True)
    return 0


def run_workload(args):
    """Other workloads of the method (same metric and timing rules), for the
    design notes: --workload sphere3d | genus3 | batch64 on one GPU."""
    import torch
    import wost_inputs as wi
    from paper_2410_18944_gb300 import api, build
    build.build()
    W = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    extra = {}
    if args.workload in ("sphere3d", "genus3"):
        return run_workload_3d(args, W, api, wi, torch, dev, flush, stream)
    else:
        jobs = wi.config_batch()
        scenes = [api.Scene(j.scene) for j in jobs]
        pts = [torch.tensor(j.points, dtype=torch.float64, device=dev) for j in jobs]
        plans = {}
        for guided in (True, False):
            specs = []
            for i, j in enumerate(jobs):
                d = dict(scene=scenes[i], points=pts[i], nwalks=j.nwalks, seed=j.seed, eps=W["eps"],
                         maxsteps=W["maxsteps"])
                if guided:
                    lo, hi = scenes[i].bbox()
                    d["field"] = api.Field(2, lo, hi, seed=1 + i)
                specs.append(d)
            plans[guided] = api.Batch(specs, guided=guided, train=1 if guided else 0)
        extra["plan"] = {("guided" if g else "plain"): p.info() for g, p in plans.items()}
        extra["points"] = sum(len(j.points) for j in jobs)
        extra["walks"] = sum(len(j.points) * j.nwalks for j in jobs)

        def solve(i, guided=True):
            flush.zero_()
            torch.cuda.synchronize()
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(stream)
            st = plans[guided].run(stream.cuda_stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]), st["walk_steps"]
    for i in range(args.warmup):
        solve(i)
    ms, steps = 0.0, 0
    for i in range(args.steps):
        t, n = solve(100 + i)
        ms += t
        steps += n
    pms, psteps = solve(999, guided=False)
    line = {"metric": METRIC, "value": steps / (ms / 1000.0), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 geometry, bf16 MLP, f64 accumulators", "data": "synthetic",
            "config": dict(W, **extra), "plain_walk_steps_per_s": psteps / (pms / 1000.0)}
    print(json.dumps(line), flush=True)
    return 0


def run_once(args):
    """One solve of (a seeded subset of) a workload, for profilers: no
    timing loop, no oracle.  --once plain|guided, --points N, --spp S,
    --workload star2d|sphere3d|genus3."""
    import torch
    import wost_inputs as wi
    from paper_2410_18944_gb300 import api, build
    build.build()
    dim = 2
    if args.workload == "sphere3d":
        sc, pts = wi.config_3d_guided(res=WORKLOADS["sphere3d"]["grid"])
        dim = 3
    elif args.workload == "genus3":
        sc, pts = wi.config_genus3(res=WORKLOADS["genus3"]["grid"])
        dim = 3
    else:
        sc, pts = make_workload()
    if args.points and args.points < len(pts):
        pts = wi.subsample(pts, args.points, seed=1)
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(dim, lo, hi)
    p = torch.tensor(pts, dtype=torch.float64, device="cuda")
    guided = args.once == "guided"
    ts = WORKLOADS.get(args.workload, {}).get("train_samples", 0)
    for rep in range(2):
        m, v, st = api.solve(S, p, args.spp, eps=WORKLOAD["eps"], maxsteps=WORKLOAD["maxsteps"], seed=rep,
                             guided=guided, field=F if guided else None, train=1 if guided else 0,
                             train_samples=ts if guided else 0)
        torch.cuda.synchronize()
        print(json.dumps({"once": args.once, "rep": rep, **{k: st[k] for k in (
            "walk_steps", "ms_walk", "ms_train", "node_visits", "prim_visits", "kernel_launches", "records")}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["star2d", *WORKLOADS], default="star2d",
                    help="star2d (the benchmark line) or another workload of the method")
    ap.add_argument("--once", choices=["plain", "guided"], default=None,
                    help="run one solve of the workload (profiling), no timing")
    ap.add_argument("--points", type=int, default=0, help="with --once: seeded subset of the query points")
    ap.add_argument("--spp", type=int, default=WORKLOAD["spp"], help="with --once: walks per point")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-relmse", action="store_true", help="skip the equal-time relMSE measurement")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the guided walk kernel from an ncu capture")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.once:
        return run_once(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "star2d":
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
