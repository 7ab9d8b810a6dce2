#!/usr/bin/env python
"""Throughput benchmark of guided walk on stars on GB300.

Headline workload (the largest single-GPU configuration): 3D Laplace with
mixed Dirichlet / zero-flux Neumann boundary on a seeded genus-3 solid -- a
sphere displaced by 0.15 Perlin noise minus three smoothly rimmed tunnels,
993,640 triangles by surface nets -- with a 30% Neumann cap and Dirichlet
data g = 1/|x - c|; queries on the 1024 x 1024 slice z = 0 masked inside
(510,479 points) at 128 walks per point; guided sampling from the 3D
hash-grid + MLP vMF mixture field with learned MIS selection, trained online
after every batch of two walks per point in minibatches of 2^18 records
(fused tcgen05 backward + Adam).  The paper trains after batches of one walk
per point of a 1024 x 1024 grid, about 2^20 walks; the slice keeps half of
its points inside the solid, so two walks per point make a batch of that
size (1.02 M walks).

One "step" is one training round of the full slice: two walks per point
(1,020,958 walks, every hot-path stage) followed by that batch's Adam steps.
W rounds warm up, K rounds are timed (CUDA events on the launching stream),
and the remaining rounds of the 128-walk solve run untimed to complete the
estimate for the equal-time relMSE.  The BVHs (about 300 MB) and the
batches are larger than L2, so no flush is needed.

Metric: walk-steps/s (loop iterations of all walks, terminal step included),
whole job over all ranks.  The line also carries the equal-time relMSE of
guided vs plain WoSt on a seeded 4096-point subset, and extra lines for the
2D star (4096 segments, 512 x 512 grid, 32 walks/point), the 81,920-triangle
icosphere with Gaussian sources (256 x 256 slice, 64 walks/point) and 64
uneven 2D scenes in one persistent launch per round under a CUDA graph.  The
star and the icosphere have far fewer points than the slice, so their
training batches hold 4 and 8 walks per point (696k and 376k walks; the
sizes measured best at equal time) and a step of theirs is one such batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica (own field and seed): the
walks partition without any data-path exchange ("scaling": "weak").
--impl reference times the CPU FP64 oracle (the test checker) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
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
DTYPE = "f32 geometry, bf16 MLP, f64 accumulators"

WORKLOADS = {
    "genus3": dict(workload="3D mixed Dirichlet/Neumann Laplace guided WoSt with learned MIS selection: genus-3 "
                            "solid (sphere displaced by 0.15 Perlin noise minus three smoothly rimmed tunnels, "
                            "993,640 triangles by surface nets), 30% Neumann cap, g = 1/|x - c|, 1024x1024 slice "
                            "z = 0 masked inside, 128 walks/point, online training after every batch of two walks per point "
                            "(1.02 M walks, the paper's 2^20-walk batch) in minibatches "
                            "of 2^18 records, 16-level 2^19-entry FP16 hash grid + 32-64-64-41 BF16 MLP, K = 8",
                   dim=3, grid=1024, spp=128, eps=1e-3, maxsteps=128, train_samples=1 << 18, subset=4096,
                   ref_factor=64, batch_wpp=2,
                   step="one training batch: two walks per point of the slice (1.02M walks) + its Adam steps",
                   l2="inputs larger than L2 (about 300 MB of BVH, 1.02M-walk batches); no flush"),
    "sphere3d": dict(workload="3D mixed Dirichlet/Neumann Poisson guided WoSt: icosphere 81,920 triangles displaced "
                              "by 0.15 Perlin noise, 30% Neumann cap, f = 4 Gaussians (sigma 0.1), g = 1/|x - c|, "
                              "256x256 slice z = 0 masked inside, 64 walks/point, online training after every batch "
                              "of 8 walks per point in minibatches of 2^18 records, 16-level 2^19-entry FP16 hash grid + 32-64-64-41 BF16 "
                              "MLP, K = 8",
                     dim=3, grid=256, spp=64, eps=1e-3, maxsteps=128, train_samples=1 << 18, subset=4096,
                     ref_factor=64, batch_wpp=8,
                     step="one training batch: 8 walks per point (376k walks) + its Adam steps",
                     l2="flushed (512 MiB write) before each step"),
    "star2d": dict(workload="2D mixed Dirichlet/Neumann guided WoSt: star polyline 4096 segments, 40% zero-flux "
                            "Neumann arc, g = x^2 - y^2, 512x512 grid masked inside, 32 walks/point, online training "
                            "after every batch of 4 walks per point in minibatches of 2^18 records, 16-level 2^16-entry FP16 hash grid + "
                            "32-64-64-33 BF16 MLP, K = 8",
                   dim=2, grid=512, spp=32, eps=1e-3, maxsteps=128, train_samples=1 << 18, subset=0,
                   ref_factor=16, batch_wpp=4,
                   step="one training batch: 4 walks per point (696k walks) + its Adam steps",
                   l2="flushed (512 MiB write) before each step"),
    "ablations": dict(workload="ablations of Sec. 6.2-6.3 and Tab. mis: on the 81,920-triangle icosphere (64 "
                               "walks/point, training batches of 8 walks/point in minibatches) the MIS modes "
                               "(uniform only c = 0, fixed c = 0.5, guiding only c = 1, learned c), sample "
                               "reflection off, K = 4 and 16 against 8 lobes, and training batches of 1, 4 and 16 "
                               "walks/point; "
                               "on "
                               "the 4096-segment star (512 walks/point) the training budget train_until_wpp in "
                               "{64, 128, 256, 512}; relMSE on the icosphere's 4096-point subset / the star's grid",
                      dim=3, eps=1e-3, maxsteps=128, step="one full solve per variant",
                      l2="flushed (512 MiB write) before each solve"),
    "batch64": dict(workload="64 independent 2D star scenes (256-16384 segments log-uniform, Neumann fraction "
                             "U(0.2, 0.5), 1k-256k points and 8-128 walks per point log-uniform), one persistent "
                             "launch per training round under a CUDA graph, guided with online training per scene "
                             "(and the plain batch for comparison)",
                    dim=2, scenes=64, eps=1e-3, maxsteps=128, step="one replay of the whole batch's graph",
                    l2="flushed (512 MiB write) before each step"),
}
HEADLINE = "genus3"


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def make_workload(key):
    import wost_inputs as wi
    W = WORKLOADS[key]
    if key == "genus3":
        return wi.config_genus3(res=W["grid"])
    if key == "sphere3d":
        return wi.config_3d_guided(res=W["grid"])
    return wi.config_star_guided(res=W["grid"])


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
def smi_gpu_id(torch, dev_index):
    """The nvidia-smi id of a torch device: its UUID (robust to
    CUDA_VISIBLE_DEVICES remapping), else the visible-device mapping."""
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [x.strip() for x in vis.split(",") if x.strip()]
    return ids[dev_index] if dev_index < len(ids) else str(dev_index)


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


def load_profile(name):
    """Per-walk-step counters of a kernel's ncu capture (profiles/*.json)."""
    try:
        return json.load(open(os.path.join(ROOT, "profiles", name)))
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_rate(sc, pts, field_params, W, seconds=12.0, seed=3, guided=True, what="the same scene"):
    """Walk-steps/s of the FP64 oracle on all host cores: guided walks (field
    frozen at the given parameters) over seeded subsamples of the points,
    one walk per point per pass, until about `seconds` have been spent."""
    import oracle
    import wost_inputs as wi
    nth = os.cpu_count() or 1
    O = oracle.Scene(sc)
    OF = oracle.Field(oracle.FieldParams(**field_params)) if guided else None
    prm = oracle.make_params(eps=W["eps"], maxsteps=W["maxsteps"], guided=int(guided), seed=seed, nthreads=nth)
    steps = walks = passes = 0
    n = nth
    t0 = time.perf_counter()
    while True:
        sample = wi.subsample(pts, n, seed=1 + passes)
        t1 = time.perf_counter()
        r = oracle.solve(O, prm, sample, passes, 1, field=OF)
        dt1 = time.perf_counter() - t1
        steps += r["steps"]
        walks += len(sample)
        passes += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
        # grow the pass while it is short, never past the remaining budget
        if dt1 < 0.25 * (seconds - el):
            n = min(len(pts), 2 * n)
    dt = time.perf_counter() - t0
    return steps / dt, dict(cores=nth, sample=f"{walks} walks ({passes} passes of one walk at seeded subsets of the "
                                              f"query points, {steps} walk-steps, {dt:.1f} s) of {what}, "
                                              f"{'guided with the field frozen' if guided else 'plain'}")


def field_params_dict(F, lo, hi, dim):
    import wost_inputs as wi
    p = F.get_params()
    d = F.desc
    return dict(dim=dim, K=d.K, L=d.levels, log2T=d.log2_table, F=d.features, H=d.hidden, base_res=d.base_res,
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
    key = args.workload if args.workload in ("genus3", "sphere3d", "star2d") else HEADLINE
    W = WORKLOADS[key]
    sc, pts = make_workload(key)
    # the field the oracle walks with: the library's default initialisation
    # needs the GPU, so a seeded field of the same shape
    lo, hi = sc.padded_bbox()
    fp = wi.random_field_params(W["dim"], 1, lo, hi, log2T=16 if W["dim"] == 2 else 19, grid_scale=1e-4,
                                w_scale=1.0)
    per, info = [], None
    for i in range(args.warmup + args.steps):
        rate, info = oracle_rate(sc, pts, fp, W, seconds=args.ref_seconds, seed=10 + i,
                                 what=f"the {key} workload")
        if i >= args.warmup:
            per.append(rate)
    value = statistics.mean(per)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * args.ref_seconds, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(W, reference_sample=info["sample"]), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
class Ctx:
    """Device, stream, L2 flush buffer and the API modules of one rank."""

    def __init__(self, torch, api, wi, dev):
        self.torch, self.api, self.wi, self.dev = torch, api, wi, dev
        self.stream = torch.cuda.current_stream()
        self.flush_buf = None

    def flush(self):
        if self.flush_buf is None:
            self.flush_buf = self.torch.empty(128 * 1024 * 1024, dtype=self.torch.float32, device=self.dev)
        self.flush_buf.zero_()

    def events(self):
        E = self.torch.cuda.Event
        return E(enable_timing=True), E(enable_timing=True)

    def timed(self, fn, flush=False):
        if flush:
            self.flush()
        self.torch.cuda.synchronize()
        e0, e1 = self.events()
        e0.record(self.stream)
        out = fn()
        e1.record(self.stream)
        self.torch.cuda.synchronize()
        return e0.elapsed_time(e1), out


def measure_l2_copy_gbs(ctx):
    """L2-resident copy bandwidth (read + write bytes), measured here: a
    24 MiB -> 24 MiB copy repeated 200 times stays in the 129 MB L2."""
    torch = ctx.torch
    n = 6 * 1024 * 1024
    a = torch.ones(n, dtype=torch.float32, device=ctx.dev)
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
    ms, _ = ctx.timed(lambda: [b.copy_(a) for _ in range(200)])
    return 200 * 2 * 4 * n / (ms / 1000.0) / 1e9


def roofline(stats, key, walk_kernel, l2_gbs):
    """Roofline of the dominant kernel (the guided walk kernel): algorithmic
    bytes per launch (visited BVH nodes and primitives, hash-grid corner
    reads, start points, FP64 accumulators, training records; counted in the
    kernel) over its average launch time (library CUDA events on the
    launching stream).  The serving level's figures (L2 bytes and issue
    activity per walk-step) come from the kernel's ncu capture on a small
    case of the same workload, scaled by this run's walk-steps per launch."""
    walk_ms = sum(s["ms_walk"] for s in stats)
    launches = sum(s["walk_launches"] for s in stats)
    steps = sum(s["walk_steps"] for s in stats)
    alg = sum(s["alg_bytes"] for s in stats)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    sec = (walk_ms / launches) / 1000.0
    achieved = (alg / launches) / sec / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": walk_kernel, "peak_source": src,
            "alg_bytes_per_walk_step": alg / steps, "walk_steps_per_launch": steps / launches}
    prof = load_profile(f"{key}_walk_counters.json")
    if prof:
        per = steps / launches
        roof["traffic"] = prof["dram_bytes_per_walk_step"] * per
        lts = prof["lts_bytes_per_walk_step"] * per / sec / 1e9
        roof["serving_level"] = {
            "level": "L2", "achieved": lts, "unit": "GB/s", "peak": l2_gbs, "peak_source": "measured L2 copy",
            "frac": lts / l2_gbs, "lts_bytes_per_walk_step": prof["lts_bytes_per_walk_step"],
            "dram_bytes_per_walk_step": prof["dram_bytes_per_walk_step"],
            "l1_bytes_per_walk_step": prof.get("l1_bytes_per_walk_step"),
            "issue_active_frac": prof.get("issue_active_frac"),
            "threads_per_inst": prof.get("threads_per_inst"),
            "capture": prof.get("capture")}
    return roof


def guided_rounds_line(ctx, key, args, rank=0, world=1, full=True):
    """One single-scene workload, round by round: W warm-up rounds, K timed
    rounds, then (full) the remaining rounds of the solve and the equal-time
    relMSE, the end-to-end rounds with host buffers and the oracle's rate."""
    torch, api, wi = ctx.torch, ctx.api, ctx.wi
    W = WORKLOADS[key]
    dim, spp = W["dim"], W["spp"]
    sc, pts_np = make_workload(key)
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(dim, lo, hi, seed=1 + rank)
    init = F.get_params()
    pts = torch.tensor(pts_np, dtype=torch.float64, device=ctx.dev)
    npts = len(pts_np)
    seed = 1000 + 7919 * rank
    common = dict(eps=W["eps"], maxsteps=W["maxsteps"], stream=ctx.stream)
    gkw = dict(guided=True, field=F, train=1, train_until_wpp=256, train_samples=W["train_samples"], seed=seed,
               **common)
    flush = "flush" in W["l2"]
    nsub = W["subset"] if W["subset"] and W["subset"] < npts else npts
    sub = np.sort(np.random.default_rng(7).choice(npts, nsub, replace=False)) if nsub < npts else np.arange(npts)
    sub_t = torch.tensor(sub, device=ctx.dev)
    acc = torch.zeros(nsub, dtype=torch.float64, device=ctx.dev)

    # a step is one training batch of B walks per point (Sec. 5.2 trains
    # after batches of one walk per point of a 1024^2 grid, about 2^20
    # walks; the smaller point sets take B walks per point per batch)
    B = W.get("batch_wpp", 1)
    nbatch = spp // B
    assert nbatch * B == spp

    def round_(r):
        ms, (m, v, st) = ctx.timed(lambda: api.solve(S, pts, B, walk_begin=r * B, batch_wpp=B, **gkw), flush=flush)
        acc.add_(m[sub_t], alpha=B)
        return ms, st

    warm = min(args.warmup, nbatch - 1)
    nsteps = max(1, min(args.steps, nbatch - warm))
    for r in range(warm):
        round_(r)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    per_ms, stats = [], []
    with ClockSampler(smi_gpu_id(torch, torch.cuda.current_device())) as clk:
        for r in range(warm, warm + nsteps):
            ms, st = round_(r)
            per_ms.append(ms)
            stats.append(st)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    total_ms, steps_all = combine_ranks(sum(per_ms), sum(s["walk_steps"] for s in stats), ctx.dev)
    value = steps_all / (total_ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": nsteps, "warmup": warm,
            "ms_per_step": total_ms / nsteps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE, "data": "synthetic",
            "config": dict(W, points=npts, parallelism=f"replicas x{world}"), "clocks": clk.summary(),
            "gpu_launches": int(round(sum(s["kernel_launches"] for s in stats) / len(stats)))}
    # every walk ends in exactly one terminal step (the closest-point query
    # that finds it in the eps-shell, or the step cap): the rate of the
    # steps that move a walk
    walks_here = sum(s["walks"] for s in stats)
    steps_here = sum(s["walk_steps"] for s in stats)
    line["non_terminal_walk_steps_per_s"] = value * (steps_here - walks_here) / max(steps_here, 1)
    if not full or rank != 0:
        return line, None
    # the rest of the solve (untimed): every round of the spp-walk estimate
    # (only the relMSE needs it)
    if not args.no_relmse:
        for r in range(warm + nsteps, nbatch):
            round_(r)
    guided_s = (sum(per_ms) / nsteps) * nbatch / 1000.0  # a full solve at the timed rate
    # plain walks: time per walk over the whole point set, in one launch of
    # at least 4 M walks (as a plain solve would run them) or all spp walks
    nplain = min(spp, max(2, -(-(1 << 22) // npts)))
    api.solve(S, pts, 1, seed=91, **common)
    pms, (mp_, vp_, stp) = ctx.timed(lambda: api.solve(S, pts, nplain, seed=92, **common), flush=flush)
    plain_rate = stp["walk_steps"] / (pms / 1000.0)
    plain_s = pms / 1000.0 * spp / nplain                 # a full plain solve at spp walks
    psub = pts[sub_t].contiguous()
    guided_mean = (acc / (B * (warm + nsteps) if args.no_relmse else spp)).cpu().numpy()
    relmse = None
    if not args.no_relmse:
        spp_ref = W["ref_factor"] * spp
        ref, rvar, _ = api.solve(S, psub, spp_ref, seed=424242, **common)
        ref, rvar = ref.cpu().numpy(), rvar.cpu().numpy()

        def rel(u):
            return float(np.mean((u - ref) ** 2 / (ref ** 2 + 1e-2)))

        def rel_c(u):      # the reference's own variance removed (an unbiased estimate)
            return float(np.mean(((u - ref) ** 2 - rvar) / (ref ** 2 + 1e-2)))
        spp_eq = max(1, int(spp * guided_s / plain_s))
        m_eq = api.solve(S, psub, spp_eq, seed=515151, **common)[0].cpu().numpy()
        m_sp = api.solve(S, psub, spp, seed=616161, **common)[0].cpu().numpy()
        relmse = {"guided": rel(guided_mean), "plain_equal_time": rel(m_eq), "plain_equal_spp": rel(m_sp),
                  "plain_spp_at_equal_time": spp_eq,
                  "equal_time_ratio_plain_over_guided": rel(m_eq) / rel(guided_mean),
                  "corrected": {"guided": rel_c(guided_mean), "plain_equal_time": rel_c(m_eq),
                                "plain_equal_spp": rel_c(m_sp),
                                "equal_time_ratio_plain_over_guided": rel_c(m_eq) / rel_c(guided_mean),
                                "note": "the reference's own per-point variance subtracted"},
                  "variance_reduction_equal_spp": rel_c(m_sp) / rel_c(guided_mean),
                  "guided_over_plain_cost_per_walk": guided_s / plain_s,
                  "subset_points": nsub, "reference": f"plain WoSt, {spp_ref} walks/point on the subset",
                  "guided_s_per_solve": guided_s, "plain_s_per_solve": plain_s}
    # end to end through the C ABI with host buffers: pinned host points in,
    # mean and variance out, every round a wost_solve call
    pts_host = torch.tensor(pts_np, dtype=torch.float64).pin_memory().numpy()
    F.set_params(init["grid"], init["W1"], init["W2"], init["W3"], init["b3"])
    e2e_steps, e2e_s = 0, 0.0
    for r in range(min(3, nbatch)):
        if flush:
            ctx.flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m, v, st = api.solve(S, pts_host, B, walk_begin=r * B, guided=True, field=F, train=1, train_until_wpp=256,
                             batch_wpp=B, train_samples=W["train_samples"], seed=seed + 1, eps=W["eps"],
                             maxsteps=W["maxsteps"])
        e2e_s += time.perf_counter() - t0
        e2e_steps += st["walk_steps"]
    line["e2e"] = {"value": e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(npts * dim * 8),
                   "d2h_bytes_per_step": int(npts * 2 * 8)}
    kern = f"guided_walk_kernel<{dim}>"
    line["roofline"] = roofline(stats, key, kern, ctx.l2_gbs)
    cpu = None
    if not args.no_cpu_baseline:
        rate, info = oracle_rate(sc, pts_np[sub] if nsub < npts else pts_np, field_params_dict(F, lo, hi, dim), W,
                                 seconds=args.cpu_seconds, what=f"the {key} workload")
        cpu = {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle", "sample": info["sample"]}
    line["cpu_baseline"] = cpu
    line["breakdown"] = {"walk_ms_per_step": sum(s["ms_walk"] for s in stats) / len(stats),
                         "train_ms_per_step": sum(s["ms_train"] for s in stats) / len(stats),
                         "walk_steps_per_step": sum(s["walk_steps"] for s in stats) / len(stats),
                         "records_per_step": sum(s["records"] for s in stats) / len(stats),
                         "adam_steps_per_step": sum(s["train_steps"] for s in stats) / len(stats)}
    line["plain_walk_steps_per_s"] = plain_rate
    line["relmse"] = relmse
    return line, F


def decode_line(ctx, F, dim, lo, hi):
    """The tensor-core decode on its own: 4 Mi positions through
    wost_field_decode (hash-grid encode + three tcgen05 BF16 MMAs per 128-row
    tile), device buffers, CUDA events on the stream."""
    torch, api = ctx.torch, ctx.api
    ndec = 1 << 22
    g = torch.Generator(device=ctx.dev)
    g.manual_seed(5)
    lo_t = torch.tensor(lo, dtype=torch.float64, device=ctx.dev)
    hi_t = torch.tensor(hi, dtype=torch.float64, device=ctx.dev)
    pts = lo_t + (hi_t - lo_t) * torch.rand((ndec, dim), dtype=torch.float64, device=ctx.dev, generator=g)
    out = torch.empty((ndec, F.nout), dtype=torch.float32, device=ctx.dev)
    ex = api.exec_defaults(stream=ctx.stream)
    for _ in range(3):
        F.decode(pts, out=out, exec_=ex)
    ms, _ = ctx.timed(lambda: F.decode(pts, out=out, exec_=ex), flush=True)
    nout = (dim + 2) * 8 + 1
    flop = 2.0 * (32 * 64 + 64 * 64 + 64 * nout)          # the method's FLOPs per decode (unpadded)
    peak = measured_peaks().get("bf16_tflops")
    tf = ndec * flop / (ms / 1000.0) / 1e12
    return {"points": ndec, "ms": ms, "decodes_per_s": ndec / (ms / 1000.0), "bound": "tensor",
            "achieved_tflops": tf, "peak_tflops": peak or 1900.0, "frac": tf / (peak or 1900.0),
            "peak_source": "measured" if peak else "fallback", "flop_per_decode": flop,
            "note": f"per point {flop / 1e3:.1f} kFLOP of BF16 MMA against {16 * 2 ** dim} hash-grid corner "
                    "gathers (L2): the encode gathers, not the tensor pipe, set the decode time"}


def batch_line(ctx, args):
    """64 scenes in one persistent launch per training round under a CUDA
    graph: guided (online training per scene) and plain."""
    torch, api, wi = ctx.torch, ctx.api, ctx.wi
    W = WORKLOADS["batch64"]
    jobs = wi.config_batch()
    scenes = [api.Scene(j.scene) for j in jobs]
    pts = [torch.tensor(j.points, dtype=torch.float64, device=ctx.dev) for j in jobs]
    plans, fields = {}, []
    for guided in (True, False):
        specs = []
        for i, j in enumerate(jobs):
            d = dict(scene=scenes[i], points=pts[i], nwalks=j.nwalks, seed=j.seed, eps=W["eps"], maxsteps=W["maxsteps"])
            if guided:
                lo, hi = scenes[i].bbox()
                d["field"] = api.Field(2, lo, hi, seed=1 + i)
                fields.append(d["field"])
            specs.append(d)
        plans[guided] = api.Batch(specs, guided=guided, train=1 if guided else 0)

    def run(guided):
        return ctx.timed(lambda: plans[guided].run(ctx.stream.cuda_stream), flush=True)
    # one replay takes about 19 s (150 M walks, 2,741 training steps): one
    # warm-up replay (the plan's autotuner already ran its calibration
    # launches) and two timed ones
    run(True)
    per, stats = [], []
    nsteps = max(1, min(args.steps, 2))
    with ClockSampler(smi_gpu_id(torch, torch.cuda.current_device())) as clk:
        for _ in range(nsteps):
            ms, st = run(True)
            per.append(ms)
            stats.append(st)
    pms, pst = run(False)
    value = sum(s["walk_steps"] for s in stats) / (sum(per) / 1000.0)
    # end to end: the points copied from pinned host memory into the plan's
    # device inputs and every job's mean copied back, around each replay
    host = [torch.tensor(j.points, dtype=torch.float64).pin_memory() for j in jobs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = 0
    for _ in range(2):
        for h, d in zip(host, pts):
            d.copy_(h, non_blocking=True)
        st = plans[True].run(ctx.stream.cuda_stream)
        outs = [m.cpu() for m in plans[True].mean]
        e2e_steps += st["walk_steps"]
    e2e_s = time.perf_counter() - t0
    npts = sum(len(j.points) for j in jobs)
    for_roof = [dict(ms_walk=s["ms_walk"], walk_launches=s["walk_launches"], walk_steps=s["walk_steps"],
                     alg_bytes=s["alg_bytes"]) for s in stats]
    line = {"value": value, "unit": UNIT, "steps": nsteps, "ms_per_step": sum(per) / nsteps,
            "config": dict(W, points=npts, walks=sum(len(j.points) * j.nwalks for j in jobs),
                           plan={"guided": plans[True].info(), "plain": plans[False].info()}),
            "clocks": clk.summary(), "plain_walk_steps_per_s": pst["walk_steps"] / (pms / 1000.0),
            "gpu_launches": int(plans[True].info()["graph_nodes"]),
            "e2e": {"value": e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(npts * 2 * 8),
                    "d2h_bytes_per_step": int(npts * 8)},
            "roofline": roofline(for_roof, "batch64", "batch_guided_kernel<2>", ctx.l2_gbs)}
    del outs
    if not args.no_cpu_baseline:
        j = jobs[0]
        lo, hi = scenes[0].bbox()
        rate, info = oracle_rate(j.scene, j.points, field_params_dict(fields[0], lo, hi, 2), W,
                                 seconds=min(args.cpu_seconds, 5.0), what="the batch's first scene")
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                                "sample": info["sample"]}
    return line


def ablation_line(ctx, args):
    """relMSE of guided variants at equal walks and at equal time (the
    plain solve's time per walk measured alongside)."""
    torch, api, wi = ctx.torch, ctx.api, ctx.wi
    out = {}

    def variants(key, specs, spp, subset, ref_factor):
        W = WORKLOADS[key]
        sc, pts_np = make_workload(key)
        S = api.Scene(sc)
        lo, hi = S.bbox()
        pts = torch.tensor(pts_np, dtype=torch.float64, device=ctx.dev)
        npts = len(pts_np)
        sub = (np.sort(np.random.default_rng(7).choice(npts, subset, replace=False)) if subset and subset < npts
               else np.arange(npts))
        sub_t = torch.tensor(sub, device=ctx.dev)
        psub = pts[sub_t].contiguous()
        common = dict(eps=W["eps"], maxsteps=W["maxsteps"], stream=ctx.stream)
        ref, rvar, _ = api.solve(S, psub, spp * ref_factor, seed=424242, **common)
        ref, rvar = ref.cpu().numpy(), rvar.cpu().numpy()

        def rel(u):   # the reference's own variance removed
            return float(np.mean(((u - ref) ** 2 - rvar) / (ref ** 2 + 1e-2)))
        nplain = min(spp, max(2, -(-(1 << 22) // npts)))
        pms, (mp, _, stp) = ctx.timed(lambda: api.solve(S, pts, nplain, seed=92, **common), flush=True)
        plain_s_per_walk = pms / 1000.0 / nplain
        m_sp = api.solve(S, psub, spp, seed=616161, **common)[0].cpu().numpy()
        res = {"plain": {"relmse_equal_spp": rel(m_sp), "s_per_solve": plain_s_per_walk * spp}}
        for name, fkw, ekw in specs:
            F = api.Field(W["dim"], lo, hi, seed=1, **fkw)
            ekw = {"batch_wpp": W.get("batch_wpp", 1), **ekw}
            ms, (m, v, st) = ctx.timed(lambda: api.solve(S, pts, spp, seed=77, guided=True, field=F, train=1,
                                                         train_samples=W.get("train_samples", 0), **common,
                                                         **ekw), flush=True)
            g_s = ms / 1000.0
            spp_eq = max(1, int(spp * g_s / (plain_s_per_walk * spp)))
            m_eq = api.solve(S, psub, spp_eq, seed=515151, **common)[0].cpu().numpy()
            rg = rel(m.cpu().numpy()[sub])
            res[name] = {"relmse_equal_spp": rg, "s_per_solve": g_s, "walk_steps_per_s": st["walk_steps"] / g_s,
                         "plain_spp_at_equal_time": spp_eq, "plain_relmse_equal_time": rel(m_eq),
                         "equal_time_ratio_plain_over_guided": rel(m_eq) / rg,
                         "variance_reduction_equal_spp": res["plain"]["relmse_equal_spp"] / rg}
            print(json.dumps({"ablation": key, "variant": name, **res[name]}), flush=True)
        return res

    out["icosphere_64wpp"] = variants("sphere3d", [
        ("learned c (default)", {}, {}),
        ("fixed c = 0.5", {}, dict(c_mode=1, c_fixed=0.5)),
        ("guiding only, c = 1", {}, dict(c_mode=1, c_fixed=1.0)),
        ("uniform only, c = 0", {}, dict(c_mode=1, c_fixed=0.0)),
        ("no sample reflection", {}, dict(reflect=0)),
        ("K = 4 lobes", dict(K=4), {}),
        ("K = 16 lobes", dict(K=16), {}),
        ("training batch of 1 walk/point", {}, dict(batch_wpp=1)),
        ("training batch of 4 walks/point", {}, dict(batch_wpp=4)),
        ("training batch of 16 walks/point", {}, dict(batch_wpp=16)),
    ], 64, 4096, 32)
    out["star_512wpp_training_budget"] = variants("star2d", [
        (f"train_until_wpp = {b}", {}, dict(train_until_wpp=b)) for b in (64, 128, 256, 512)
    ], 512, 0, 4)
    return out


def run_ours(args):
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import wost_inputs as wi
    from paper_2410_18944_gb300 import api, build
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ctx = Ctx(torch, api, wi, dev)
    ctx.l2_gbs = measure_l2_copy_gbs(ctx)
    if args.workload == "ablations":
        if rank == 0:
            res = ablation_line(ctx, args)
            print(json.dumps({"metric": METRIC, "unit": UNIT, "impl": "ours",
                              "config": dict(WORKLOADS["ablations"]), "ablations": res}), flush=True)
        return 0
    key = args.workload if args.workload in ("genus3", "sphere3d", "star2d") else HEADLINE
    line, F = guided_rounds_line(ctx, key, args, rank, world, full=True)
    if rank != 0:
        return 0
    lo, hi = F.desc.lo[:WORKLOADS[key]["dim"]], F.desc.hi[:WORKLOADS[key]["dim"]]
    line["decode"] = decode_line(ctx, F, WORKLOADS[key]["dim"], list(lo), list(hi))
    line["l2_copy_gbs"] = ctx.l2_gbs
    if not args.no_extras and key == HEADLINE:
        extras = {}
        xargs = argparse.Namespace(**vars(args))
        xargs.cpu_seconds = min(args.cpu_seconds, 6.0)
        for k in ("star2d", "sphere3d"):
            l, _ = guided_rounds_line(ctx, k, xargs, full=True)
            extras[k] = {x: l[x] for x in ("value", "unit", "steps", "warmup", "ms_per_step", "config", "clocks",
                                           "gpu_launches", "e2e", "roofline", "cpu_baseline", "breakdown",
                                           "plain_walk_steps_per_s", "relmse")}
        extras["batch64"] = batch_line(ctx, xargs)
        line["extras"] = extras
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
    key = args.workload if args.workload in ("genus3", "sphere3d", "star2d") else HEADLINE
    W = WORKLOADS[key]
    sc, pts = make_workload(key)
    if args.points and args.points < len(pts):
        pts = wi.subsample(pts, args.points, seed=1)
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(W["dim"], lo, hi)
    p = torch.tensor(pts, dtype=torch.float64, device="cuda")
    guided = args.once == "guided"
    spp = args.spp or W.get("spp", 1)
    for rep in range(2):
        m, v, st = api.solve(S, p, spp, eps=W["eps"], maxsteps=W["maxsteps"], seed=rep, guided=guided,
                             field=F if guided else None, train=1 if guided else 0,
                             train_samples=W["train_samples"] if guided else 0, batch_wpp=W.get("batch_wpp", 1))
        torch.cuda.synchronize()
        print(json.dumps({"once": args.once, "rep": rep, **{k: st[k] for k in (
            "walk_steps", "ms_walk", "ms_train", "node_visits", "prim_visits", "dir_prim_visits", "sil_prim_visits",
            "neu_prim_visits", "kernel_launches", "records", "walk_launches")}}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=list(WORKLOADS), default=HEADLINE,
                    help="genus3 (the benchmark line) or another workload of the method as the main line")
    ap.add_argument("--once", choices=["plain", "guided"], default=None,
                    help="run one solve of the workload (profiling), no timing")
    ap.add_argument("--points", type=int, default=0, help="with --once: seeded subset of the query points")
    ap.add_argument("--spp", type=int, default=0, help="with --once: walks per point (default: the workload's)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-relmse", action="store_true", help="skip the equal-time relMSE measurement")
    ap.add_argument("--no-extras", action="store_true", help="the main line only")
    ap.add_argument("--batch-wpp", type=int, default=0,
                    help="walks per point in one training batch of the main workload (default: the workload's)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.batch_wpp > 0:
        W = WORKLOADS[args.workload]
        W["batch_wpp"] = args.batch_wpp
        W["workload"] += f"; training batches of {args.batch_wpp} walks per point"
    if args.once:
        return run_once(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
