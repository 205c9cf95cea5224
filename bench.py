#!/usr/bin/env python
"""Throughput of cosine mean-shift with OSOP on 512x512, d = 16 frames.

One step = B synthetic frames (512x512, 131072 foreground pixels, 60 vMF
cells, kappa ~ U[20, 200], 2% outliers) clustered end to end on the GPU:
ingest, every OSOP round (seed selection, shift iterations, merge, coverage,
N schedule) and labelling. The headline form is BF16-batched: all B frames in
one CUDA graph (ms_batch_run), BF16 tensor-core shift with the FP32 recheck
band. The plain FP32 form (one frame at a time, host round loop) is measured
in the same run for comparison. Embeddings are resident in HBM before timing;
L2 is flushed between steps. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--frames B]
                  [--form bf16-batched|fp32-batched|fp32|bf16] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank clusters its own frames: replicas,
weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "512² d=16 frames/s, FP32 vs BF16-batched at ≥99.9% label match; % TC peak"
WORKLOAD = ("512x512 frame, 131072 foreground px, d=16, 60 vMF cells (log-normal sizes, median "
            "2000 px, kappa~U[20,200]) + 2% uniform outliers; flat kernel c=0.9, tol 1e-6, OSOP "
            "gamma=0.9 N_initial=128 L=2 H=8")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
SHIFT_SRC = os.path.join(ROOT, "paper_2007_14283_gb300", "csrc", "ms_shift_fp32.cu")
SHIFT_TC_SRC = os.path.join(ROOT, "paper_2007_14283_gb300", "csrc", "ms_shift_tc.cu")
C2_STATS = os.path.join(ROOT, "tests", "golden", "c2_oracle_stats.json")
FP32_LANES_PER_SM = 128
N_FG, DIM = 131072, 16
FORMS = ("bf16-batched", "fp32-batched", "fp32", "bf16")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--frames", type=int, default=64, help="frames per step (per GPU)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=FORMS, default="bf16-batched")
    ap.add_argument("--compare", default="fp32",
                    help="comma-separated other forms measured on --compare-frames frames ('' for none)")
    ap.add_argument("--compare-frames", type=int, default=8)
    ap.add_argument("--compare-steps", type=int, default=2)
    ap.add_argument("--cpu", choices=["full", "sample", "none"], default="full",
                    help="oracle baseline: one full frame (also gives the label match), a seed sample, or none")
    ap.add_argument("--cpu-seeds", type=int, default=8192, help="seeds in the oracle's sampled run")
    ap.add_argument("--cpu-runs", type=int, default=3,
                    help="--cpu full: also the median of this many sampled runs and a one-core run (0: none)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-vmf", action="store_true", help="skip the smooth-kernel (vMF) forward/adjoint leg")
    ap.add_argument("--video-frames", type=int, default=16,
                    help="frames of the video-form leg (drifting 512x512 sequence; 0 skips it)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched forms: skip the work-split autotuner (keep the canonical split)")
    ap.add_argument("--eager", action="store_true",
                    help="batched forms: issue the graph's kernels as plain launches (for profilers)")
    ap.add_argument("--shift-only", type=int, default=0, metavar="SEEDS",
                    help="time one shift iteration of SEEDS seeds on frame 0 (fp32 or bf16 form) and exit")
    ap.add_argument("--tc-shape", type=int, default=0,
                    help="with --shift-only: the tensor-core shift kernel's tile shape (ms_config.tc_shape)")
    ap.add_argument("--suite", action="store_true",
                    help="the paper's simulation suite (Table 1 sizes, Appendix A overlap, Tables 3-4) and exit")
    ap.add_argument("--volume", action="store_true", help="one 3D volume (128x256x256 voxels) and exit")
    ap.add_argument("--vmf-only", action="store_true",
                    help="time only the smooth-kernel forward and adjoint (differentiable configuration) and exit")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(v, ws, op):
    """max or sum of a scalar over the ranks (a CPU tensor under gloo)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units, seconds, ws):
    """Replicas' whole-job throughput: the units all ranks processed over the
    slowest rank's time. Returns (rate, slowest time)."""
    t = reduce_over_ranks(seconds, ws, "max")
    return reduce_over_ranks(units, ws, "sum") / t, t


class Clocks:
    """nvidia-smi samples every 200 ms while running (the GPU this rank uses)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def load_peaks():
    try:
        return json.load(open(PEAKS))
    except (OSError, ValueError):
        return {}


def shift_traffic_per_unit(kernel):
    """DRAM bytes per frame-iteration (one launch's pass over one frame) of the
    shift kernel from the committed ncu summary, valid only while the kernel
    source is unchanged."""
    src = SHIFT_TC_SRC if kernel == "k_shift_tc" else SHIFT_SRC
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(TRAFFIC):
            if line.startswith("#") or not line.strip():
                continue
            name, per_unit, src_hash = line.split()[:3]
            if name == kernel and src_hash == h:
                return float(per_unit)
    except (OSError, ValueError):
        pass
    return None


def frame_seeds(rank, B):
    """Seeds of the B frames a rank clusters; ranks' shards are disjoint."""
    if not 0 <= B <= 1000:
        raise ValueError("at most 1000 frames per rank keep the ranks' seeds disjoint")
    return [rank * 1000 + i for i in range(B)]


def c2_frames(rank, B):
    import synth
    return [synth.frame_c2(seed=s) for s in frame_seeds(rank, B)]


def c2_seed_iters_per_frame():
    try:
        return float(json.load(open(C2_STATS))["seed_iters"])
    except (OSError, ValueError, KeyError):
        return None


def host_threads():
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or len(os.sched_getaffinity(0))


def oracle_sample(frame, n_seeds):
    """Time the oracle's shift rounds on the first n_seeds positions of the
    frame's seed order; returns (seconds, seed-iterations)."""
    import numpy as np
    import oracle
    P, pn, _ = oracle.normalize(frame.emb, frame.mask)
    perm = [oracle.lib().or_perm_at(j, P.shape[0], *oracle.perm_params(P.shape[0])) for j in range(n_seeds)]
    X0 = P[np.asarray(perm)]
    t0 = time.perf_counter()
    r = oracle.shift_round(P, pn, X0, gamma=0.9)
    return time.perf_counter() - t0, r["seed_iters"]


def oracle_sample_single_core(n_seeds):
    """The same bounded sample timed on one host core: a child process with
    OMP_NUM_THREADS=1 (the oracle's OpenMP team size is fixed when it loads).
    Returns (seconds, seed-iterations)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "f = bench.c2_frames(0, 1)[0]; dt, si = bench.oracle_sample(f, %d); "
            "print(json.dumps([dt, si]))" % (ROOT, n_seeds))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    dt, si = json.loads(out.stdout.strip().splitlines()[-1])
    return dt, si


def label_match(gpu_labels, ref_labels, gpu_modes, ref_modes):
    """Share of foreground pixels labelled identically. Both sides keep modes
    in the same deterministic order, so when the mode lists agree one to one
    (same count, 1 - cos <= 1e-5 pairwise in order) the maps are compared
    index by index; otherwise clusters are matched greedily by overlap (a
    lower bound on the optimal matching)."""
    import numpy as np
    a, b = np.asarray(ref_labels), np.asarray(gpu_labels)
    fg = a >= 0
    bg_ok = bool(((a < 0) == (b < 0)).all())
    a, b = a[fg], b[fg]
    g = np.asarray(gpu_modes, np.float64)
    r = np.asarray(ref_modes, np.float64)
    errs = None
    if g.shape == r.shape and g.size:
        errs = 1.0 - (g * r).sum(1) / (np.linalg.norm(g, axis=1) * np.linalg.norm(r, axis=1))
    if errs is not None and errs.max() <= 1e-5:
        return float((a == b).mean()), "same mode order", float(errs.max()), bg_ok
    pairs = a.astype(np.int64) * (int(b.max()) + 1) + b
    key, cnt = np.unique(pairs, return_counts=True)
    order = np.argsort(-cnt, kind="stable")
    used_a, used_b, hit = set(), set(), 0
    nb = int(b.max()) + 1
    for k, c in zip(key[order], cnt[order]):
        ia, ib = int(k // nb), int(k % nb)
        if ia in used_a or ib in used_b:
            continue
        used_a.add(ia)
        used_b.add(ib)
        hit += int(c)
    err = None
    if g.size and r.size:
        gn = g / np.linalg.norm(g, axis=1, keepdims=True)
        rn = r / np.linalg.norm(r, axis=1, keepdims=True)
        err = float((1.0 - (gn @ rn.T).max(axis=1)).max())
    return hit / max(1, a.size), "greedy overlap matching", err, bg_ok


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank):
    """The FP64 oracle as it stands on the host cores: each step times a
    bounded sample (the first --cpu-seeds seeds of a frame's order shifted to
    the gamma stop) and scales it to frames/s."""
    if rank != 0:
        return
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # the other ranks do no work: the oracle gets every host core, as at
        # N = 1 (torchrun's default of one thread per rank would otherwise
        # hold; the OpenMP team is sized when the oracle library loads)
        os.environ["OMP_NUM_THREADS"] = str(len(os.sched_getaffinity(0)))
    frame = c2_frames(0, 1)[0]
    per_frame = c2_seed_iters_per_frame()
    for _ in range(args.warmup):
        oracle_sample(frame, max(16, args.cpu_seeds // 8))
    times, its = [], []
    for _ in range(args.steps):
        dt, si = oracle_sample(frame, args.cpu_seeds)
        times.append(dt)
        its.append(si)
    frame_s = sum(times) / sum(its) * per_frame if per_frame else float("nan")
    value = 1.0 / frame_s
    sample = (f"{args.cpu_seeds} seeds of the frame's seed order shifted to the gamma stop by the oracle "
              f"({sum(its) // args.steps} seed-iterations per step), scaled by the oracle's "
              f"{int(per_frame or 0)} seed-iterations per full frame; merge/cover/label not included")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic vMF frames", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": host_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
class Runner:
    """One form of the method over a fixed list of device-resident frames."""

    def __init__(self, ms, form, frames, dev, eager=False, autotune=False):
        import torch
        self.ms, self.form, self.frames = ms, form, frames
        self.batched = form.endswith("batched")
        prec = ms.MS_BF16 if form.startswith("bf16") else ms.MS_FP32
        self.cfg = ms.ms_config_default(dim=DIM, precision=prec)
        self.embs = [torch.from_numpy(f.emb).to(dev) for f in frames]
        self.masks = [torch.from_numpy(f.mask).to(dev) for f in frames]
        self.eager_passes = 0
        self.tuning = None
        if self.batched:
            self.batch = ms.ms_batch_create(self.cfg, self.embs, self.masks)
            if autotune:
                self.tuning = ms.ms_batch_autotune(self.batch, reps=2)
            if eager:
                ms.ms_batch_run(self.batch)
                self.eager_passes = ms.ms_batch_stats(self.batch, -1)["reserved0"]
            else:
                ms.ms_batch_profile(self.batch, True)
            self.labels = self.batch.labels
        else:
            self.labels = [torch.empty(f.emb.shape[0], dtype=torch.int32, device=dev) for f in frames]

    def step(self):
        """Cluster every frame once; returns counters of this step."""
        ms = self.ms
        if self.batched:
            if self.eager_passes:
                ms.ms_batch_run_eager(self.batch, self.eager_passes)
            else:
                ms.ms_batch_run(self.batch)
            st = ms.ms_batch_stats(self.batch, -1)
            return {"frames": len(self.frames), "launches": st["launches"], "shift_ms": st["shift_ms"],
                    "shift_launches": st["shift_launches"], "seed_iters": st["seed_iters"],
                    "modes": st["n_modes"], "passes": st["reserved0"], "band_pairs": st["band_pairs"],
                    "frame_iters": st["iters_total"]}
        agg = {"frames": 0, "launches": 0, "shift_ms": 0.0, "shift_launches": 0, "seed_iters": 0, "modes": 0,
               "passes": 0, "band_pairs": 0, "frame_iters": 0}
        for f, (e, m, l) in enumerate(zip(self.embs, self.masks, self.labels)):
            self.cfg.frame_id = f  # the batch gives frame f the seed order of frame_id f
            ctx = ms.ms_create(self.cfg, e, m)
            ms.ms_profile(ctx, True)
            ms.ms_run(ctx, l)
            st = ms.ms_stats_get(ctx)
            ctx.close()
            agg["frames"] += 1
            for k in ("launches", "shift_ms", "shift_launches", "seed_iters", "band_pairs"):
                agg[k] += st[k]
            agg["frame_iters"] += st["iters_total"]
            agg["modes"] += st["n_modes"]
        return agg

    def modes(self, f):
        ms = self.ms
        if self.batched:
            return ms.ms_batch_modes(self.batch, f)
        return ms.cluster(self.embs[f], self.masks[f], precision=self.cfg.precision,
                          frame_id=f).modes.cpu().numpy()

    def close(self):
        if self.batched:
            self.batch.close()


def timed(runner, steps, warmup, ws, flush, stream):
    import torch
    for _ in range(warmup):
        runner.step()
    torch.cuda.synchronize()
    step_ms, tot = [], {}
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier(ws)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        agg = runner.step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        step_ms.append(ev0.elapsed_time(ev1))
        for k, v in agg.items():
            tot[k] = tot.get(k, 0) + v
    return step_ms, tot


def roofline_of(form, tot, step_ms, clk, n_sm):
    flops = 4.0 * DIM * N_FG * tot["seed_iters"]
    achieved = flops / (tot["shift_ms"] / 1e3) / 1e12 if tot["shift_ms"] > 0 else None
    sm_mhz = clk.get("sm_mhz") or 1455.0
    if form.startswith("bf16"):
        peaks = load_peaks()
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        bound, kernel = "tensor", "k_shift_tc"
        peak_source = ("of measured: cuBLAS bf16 dense, sustained (MEASURED_PEAKS.json)"
                       if peaks.get("bf16_tflops_sustained") else "of fallback: 1.7 PFLOP/s sustained")
    else:
        peak = n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        bound, kernel = "alu", "k_shift_fp32"
        peak_source = (f"FP32 FMA peak = {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_mhz:.0f} MHz "
                       "(median SM clock sampled under load)")
    tpu = shift_traffic_per_unit(kernel)
    per_launch_si = tot["seed_iters"] / max(1, tot["shift_launches"])
    per_launch_fi = tot.get("frame_iters", 0) / max(1, tot["shift_launches"])
    return {"bound": bound, "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": (tpu * per_launch_fi) if (tpu and per_launch_fi) else None,
            "traffic_basis": "ncu dram bytes of one frame-iteration (profiles/ncu_traffic.txt) x "
                             f"{per_launch_fi:.2f} frame-iterations per launch",
            "peak_source": peak_source,
            "algorithmic": f"4*d*n flops per seed-iteration (d={DIM}, n={N_FG}); "
                           f"{per_launch_si:.0f} seed-iterations per launch on average",
            "timing": ("GPU global-timer ticks in one-thread kernels around each shift launch inside the graph "
                       "(includes one launch gap per launch)" if form.endswith("batched")
                       else "CUDA events around each shift launch on the library's stream"),
            "shift_share_of_step": (tot["shift_ms"] / sum(step_ms)) if step_ms else None,
            "shift_launches": tot["shift_launches"],
            "avg_launch_ms": tot["shift_ms"] / max(1, tot["shift_launches"])}


def vmf_leg(n_sm, clk):
    """Smooth-kernel form on the differentiable configuration: N = 65536 pixels,
    M = 1024 seeds, d = 16, kappa = 20, T = 10. Times ms_vmf_forward and
    ms_vmf_backward (CUDA events, median of 5 after 2 warm-ups), in FP32 and
    on the tensor cores (MS_BF16: forward steps and both adjoint passes).

    Bound: FP32 FMA on the CUDA cores. Per seed-pixel pair and step the
    forward does the 16-term dot product and the 16-term weighted sum (4d = 64
    flops) and one exp; the adjoint re-runs the forward (64), then pass A's two
    dot products and weighted sum (96) and pass B's two dot products and two
    weighted sums (128): 288 flops and two exps. The exps (one special-function
    result per pair, 16 per SM per clock) bind well below the FMAs."""
    import torch

    import paper_2007_14283_gb300 as ms
    import synth
    prob = synth.vmf_problem_c5(seed=0, N=65536, M=1024, K=32)
    P = torch.from_numpy(prob["P"]).cuda()
    X0 = torch.from_numpy(prob["X0"]).cuda()
    G = (torch.from_numpy(prob["target"]).cuda() - X0) * 2.0
    kappa, T = 20.0, 10
    stream = torch.cuda.current_stream()

    def timed_ms(fn):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)
    fwd = timed_ms(lambda: ms.ms_vmf_forward(P, X0, kappa, T))
    bwd = timed_ms(lambda: ms.ms_vmf_backward(P, X0, kappa, T, G))
    pairs = 65536 * 1024 * T
    sm_mhz = clk.get("sm_mhz") or 2070.0
    fma_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 TFLOP/s: 128 FMA lanes per SM
    f_tf = 64 * pairs / (fwd * 1e-3) / 1e12
    b_tf = 288 * pairs / (bwd * 1e-3) / 1e12
    # BF16 form: every forward step on the tensor cores (k_vmf_tc + its reduce);
    # a step's time is the slope between T = 10 and T = 1 calls (the call's
    # fixed cost -- packing the pixels, one synchronisation -- cancels).
    BF = ms.MS_BF16
    fwd_b = timed_ms(lambda: ms.ms_vmf_forward(P, X0, kappa, T, precision=BF))
    fwd_b1 = timed_ms(lambda: ms.ms_vmf_forward(P, X0, kappa, 1, precision=BF))
    bwd_b = timed_ms(lambda: ms.ms_vmf_backward(P, X0, kappa, T, G, precision=BF))
    bwd_b1 = timed_ms(lambda: ms.ms_vmf_backward(P, X0, kappa, 1, G, precision=BF))
    step_b = (fwd_b - fwd_b1) / (T - 1)
    # one reverse step (k_vmf_gy, the packing, both tensor-core passes and
    # their reduces): the backward's slope between T = 10 and T = 1 minus the
    # re-run forward's step; 224 flops per pair (pass A 96, pass B 128)
    adj_b = (bwd_b - bwd_b1) / (T - 1) - step_b
    bf16_peak = load_peaks().get("bf16_tflops")
    step_tf = 64 * 65536 * 1024 / (step_b * 1e-3) / 1e12
    adj_tf = 224 * 65536 * 1024 / (adj_b * 1e-3) / 1e12
    xf = ms.ms_vmf_forward(P, X0, kappa, T)
    xb = ms.ms_vmf_forward(P, X0, kappa, T, precision=BF)
    gf = ms.ms_vmf_backward(P, X0, kappa, T, G)
    gb = ms.ms_vmf_backward(P, X0, kappa, T, G, precision=BF)
    grad_rel = [float(((b - f).norm() / f.norm()).item()) for b, f in zip(gb, gf)]
    return {"config": "N=65536 pixels, M=1024 seeds, d=16, kappa=20, T=10 (synthetic vMF cells)",
            "forward_ms": fwd, "backward_ms": bwd,
            "bound": "fp32 fma", "unit": "TFLOP/s",
            "forward_achieved": f_tf, "backward_achieved": b_tf, "peak": fma_peak,
            "forward_frac": f_tf / fma_peak, "backward_frac": b_tf / fma_peak,
            "algorithmic": "64 flops per seed-pixel pair and step (forward); 288 (adjoint, with the re-run forward)",
            "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flops x {sm_mhz:.0f} MHz (nominal CUDA-core rate)",
            "bf16": {"forward_ms": fwd_b, "forward_T1_ms": fwd_b1, "backward_ms": bwd_b, "backward_T1_ms": bwd_b1,
                     "step_ms": step_b, "adjoint_step_ms": adj_b,
                     "bound": "tensor", "step_achieved": step_tf, "adjoint_step_achieved": adj_tf, "peak": bf16_peak,
                     "step_frac": (step_tf / bf16_peak) if bf16_peak else None,
                     "adjoint_step_frac": (adj_tf / bf16_peak) if bf16_peak else None,
                     "peak_source": "of measured: cuBLAS bf16 dense, burst (MEASURED_PEAKS.json)",
                     "max_abs_diff_vs_fp32_form": float((xb - xf).abs().max().item()),
                     "grad_rel_diff_vs_fp32_form": {"dP": grad_rel[0], "dX0": grad_rel[1]},
                     "note": "forward steps and both adjoint passes on the tensor cores"}}


def d32_leg(n_sm):
    """The 32-dimensional case on one 512x512 frame shaped like the headline
    workload (131072 foreground pixels, d = 32): whole-frame time of the FP32
    and BF16 forms through ms_run, and one shift launch of 4096 seeds (the
    tensor-core form is two 16-dimensional halves). Algorithmic work: 4d flops
    per seed-pixel pair."""
    import torch

    import paper_2007_14283_gb300 as ms
    import synth
    f = synth.frame_c2(seed=0, d=32)
    e = torch.from_numpy(f.emb).cuda()
    m = torch.from_numpy(f.mask).cuda()
    out = {"config": "512x512 frame, 131072 foreground pixels, d=32 (synthetic vMF cells)"}
    for name, prec in (("fp32", ms.MS_FP32), ("bf16", ms.MS_BF16)):
        ts = []
        for rep in range(3):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            res = ms.cluster(e, m, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            if rep:
                ts.append(e0.elapsed_time(e1))
        cfg = ms.ms_config_default(dim=32, precision=prec)
        st_ms = []
        for rep in range(5):
            ctx = ms.ms_create(cfg, e, m)
            ms.ms_profile(ctx, True)
            seeded = ms.ms_seed_batch(ctx, 4096)
            try:
                ms.ms_iterate(ctx, 1)
            except ms.MsError as err:
                if err.status != ms.MS_ERR_NOT_CONVERGED:
                    raise
            st_ms.append(ms.ms_stats_get(ctx)["shift_ms"])
            ctx.close()
        t = statistics.median(st_ms[1:])
        out[name] = {"frame_ms": statistics.median(ts), "modes": int(res.modes.shape[0]),
                     "shift_4096_seeds_ms": t,
                     "shift_tflops": 4.0 * 32 * N_FG * seeded / (t * 1e-3) / 1e12}
    return out


def kernel_variants_leg(n_sm, clk):
    """Other distances and profiles (ms_kernel_shift) at the differentiable
    configuration's size: N = 65536 vectors, M = 1024 seeds, d = 16, T = 10.
    CUDA events, median of 3 after a warm-up. Bound: FP32 FMA; per seed-vector
    pair and step 2d flops for the distance (cosine: d FMAs of the dot
    product; Euclidean: a subtraction and an FMA per component) and 2d for
    the weighted sum."""
    import torch

    import paper_2007_14283_gb300 as ms
    import synth
    prob = synth.vmf_problem_c5(seed=0, N=65536, M=1024, K=32)
    P = torch.from_numpy(prob["P"]).cuda()
    X0 = torch.from_numpy(prob["X0"]).cuda()
    stream = torch.cuda.current_stream()
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    out = []
    names = {ms.MS_DIST_COSINE: "cosine", ms.MS_DIST_EUCLID: "euclidean"}
    pnames = {ms.MS_PROFILE_FLAT: "flat", ms.MS_PROFILE_EPANECHNIKOV: "epanechnikov",
              ms.MS_PROFILE_GAUSSIAN: "gaussian"}
    for dist, h in ((ms.MS_DIST_COSINE, 0.1), (ms.MS_DIST_EUCLID, 0.45)):
        for prof in (ms.MS_PROFILE_FLAT, ms.MS_PROFILE_EPANECHNIKOV, ms.MS_PROFILE_GAUSSIAN):
            ms.ms_kernel_shift(P, X0, dist, prof, h, 10)
            ts = []
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ms.ms_kernel_shift(P, X0, dist, prof, h, 10)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            t = statistics.median(ts)
            tf = 4 * 16 * 65536 * 1024 * 10 / (t * 1e-3) / 1e12
            out.append({"distance": names[dist], "profile": pnames[prof], "h": h, "ms": t,
                        "achieved_tflops": tf, "frac_fp32_peak": tf / peak})
    return {"config": "N=65536, M=1024, d=16, T=10 (synthetic vMF cells)", "rows": out,
            "peak_tflops": peak, "algorithmic": "4d flops per seed-vector pair and step"}


def video_leg(n_frames=16):
    """Video form on a drifting 512x512 sequence (the C2 frame recipe; cell means
    drift 0.02 rad per frame): BF16, the seed count N carried from frame to
    frame and the next frame bound on a second stream (ms_video_run), against
    the same frames clustered independently (ms_create + ms_run, N restarting at
    N_initial). Frames/s from CUDA events on the stream, after one warm-up pass."""
    import torch

    import paper_2007_14283_gb300 as ms
    import synth
    fs = synth.video_sequence(seed=11, T=n_frames)
    embs = [torch.from_numpy(f.emb).cuda() for f in fs]
    masks = [torch.from_numpy(f.mask).cuda() for f in fs]
    labels = [torch.empty(f.emb.shape[0], dtype=torch.int32, device="cuda") for f in fs]
    cfg = ms.ms_config_default(dim=DIM, precision=ms.MS_BF16)
    stream = torch.cuda.current_stream()

    def timed_s(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    def video(restart=0):
        c = ms.ms_config_default(dim=DIM, precision=ms.MS_BF16, video_restart=restart)
        with ms.ms_video_create(c, max(f.emb.shape[0] for f in fs)) as v:
            _, n_start, n_modes = ms.ms_video_run(v, embs, masks, labels)
        return n_start, n_modes

    def independent():
        for t, (e, m, lab) in enumerate(zip(embs, masks, labels)):
            c = ms.ms_config_default(dim=DIM, precision=ms.MS_BF16, frame_id=t)
            ctx = ms.ms_create(c, e, m)
            try:
                ms.ms_run(ctx, lab)
            finally:
                ctx.close()
    tv, (n_start, n_modes) = timed_s(video)
    tr, _ = timed_s(lambda: video(1))
    ti, _ = timed_s(independent)
    return {"config": f"{n_frames} consecutive 512x512 frames (131072 foreground px, 60 cells drifting 0.02 rad "
                      "per frame), BF16 single-frame form",
            "video_frames_per_s": n_frames / tv, "video_restart_frames_per_s": n_frames / tr,
            "independent_frames_per_s": n_frames / ti,
            "n_start": n_start, "modes_per_frame": sum(n_modes) / max(1, len(n_modes)),
            "api": "ms_video_run (N carried, next frame bound on a second stream; video_restart = 1: N back at "
                   "N_initial each frame) vs ms_create + ms_run per frame"}


PAPER_TABLE1_OURS_S = {1000: 1.624, 2000: 1.618, 5000: 1.664, 10000: 1.698, 20000: 1.747, 50000: 1.892,
                       100000: 2.107, 200000: 2.692}  # Table 1, "Ours" (half a Tesla K80), context only


def _cluster_timed(ms, emb, mask, reps=3, **cfg):
    """Median seconds of ms_create + ms_run on device-resident inputs (CUDA
    events, after one warm-up), with the last run's labels, modes and counters."""
    import torch
    stream = torch.cuda.current_stream()
    ts, res = [], None
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ms.cluster(emb, mask, **cfg)
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(ts), res


def run_suite(args):
    """The paper's simulation suite on synthetic inputs (Sec. 4.2 Table 1,
    Appendix A, Sec. 4.3 Tables 3-4), one JSON line.

    table1: n = 1K..200K points, 18-d, 10 orthogonal/opposite blob clusters,
      sigma = 0.01, h = 0.1 (c = 0.9): GPU seconds per frame (FP32 form; d = 18)
      and workspace MB beside the paper's own "Ours" row, the oracle's seconds on
      the host cores up to 20K points, and label agreement with the truth.
    appendix_a: 1000 x 1000 x 18 frames of 8 discs (diameter 250) at growing
      overlap, P = 0.95, L = 2, H = 8: modes found, label agreement with the
      truth, rounds, seeds, seconds.
    tables_3_4: a drifting 512 x 512 sequence through the video form (N carried
      across frames) with N_initial in {64, 128, 256} and H in {4, 8, 16}:
      seconds per frame."""
    import numpy as np
    import torch

    import oracle
    import paper_2007_14283_gb300 as ms
    import synth
    from tests.parity_util import matched_agreement
    ms.load()
    torch.cuda.set_device(0)
    out = {"suite": True}
    rows = []
    for n in (1000, 2000, 5000, 10000, 20000, 50000, 100000, 200000):
        emb, truth = synth.orthogonal_blobs(seed=n, n=n, d=18, K=10, sigma=0.01)
        e = torch.from_numpy(emb).cuda()
        t, res = _cluster_timed(ms, e, None, precision=ms.MS_FP32)
        lab = res.labels.cpu().numpy()
        row = {"n": n, "gpu_s": t, "gpu_workspace_mb": res.stats["workspace_bytes"] / 2 ** 20,
               "modes": res.stats["n_modes"], "label_agreement_truth": matched_agreement(truth, lab),
               "paper_ours_s": PAPER_TABLE1_OURS_S[n]}
        if n <= 20000:
            t0 = time.perf_counter()
            ref = oracle.run(emb)
            row["oracle_s"] = time.perf_counter() - t0
            row["labels_equal_oracle"] = bool(np.array_equal(ref.labels, lab))
        rows.append(row)
    out["table1"] = {"rows": rows, "cores": host_threads(),
                     "data": "synth.orthogonal_blobs: 18-d, 10 clusters at +/- e_j, sigma 0.01"}
    arows = []
    for ov in (0.0, 0.1, 0.2, 0.3):
        f = synth.overlap_discs(seed=1, overlap=ov)
        e, m = torch.from_numpy(f.emb).cuda(), torch.from_numpy(f.mask).cuda()
        t, res = _cluster_timed(ms, e, m, reps=1, precision=ms.MS_FP32, P_target=0.95)
        fg = f.mask.astype(bool)
        arows.append({"overlap": ov, "fg_fraction": f.info["fg_fraction"], "modes": res.stats["n_modes"],
                      "label_agreement_truth": matched_agreement(f.truth[fg], res.labels.cpu().numpy()[fg]),
                      "rounds": res.stats["rounds"], "seeds": res.stats["seeds"], "gpu_s": t})
    out["appendix_a"] = {"rows": arows, "config": "1000x1000x18, 8 discs of diameter 250, no noise, P = 0.95"}
    fs = synth.video_sequence(seed=21, T=8)
    embs = [torch.from_numpy(f.emb).cuda() for f in fs]
    masks = [torch.from_numpy(f.mask).cuda() for f in fs]
    ab = []
    for key, vals in (("n_initial", (64, 128, 256)), ("H", (4.0, 8.0, 16.0))):
        for val in vals:
            cfg = ms.ms_config_default(dim=DIM, precision=ms.MS_BF16, **{key: val})
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with ms.ms_video_create(cfg, max(f.emb.shape[0] for f in fs)) as v:
                _, n_start, n_modes = ms.ms_video_run(v, embs, masks)
            torch.cuda.synchronize()
            ab.append({key: val, "s_per_frame": (time.perf_counter() - t0) / len(fs), "n_start": n_start,
                       "modes_per_frame": sum(n_modes) / len(n_modes)})
    out["tables_3_4"] = {"rows": ab, "config": "8 consecutive 512x512 frames (C2 recipe, 0.02 rad drift), "
                                               "video form, BF16"}
    print(json.dumps(out), flush=True)


def run_volume(args):
    """3D volume (the paper's stated 2D limitation, Sec. 5.3): 128 x 256 x 256
    voxels, half foreground (4.19M vectors), 400 ellipsoidal vMF cells, BF16
    single-frame form. Seconds per volume (CUDA events) and sampled checks:
    labels are the FP64 argmax over the GPU's modes, every sampled voxel is
    covered, modes are fixed points."""
    import numpy as np
    import torch

    import paper_2007_14283_gb300 as ms
    import synth
    ms.load()
    torch.cuda.set_device(0)
    f = synth.volume(seed=0)
    e, m = torch.from_numpy(f.emb).cuda(), torch.from_numpy(f.mask).cuda()
    t, res = _cluster_timed(ms, e, m, reps=1, precision=ms.MS_BF16)
    st = res.stats
    fg = np.flatnonzero(f.mask)
    rng = np.random.default_rng(0)
    idx = rng.choice(fg, size=2000, replace=False)
    P = f.emb[idx].astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    M = res.modes.cpu().numpy().astype(np.float64)
    M /= np.linalg.norm(M, axis=1, keepdims=True)
    S = P @ M.T
    lab = res.labels.cpu().numpy()[idx]
    top = np.sort(S, axis=1)
    safe = top[:, -1] - top[:, -2] > 1e-5
    out = {"volume": True, "shape": list(f.info["shape"]), "voxels": int(f.emb.shape[0]), "n_fg": int(fg.size),
           "gpu_s": t, "seconds_per_mvoxel_fg": t / (fg.size / 1e6), "modes": st["n_modes"],
           "rounds": st["rounds"], "seeds": st["seeds"], "seed_iters": st["seed_iters"],
           "workspace_gb": st["workspace_bytes"] / 2 ** 30,
           "sampled_labels_equal_fp64_argmax": float((np.argmax(S, axis=1)[safe] == lab[safe]).mean()),
           "sampled_covered": float((top[:, -1] >= 0.9 - 1e-6).mean())}
    print(json.dumps(out), flush=True)


def e2e_leg(args, runner, ws):
    """Frames/s through the host-buffer entry points (pinned buffers in, labels out)."""
    import torch
    ms = runner.ms
    frames = runner.frames
    h_embs = [torch.from_numpy(f.emb).pin_memory() for f in frames]
    h_masks = [torch.from_numpy(f.mask).pin_memory() for f in frames]
    h_labels = [torch.empty(f.emb.shape[0], dtype=torch.int32).pin_memory() for f in frames]
    h2d = sum(e.numel() * 4 + m.numel() for e, m in zip(h_embs, h_masks))
    d2h = sum(l.numel() * 4 for l in h_labels)

    def one():
        if runner.batched:
            ms.ms_batch_run_host(runner.batch, h_embs, h_masks, h_labels)
        else:
            for e, m, l in zip(h_embs, h_masks, h_labels):
                ms.ms_run_host(runner.cfg, e, m, l)
    one()
    torch.cuda.synchronize()
    barrier(ws)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    walls = []
    for _ in range(args.e2e_steps):
        w0 = time.perf_counter()
        one()
        walls.append(1e3 * (time.perf_counter() - w0))
    torch.cuda.synchronize()
    value, _ = whole_job_rate(args.e2e_steps * len(frames), time.perf_counter() - t0, ws)
    # one device-resident step right after, on the same clock state: the
    # difference to the host-buffer steps is the copies' share
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    runner.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    assert torch.equal(h_labels[0], runner.labels[0].cpu()), "host-buffer run disagrees with the device run"
    api = "ms_batch_run_host" if runner.batched else "ms_run_host"
    return {"value": value, "unit": "frames/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": api, "steps": args.e2e_steps, "step_wall_ms": walls,
            "device_step_ms_after": ev0.elapsed_time(ev1), "clocks": clk}


def phase_leg(runner):
    """One untimed extra step with the phase timers on (profiling level 2):
    where a step's time goes inside the graph, by phase (ncu does not look
    inside conditional graph bodies). Restores the shift timers alone."""
    import torch
    ms = runner.ms
    ms.ms_batch_profile(runner.batch, 2)
    ms.ms_batch_run(runner.batch)
    torch.cuda.synchronize()
    out = ms.ms_batch_phase_ms(runner.batch)
    ms.ms_batch_profile(runner.batch, 1)
    tot = sum(out.values())
    return {"ms": out, "share": {k: v / tot for k, v in out.items()} if tot > 0 else None,
            "note": "one extra untimed step with one-thread global-timer kernels between the graph's phases"}


def run_ours(args, rank, ws, local):
    import torch

    import paper_2007_14283_gb300 as ms
    ms.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    frames = c2_frames(rank, args.frames)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    main = Runner(ms, args.form, frames, dev, eager=args.eager,
                  autotune=args.form.endswith("batched") and not args.no_autotune)
    clocks = Clocks(local)
    clocks.start()
    step_ms, tot = timed(main, args.steps, args.warmup, ws, flush, stream)
    clk = clocks.stop()
    value, t_total = whole_job_rate(tot["frames"], sum(step_ms) / 1e3, ws)
    launches = int(reduce_over_ranks(tot["launches"], ws, "sum"))   # every rank takes part
    roofline = roofline_of(args.form, tot, step_ms, clk, n_sm)
    forms = {args.form: {"value": value, "frames_per_step": args.frames, "steps": args.steps,
                         "ms_per_frame": sum(step_ms) / max(1, tot["frames"]),
                         "roofline_frac": roofline["frac"]}}
    e2e = e2e_leg(args, main, ws) if args.e2e_steps > 0 else None
    phases = phase_leg(main) if main.batched and not args.eager else None

    for other in [f for f in args.compare.split(",") if f and f != args.form]:
        r = Runner(ms, other, frames[: args.compare_frames], dev)
        c_clocks = Clocks(local)
        c_clocks.start()
        sm_, tt = timed(r, args.compare_steps, 1, ws, flush, stream)
        c_clk = c_clocks.stop()
        v, _ = whole_job_rate(tt["frames"], sum(sm_) / 1e3, ws)
        rf = roofline_of(other, tt, sm_, c_clk, n_sm)
        same = all(torch.equal(a, b) for a, b in zip(r.labels, main.labels)) if other.split("-")[0] == \
            args.form.split("-")[0] else None
        forms[other] = {"value": v, "frames_per_step": len(r.frames), "steps": args.compare_steps,
                        "ms_per_frame": sum(sm_) / max(1, tt["frames"]), "roofline_frac": rf["frac"],
                        "roofline_bound": rf["bound"], "labels_identical_to_headline": same,
                        "clocks_sm_mhz": c_clk.get("sm_mhz")}
        r.close()

    # The untimed legs below run on rank 0 of a one-GPU run only: no collective
    # may sit inside them, and with N > 1 the other GPUs would wait idle.
    extras = rank == 0 and ws == 1
    vmf = None
    if extras and not args.no_vmf:
        vmf = vmf_leg(n_sm, clk)
    video = None
    if extras and args.video_frames > 0:
        video = video_leg(args.video_frames)
    kvar, d32 = None, None
    if extras and not args.no_vmf:
        kvar = kernel_variants_leg(n_sm, clk)
        d32 = d32_leg(n_sm)
    cpu, parity = None, None
    if extras and args.cpu != "none":
        import oracle
        if args.cpu == "full":
            f0 = frames[0]
            t0 = time.perf_counter()
            ref = oracle.run(f0.emb, f0.mask)
            dt = time.perf_counter() - t0
            cpu = {"value": 1.0 / dt, "unit": "frames/s", "cores": host_threads(), "kind": "oracle",
                   "sample": f"one full frame (frame 0 of the step): every OSOP round, merge, coverage and "
                             f"labelling in FP64, {dt:.1f} s"}
            per_frame = c2_seed_iters_per_frame()
            if per_frame and args.cpu_runs > 0:
                # the bounded seed sample, median of cpu_runs runs on every core and one run on one core
                rates = []
                for _ in range(args.cpu_runs):
                    sdt, ssi = oracle_sample(f0, args.cpu_seeds // 4)
                    rates.append(1.0 / (sdt / ssi * per_frame))
                sdt1, ssi1 = oracle_sample_single_core(args.cpu_seeds // 8)
                cpu["sample_median"] = {
                    "value": statistics.median(rates), "runs": len(rates), "cores": host_threads(),
                    "sample": f"{args.cpu_seeds // 4} seeds shifted to the gamma stop, scaled by the oracle's "
                              f"{int(per_frame)} seed-iterations per frame; merge/cover/label not included"}
                cpu["single_core"] = {
                    "value": 1.0 / (sdt1 / ssi1 * per_frame), "cores": 1,
                    "sample": f"{args.cpu_seeds // 8} seeds ({ssi1} seed-iterations, {sdt1:.1f} s) on one core, "
                              f"scaled likewise"}
            # the small single-frame configuration (64 x 64, 4096 unit vectors, 8 vMF clusters), whole
            import synth
            c1 = synth.frame_c1(seed=0)
            c1_runs = []
            for _ in range(3):
                t1 = time.perf_counter()
                oracle.run(c1.emb)
                c1_runs.append(time.perf_counter() - t1)
            cpu["c1_frame"] = {"seconds_per_frame": statistics.median(c1_runs), "runs": 3, "cores": host_threads(),
                               "sample": "one 64x64 frame (4096 pixels, d=16, 8 vMF clusters), every step of the "
                                         "method in FP64; median of 3"}
            match, how, err, bg_ok = label_match(main.labels[0].cpu().numpy(), ref.labels, main.modes(0),
                                                 ref.modes)
            parity = {"frame": 0, "label_match": match, "method": how, "mode_err_max": err,
                      "background_identical": bg_ok, "modes_gpu": int(main.modes(0).shape[0]),
                      "modes_oracle": int(ref.modes.shape[0])}
        else:
            per_frame = c2_seed_iters_per_frame()
            dt, si = oracle_sample(frames[0], args.cpu_seeds)
            if per_frame:
                cpu = {"value": 1.0 / (dt / si * per_frame), "unit": "frames/s", "cores": host_threads(),
                       "kind": "oracle",
                       "sample": f"{args.cpu_seeds} seeds of frame 0's seed order shifted to the gamma stop "
                                 f"({si} seed-iterations, {dt:.1f} s), scaled by the oracle's {int(per_frame)} "
                                 f"seed-iterations per full frame; merge/cover/label not included"}
    main.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16+f32" if args.form.startswith("bf16") else "f32",
                "data": "synthetic vMF frames shaped like 512x512 microscopy (seeded generator)",
                "config": {"workload": WORKLOAD, "form": args.form + (" (eager launches)" if args.eager else ""),
                           "frames_per_step": args.frames,
                           "l2": "flushed (256 MB write) before every step; inputs also exceed L2",
                           "parallelism": f"replicas x{ws}",
                           "seed_iters_per_frame": tot["seed_iters"] / max(1, tot["frames"]),
                           "modes_per_frame": tot["modes"] / max(1, tot["frames"]),
                           "graph_passes_per_step": tot.get("passes", 0) / max(1, args.steps),
                           "autotune": main.tuning,
                           "fp32_rechecked_pair_fraction": tot.get("band_pairs", 0) /
                           max(1.0, float(tot["seed_iters"]) * N_FG)},
                "roofline": roofline, "batch_phases": phases, "forms": forms, "smooth_kernel": vmf, "kernel_variants": kvar, "d32": d32,
                "video": video,
                "parity_vs_oracle": parity,
                "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)


def run_shift_only(args):
    """One shift launch (one iteration of the shift loop of Algorithm 2) of a fixed seed
    batch through the public API: the dominant kernel alone, with a known
    number of seed-iterations per launch."""
    import torch

    import paper_2007_14283_gb300 as ms
    ms.load()
    torch.cuda.set_device(0)
    f = c2_frames(0, 1)[0]
    e = torch.from_numpy(f.emb).cuda()
    m = torch.from_numpy(f.mask).cuda()
    prec = ms.MS_BF16 if args.form.startswith("bf16") else ms.MS_FP32
    cfg = ms.ms_config_default(dim=DIM, precision=prec, tc_shape=args.tc_shape)
    times = []
    for rep in range(args.warmup + args.steps):
        ctx = ms.ms_create(cfg, e, m)
        ms.ms_profile(ctx, True)
        seeded = ms.ms_seed_batch(ctx, args.shift_only)
        try:
            ms.ms_iterate(ctx, 1)
        except ms.MsError as err:  # one iteration rarely converges a seed
            if err.status != ms.MS_ERR_NOT_CONVERGED:
                raise
        st = ms.ms_stats_get(ctx)
        ctx.close()
        if rep >= args.warmup:
            times.append(st["shift_ms"])
    t = statistics.median(times)
    flops = 4.0 * DIM * N_FG * seeded
    print(json.dumps({"shift_only": True, "form": args.form, "tc_shape": args.tc_shape, "seeds": seeded, "n": N_FG,
                      "median_ms": t, "algorithmic_tflops": flops / (t * 1e-3) / 1e12}), flush=True)


def main():
    args = parse()
    if args.shift_only > 0:
        run_shift_only(args)
        return
    if args.suite:
        run_suite(args)
        return
    if args.volume:
        run_volume(args)
        return
    if args.vmf_only:
        import torch

        import paper_2007_14283_gb300 as ms
        ms.load()
        torch.cuda.set_device(0)
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        print(json.dumps({"vmf_only": True, **vmf_leg(n_sm, {})}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, int(os.environ.get("RANK", "0")))
        return
    rank, ws, local = dist_setup()
    run_ours(args, rank, ws, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
