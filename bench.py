"""Benchmark of the Gaussian-mixture interpolation hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmi|reference]

Headline workload (one "step" = one forward pass, binning included, of one
synthetic image): a 512^2 source grid jittered by U[-0.5, 0.5] px, upsampled
x2 to 1024 x 1024 x 3 float32 with sigma = 1 px, exact mode, k = 6.  ``value``
is interpolated output Mpix/s (H*W per step, all ranks) through
``gmi.interpolate(..., graph=True)`` (the four kernels replayed as one CUDA
graph), timed with CUDA events per step on the launching stream with L2
flushed (256 MB write) between steps; ``plain_launch`` is the same without
graph replay; ``e2e`` repeats the measurement through the host-buffer call
(``gmi.interpolate_host``, the C ABI's gmi_forward_host: pinned inputs
uploaded, the kernels, the image downloaded, replayed as one CUDA graph) with
the host<->device copies inside the timed region, the steps queued behind a
device spin as the headline's are; ``e2e.host_paced`` gives the same calls
issued one at a time, the host's per-call time inside the steps.

Further objects on the same line: the dominant kernel's roofline, the FP64
oracle's CPU throughput, SM clocks sampled during the timed region and, as
they are built, the batched, fwd+bwd and serving workloads.

``--impl reference`` times the FP64 oracle (the CPU reference of this build)
on a bounded pixel sample of the same workload, per step.

Multi-GPU: replicas only (each rank runs the same workload on its own GPU;
weak scaling); ranks synchronise with a barrier and the max time is reported.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
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

METRIC = "interpolated Mpix/s (batched+served vs plain launch); p50/p99 latency; fwd+bwd Mpix/s"
WORKLOAD = ("upsample_1024: 512^2 source grid jittered U[-0.5,0.5] px -> 1024x1024x3 float32, "
            "sigma=1.0 px, exact mode, k=6, values from a smooth random field")
L2_FLUSH_BYTES = 256 << 20
FP32_PER_SM_CLK = 128    # FP32 FMA results per SM per clock (4 x 32 lanes; measured ~123)
SFU_PER_SM_CLK = 32      # ex2 results per SM per clock on B300 (measured 32.0)
FP32_OPS_PER_PAIR = 8    # per algorithmic pair: ~4 for d^2, 1 exponent scale, C + 1 = 4 accumulations (C = 3)
SM_MAX_MHZ = 2032.0      # B300 maximum SM clock
LAUNCHES_PER_FORWARD = 4  # headline forward: count, one-launch scan, scatter+plan, near (no far kernel: none queued)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gmi", choices=["gmi", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: the default micro-tile and bin rule instead of the autotuned ones (for ncu "
                         "captures, whose serialised timings mislead the autotuner)")
    ap.add_argument("--only", choices=["batched", "fwd_bwd", "serving", "reconstruction", "point_optimization",
                                       "per_point_sigma"],
                    help="run only this secondary workload and print its object (for profiling it)")
    return ap.parse_args()


def replica_throughput(pixels_per_step: int, steps: int, world: int, t_max_ms: float) -> float:
    """Whole-job Mpix/s of `world` replicas that each ran `steps` steps of
    `pixels_per_step` output pixels, the slowest taking t_max_ms."""
    return pixels_per_step * steps * world / (t_max_ms * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class Dist:
    """Barrier and max-reduce over ranks when launched under torchrun: NCCL
    between GPUs, gloo for CPU devices (the multi-rank tests).  Replicas only:
    the workload does not shard, so no data crosses ranks."""

    def __init__(self, world, device):
        self.world = world
        self.device = device
        if world > 1:
            import torch.distributed as dist
            if device.type == "cuda":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, v: float) -> float:
        if self.world == 1:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_pairs(im, k=6.0):
    """Pairs (pixel, point) with d^2 <= m_q + k^2 sigma^2 (the radius rule of
    exact mode): the work the method must do, counted with a k-d tree."""
    from scipy.spatial import cKDTree
    yy, xx = np.meshgrid(np.arange(im.H) + 0.5, np.arange(im.W) + 0.5, indexing="ij")
    q = np.stack([xx.ravel(), yy.ravel()], 1)
    tree = cKDTree(im.points.astype(np.float64))
    d, _ = tree.query(q, workers=-1)
    rad = np.sqrt(d * d + (k * im.sigma) ** 2) * (1 + 1e-9)
    cnt = tree.query_ball_point(q, rad, return_length=True, workers=-1)
    return int(np.sum(cnt))


def near_kernel_traffic():
    """DRAM bytes per launch of the near kernel from the committed ncu summary,
    or None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "near_kernel_upsample_1024.txt")
    src = os.path.join(ROOT, "paper_2012_13257_b300", "csrc", "gather_staged.cu")
    if not os.path.exists(path):
        return None
    want = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    kv = {}
    for line in open(path):
        if ":" in line:
            k_, v_ = line.split(":", 1)
            kv[k_.strip()] = v_.strip()
    if kv.get("source_sha256_16") != want:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(im, target_s=12.0):
    """FP64 oracle (as it stands) on a bounded random pixel sample of the
    workload, on this host's cores; Mpix/s extrapolates exactly because every
    pixel costs the same N pair evaluations."""
    import oracle
    rng = np.random.default_rng(123)
    n = 64
    while True:
        pix = rng.integers(0, im.H * im.W, n)
        t0 = time.perf_counter()
        oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)
        t = time.perf_counter() - t0
        if t >= 10.0 or n >= 1 << 20:
            break
        n = int(n * min(8.0, max(1.2, target_s / max(t, 1e-3))))
    return {"value": n / t / 1e6, "unit": "Mpix/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d random pixels of the %dx%d image (%d points each), %.1f s" % (n, im.H, im.W, im.N, t)}


def pair_estimate(imgs, k=6.0, frac=16, seed=0):
    """Algorithmic pairs of a batch, estimated on a 1/frac random pixel sample
    of every image (k-d tree counts as in algorithmic_pairs)."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    total = 0.0
    for im in imgs:
        if im.N == 0:
            continue
        n = max(64, im.H * im.W // frac)
        pix = rng.integers(0, im.H * im.W, n)
        q = np.stack([pix % im.W + 0.5, pix // im.W + 0.5], 1)
        tree = cKDTree(im.points.astype(np.float64))
        d, _ = tree.query(q, workers=-1)
        cnt = tree.query_ball_point(q, np.sqrt(d * d + (k * im.sigma) ** 2) * (1 + 1e-9), return_length=True,
                                    workers=-1)
        total += float(np.mean(cnt)) * im.H * im.W
    return total


def prequeue(steps, per_step_s=400e-6):
    """A device spin long enough for the host to enqueue `steps` steps behind
    it, so that no timed step waits for the host inside its events (the spin
    runs before the first start event, outside the timed region).  Returns an
    event recorded right after the spin: if it has already completed once the
    host has queued the timed steps, the host did not keep ahead of the device
    (see queued_in_time)."""
    import torch
    torch.cuda._sleep(int(steps * per_step_s * SM_MAX_MHZ * 1e6))
    ev = torch.cuda.Event()
    ev.record()
    return ev


def queued_in_time(spin_done) -> bool:
    """True while the device is still in the spin, i.e. every timed step was
    enqueued before the device reached it."""
    return not spin_done.query()


def step_stats(ms):
    """Spread of the per-step times behind ms_per_step (their mean): median,
    min and max in ms (this rank's)."""
    s = sorted(ms)
    return {"median": s[len(s) // 2], "min": s[0], "max": s[-1]} if s else None


def timed_steps(fn, steps, flush, stream, queued=False, info=None):
    """Per-step CUDA-event times (ms) with an untimed L2 flush before each
    step; with `queued`, the steps are enqueued behind a device spin (device
    time only; otherwise a slow host can leave the device idle inside a
    step's events).  If the host fell behind the spin, the queued run is
    repeated once with a spin four times as long; `info` (a dict) receives
    queue_ok (whether the steps kept ahead of the device)."""
    import torch
    per_step = 400e-6
    for attempt in range(2 if queued else 1):
        st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        spin = None
        if queued:
            spin = prequeue(steps + 1, per_step)
            flush.zero_()
            fn()   # one more warm-up step in the queue, so no timed step starts the queued run
        for k in range(steps):
            flush.zero_()
            st[k].record(stream)
            fn()
            en[k].record(stream)
        ok = queued_in_time(spin) if spin is not None else None
        torch.cuda.synchronize()
        if ok is not False:
            break
        per_step *= 4
    if info is not None and queued:
        info["queue_ok"] = ok
    return [a.elapsed_time(b) for a, b in zip(st, en)]


def e2e_pipelined(gmi, im, hP, hV, steps, D, world):
    """End to end with consecutive steps overlapped, through the same public
    host-buffer call as ``e2e`` (``gmi.interpolate_host``, the C ABI's
    gmi_forward_host, graph replay): the steps alternate between two CUDA
    streams, each with its own workspace and pinned output buffer, so one
    step's download overlaps the next one's upload and kernels (the copy
    engines of the two directions run side by side).  Every step still
    uploads its inputs from pinned host memory and downloads its image.
    Timed from the first call to the last download (no L2 flush: the steps
    overlap)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    hO = [torch.empty((im.H, im.W, im.C), dtype=torch.float32).pin_memory() for _ in range(2)]

    def run(k_steps, first=None, last=None):
        base = torch.cuda.current_stream(dev)
        if first is not None:
            first.record(base)
        for s in streams:
            s.wait_stream(base)
        for k in range(k_steps):
            j = k % 2
            with torch.cuda.stream(streams[j]):
                gmi.interpolate_host(hP, hV, im.sigma, im.H, im.W, out=hO[j], graph=True)
        for s in streams:
            base.wait_stream(s)
        if last is not None:
            last.record(base)

    run(4)
    torch.cuda.synchronize()
    D.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run(steps, t0, t1)
    torch.cuda.synchronize()
    total = D.max(t0.elapsed_time(t1))
    return {"value": replica_throughput(im.H * im.W, steps, world, total), "unit": "Mpix/s",
            "h2d_bytes_per_step": int(hP.numel() * 4 + hV.numel() * 4), "d2h_bytes_per_step": int(hO[0].numel() * 4),
            "ms_per_step": total / steps,
            "note": "gmi_forward_host on two alternating streams: uploads, kernels and downloads of consecutive "
                    "steps overlap"}


def _sig(v, digits=4):
    """A float rounded to `digits` significant digits (short JSON)."""
    if isinstance(v, float) and v == v and v not in (float("inf"), float("-inf")) and v != 0.0:
        from math import floor, log10
        return round(v, digits - 1 - int(floor(log10(abs(v)))))
    return v


def summary(d, keys, **sub):
    """The named keys of a result dict, rounded, with the named keys of its
    sub-objects; an error result passes through."""
    if not isinstance(d, dict) or "error" in d:
        return d
    out = {k: _sig(d[k]) for k in keys if k in d}
    for name, ks in sub.items():
        if isinstance(d.get(name), dict):
            out[name] = {k: _sig(d[name][k]) for k in ks if k in d[name]}
    return out


def e2e_breakdown(gmi, im, hP, hV, hO, steps, flush, stream):
    """Where the end-to-end step's time goes: the same step as four pieces on
    one stream with events between them (pinned upload of points and values,
    the graph-replayed forward, the download of the image), L2 flushed before
    each step.  The pieces are timed separately from the e2e number above
    (which runs them as one captured graph through gmi_forward_host)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    dP = torch.empty(hP.shape, dtype=hP.dtype, device=dev)
    dV = torch.empty(hV.shape, dtype=hV.dtype, device=dev)
    dO = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)

    def once(ev=None):
        if ev:
            ev[0].record(stream)
        dP.copy_(hP, non_blocking=True)
        dV.copy_(hV, non_blocking=True)
        if ev:
            ev[1].record(stream)
        gmi.interpolate(dP, dV, im.sigma, im.H, im.W, out=dO, graph=True)
        if ev:
            ev[2].record(stream)
        hO.copy_(dO, non_blocking=True)
        if ev:
            ev[3].record(stream)
    for _ in range(3):
        once()
    torch.cuda.synchronize()
    acc = [0.0, 0.0, 0.0]
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        once(ev)
        torch.cuda.synchronize()
        for i in range(3):
            acc[i] += ev[i].elapsed_time(ev[i + 1])
    up, comp, down = (a / steps for a in acc)
    return {"upload_ms": up, "compute_ms": comp, "download_ms": down, "sum_ms": up + comp + down,
            "upload_gbs": (hP.numel() + hV.numel()) * 4 / (up * 1e-3) / 1e9,
            "download_gbs": hO.numel() * 4 / (down * 1e-3) / 1e9}


def bench_batched(dev, steps, warmup, flush, stream, autotune=True):
    """64 uneven clustered images (sides log-uniform in [128, 1024],
    N = 0.25 H W, sigma U[0.5, 2]): one batched graph launch per step versus
    64 plain single-image launches, autotuned bin sizes and micro-tile."""
    import torch
    import paper_2012_13257_b300 as gmi
    from paper_2012_13257_b300.autotune import Autotuner, bucket
    import workloads as wl
    imgs = wl.batched_uneven()
    dimgs = [{"points": torch.as_tensor(im.points, device=dev), "values": torch.as_tensor(im.values, device=dev),
              "sigma": im.sigma, "H": im.H, "W": im.W,
              "out": torch.empty((im.H, im.W, 3), dtype=torch.float32, device=dev)} for im in imgs]
    # autotune one representative image per bucket (the largest), in a scratch cache
    tuner = Autotuner(path=os.path.join(tempfile.gettempdir(), "gmi_autotune_bench.json"))
    rep = {}
    for i, im in enumerate(imgs):
        key = bucket(im.sigma, im.N / float(im.H * im.W), 3)
        if key not in rep or im.H * im.W > imgs[rep[key]].H * imgs[rep[key]].W:
            rep[key] = i
    t0 = time.perf_counter()
    # without tuning: the 4x4 micro-tile, the automatic bin rule and the staged gather
    work, gwork = ({1: 1}, {"staged": 1}) if not autotune else ({}, {})
    for key, i in (rep.items() if autotune else ()):
        best, _ = tuner.tune(dimgs[i]["points"], dimgs[i]["values"], imgs[i].sigma, imgs[i].H, imgs[i].W,
                             reps=3, warmup=1, save=False)
        px = sum(im.H * im.W for im in imgs if bucket(im.sigma, im.N / float(im.H * im.W), 3) == key)
        work[best["variant"]] = work.get(best["variant"], 0) + px
        gwork[best["gather"]] = gwork.get(best["gather"], 0) + px
        for j, im in enumerate(imgs):
            if bucket(im.sigma, im.N / float(im.H * im.W), 3) == key:
                dimgs[j]["bin_px"] = best["bin_px"]
    # one launch takes one micro-tile and one gather: those the most pixels' buckets chose
    variant = max(work, key=work.get)
    gather = max(gwork, key=gwork.get)
    tune_s = time.perf_counter() - t0
    plan = gmi.BatchPlan(64, sum(im.N for im in imgs), sum(im.H * im.W for im in imgs), 3, variant=variant,
                         gather=gather)
    for _ in range(max(3, warmup)):
        plan.forward(dimgs, use_graph=True)
    torch.cuda.synchronize()
    qinfo = {}
    tb = timed_steps(lambda: plan.forward(dimgs, use_graph=True), steps, flush, stream, queued=True, info=qinfo)
    # per-stage times of the same batched forward (events around each stage,
    # no graph), for the near kernel's roofline
    from paper_2012_13257_b300 import _lib
    L = _lib.load()
    L.gmi_profile_enable(1)
    L.gmi_profile_read(None, None, 1)
    torch.cuda._sleep(int(steps * 2e-3 * SM_MAX_MHZ * 1e6))
    for _ in range(steps):
        flush.zero_()
        plan.forward(dimgs, use_graph=False)
    torch.cuda.synchronize()
    st_ms = (ctypes.c_double * 4)()
    st_n = (ctypes.c_int * 4)()
    L.gmi_profile_read(st_ms, st_n, 1)
    L.gmi_profile_enable(0)
    stage = {name: (st_ms[i] / st_n[i] if st_n[i] else None) for i, name in enumerate(_lib.STAGES)}

    def plain():
        for d in dimgs:
            gmi.interpolate(d["points"], d["values"], d["sigma"], d["H"], d["W"], out=d["out"], gather=gather)
    for _ in range(2):
        plain()
    torch.cuda.synchronize()
    tp = timed_steps(plain, steps, flush, stream)
    px = sum(im.H * im.W for im in imgs)
    pairs = pair_estimate(imgs)
    mb = px / (sum(tb) / steps * 1e-3) / 1e6
    mp = px / (sum(tp) / steps * 1e-3) / 1e6
    plan.close()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_PER_SM_CLK / FP32_OPS_PER_PAIR * SM_MAX_MHZ * 1e6 / 1e9
    near_ms = stage["near"]
    achieved = pairs / (near_ms * 1e-3) / 1e9 if near_ms else None
    return {"value": mb, "unit": "Mpix/s", "ms_per_step": sum(tb) / steps, "plain_per_image_value": mp,
            "plain_ms_per_step": sum(tp) / steps, "speedup_vs_plain": mb / mp, "images": len(imgs),
            "pixels": px, "points": int(sum(im.N for im in imgs)), "queue_ok": qinfo.get("queue_ok"),
            "pairs_est": pairs, "pair_rate_gpair_s": pairs / (sum(tb) / steps * 1e-3) / 1e9,
            "stage_ms": stage,
            "roofline": {"bound": "alu", "kernel": "near gather (batched)", "launch_ms": near_ms,
                         "pairs_per_launch": pairs, "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                         "frac": achieved / peak if achieved else None,
                         "frac_step": pairs / (sum(tb) / steps * 1e-3) / 1e9 / peak,
                         "peak_basis": "FP32 pipe at %.0f MHz, %d FP32 ops per algorithmic pair" %
                                       (SM_MAX_MHZ, FP32_OPS_PER_PAIR)},
            "autotune": {"variant": variant, "gather": gather, "buckets": len(rep), "tune_s": tune_s,
                         "on": bool(autotune)},
            "workload": "64 images, sides log-uniform [128,1024], N=0.25HW clustered (8 clusters), "
                        "sigma U[0.5,2], RGB f32; one CUDA-graph batched launch per step vs 64 plain launches"}


def bench_fwd_bwd(dev, steps, warmup, flush, stream):
    """16 images 512x512x3 from 65,536 clustered points each, sigma = 1:
    forward + backward (values, positions, sigma) through the batched
    torch.autograd.Function (one graph-replayed forward launch and one
    batched backward for all 16 images); the same through the per-image
    autograd op for comparison."""
    import torch
    import paper_2012_13257_b300 as gmi
    import workloads as wl
    imgs, grad = wl.fwd_bwd_512()
    P = [torch.as_tensor(im.points, device=dev).requires_grad_(True) for im in imgs]
    V = [torch.as_tensor(im.values, device=dev).requires_grad_(True) for im in imgs]
    S = [torch.tensor(im.sigma, dtype=torch.float32, device=dev, requires_grad=True) for im in imgs]
    G = torch.as_tensor(grad, device=dev)
    plan = gmi.BatchPlan(len(imgs), sum(im.N for im in imgs), sum(im.H * im.W for im in imgs), 3)
    sizes = [(im.H, im.W) for im in imgs]

    Ps = torch.stack([p.detach() for p in P]).requires_grad_(True)
    Vs = torch.stack([v.detach() for v in V]).requires_grad_(True)
    Ss = torch.tensor([im.sigma for im in imgs], dtype=torch.float32, device=dev, requires_grad=True)
    H, W = imgs[0].H, imgs[0].W

    def step():
        out = gmi.gmi_interpolate_stacked(plan, Ps, Vs, Ss, H, W)
        out.backward(G)

    def step_list():
        outs = gmi.gmi_interpolate_batch(plan, P, V, S, sizes)
        torch.autograd.backward(outs, [G[b] for b in range(len(imgs))])

    def step_single():
        for b, im in enumerate(imgs):
            gmi.gmi_interpolate(P[b], V[b], S[b], im.H, im.W).backward(G[b])
    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    t = timed_steps(step, steps, flush, stream)
    for _ in range(2):
        step_single()
        step_list()
    torch.cuda.synchronize()
    t1 = timed_steps(step_single, max(3, steps // 4), flush, stream)
    t2 = timed_steps(step_list, max(3, steps // 4), flush, stream)
    plan.close()
    px = sum(im.H * im.W for im in imgs)
    return {"value": px / (sum(t) / steps * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_step": sum(t) / steps,
            "per_image_autograd_value": px / (sum(t1) / len(t1) * 1e-3) / 1e6,
            "per_image_ms_per_step": sum(t1) / len(t1),
            "list_batched_autograd_value": px / (sum(t2) / len(t2) * 1e-3) / 1e6,
            "images": len(imgs), "pixels": px,
            "workload": "16 x 512x512x3 f32 from 65,536 clustered points, sigma=1, upstream N(0,1); "
                        "forward + backward w.r.t. values, positions and sigma via the stacked batched "
                        "torch.autograd.Function (list-batched and per-image autograd ops for comparison)"}


def pp_pairs(im, sig, k):
    """Pairs (pixel, point) with d <= k sigma_i: the per-point truncated
    method's work, counted with a k-d tree over the pixel centres."""
    from scipy.spatial import cKDTree
    yy, xx = np.meshgrid(np.arange(im.H) + 0.5, np.arange(im.W) + 0.5, indexing="ij")
    tree = cKDTree(np.stack([xx.ravel(), yy.ravel()], 1))
    cnt = tree.query_ball_point(im.points.astype(np.float64), k * sig.astype(np.float64), return_length=True,
                                workers=-1)
    return int(np.sum(cnt))


def pp_oracle_rate(im, sig, k, target_s=4.0):
    """The FP64 per-point oracle on a bounded random pixel sample (Mpix/s)."""
    import oracle
    rng = np.random.default_rng(321)
    n = 64
    while True:
        pix = rng.integers(0, im.H * im.W, n)
        t0 = time.perf_counter()
        oracle.forward_pp(im.points, im.values, sig, im.H, im.W, mode=oracle.TRUNCATED, k=k, pixels=pix)
        t = time.perf_counter() - t0
        if t >= target_s or n >= 1 << 20:
            break
        n = int(n * min(8.0, max(1.2, 1.2 * target_s / max(t, 1e-3))))
    return {"value": n / t / 1e6, "unit": "Mpix/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d random pixels, %.1f s" % (n, t)}

def bench_per_point_sigma(dev, steps, warmup, flush, stream, lo=0.5, hi=1.5, k=3.0):
    """The 1024^2 upsampling workload with a sigma per point (log-uniform in
    [lo, hi] px, bound hi, truncated at k sigma_i): the graph-replayed forward
    and forward + backward (positions, values, every sigma_i) through the
    autograd op, beside the same calls with one shared sigma = hi (the same
    search window)."""
    import torch
    import paper_2012_13257_b300 as gmi
    import workloads as wl
    im = wl.upsample_1024()
    P = torch.as_tensor(im.points, device=dev)
    V = torch.as_tensor(im.values, device=dev)
    S = torch.as_tensor(wl.point_sigmas(22, im.N, lo, hi), device=dev)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)
    G = torch.randn((im.H, im.W, im.C), generator=torch.Generator(device=dev).manual_seed(9), device=dev)

    def fwd_pp():
        gmi.interpolate_pp(P, V, S, hi, im.H, im.W, radius_sigmas=k, mode="truncated", graph=True, out=out)

    def fwd_pp_exact():
        gmi.interpolate_pp(P, V, S, hi, im.H, im.W, mode="exact", graph=True, out=out)

    def fwd_shared():
        gmi.interpolate(P, V, hi, im.H, im.W, mode="truncated", radius_sigmas=k, graph=True, out=out)

    Sxy = torch.as_tensor(wl.point_sigmas(23, im.N, lo, hi, axes=2), device=dev)

    def fwd_aniso():
        gmi.interpolate_pp(P, V, Sxy, hi, im.H, im.W, radius_sigmas=k, mode="truncated", graph=True, out=out)

    Scov = torch.as_tensor(wl.point_cov(24, im.N, lo, hi, rmax=0.9), device=dev)

    cov_bound = wl.cov_bound(Scov.cpu().numpy())

    def fwd_cov():
        gmi.interpolate_pp(P, V, Scov, cov_bound, im.H, im.W, radius_sigmas=k, mode="truncated", graph=True,
                           out=out)

    def fwd_cov_exact():
        gmi.interpolate_pp(P, V, Scov, cov_bound, im.H, im.W, mode="exact", graph=True, out=out)

    Pg, Vg, Sg = (t.clone().requires_grad_(True) for t in (P, V, S))
    sg = torch.tensor(hi, dtype=torch.float32, device=dev, requires_grad=True)

    def fb_pp():
        gmi.gmi_interpolate_pp(Pg, Vg, Sg, hi, im.H, im.W, radius_sigmas=k, mode="truncated").backward(G)

    def fb_pp_exact():
        gmi.gmi_interpolate_pp(Pg, Vg, Sg, hi, im.H, im.W, mode="exact").backward(G)

    def fb_shared():
        gmi.gmi_interpolate(Pg, Vg, sg, im.H, im.W, mode="truncated", radius_sigmas=k).backward(G)

    res = {}
    for name, fn in (("forward_pp", fwd_pp), ("forward_shared", fwd_shared), ("forward_aniso", fwd_aniso),
                     ("forward_cov", fwd_cov), ("forward_pp_exact", fwd_pp_exact),
                     ("forward_cov_exact", fwd_cov_exact),
                     ("fwd_bwd_pp", fb_pp), ("fwd_bwd_pp_exact", fb_pp_exact),
                     ("fwd_bwd_shared", fb_shared)):
        for _ in range(max(3, warmup)):
            fn()
        torch.cuda.synchronize()
        t = timed_steps(fn, steps, flush, stream, queued=name.startswith("forward"))
        ms = sum(t) / len(t)
        res[name] = {"ms_per_step": ms, "value": im.H * im.W / (ms * 1e-3) / 1e6}
    res["unit"] = "Mpix/s"
    # near-kernel time of the per-point forward (stage events, queued behind a
    # device spin), against the algorithmic pairs d <= k sigma_i
    from paper_2012_13257_b300 import _lib
    L = _lib.load()
    L.gmi_profile_enable(1)
    L.gmi_profile_read(None, None, 1)
    torch.cuda._sleep(int(steps * 200e-6 * SM_MAX_MHZ * 1e6))
    for _ in range(steps):
        flush.zero_()
        gmi.interpolate_pp(P, V, S, hi, im.H, im.W, radius_sigmas=k, mode="truncated", out=out)
    torch.cuda.synchronize()
    st_ms = (ctypes.c_double * 4)()
    st_n = (ctypes.c_int * 4)()
    L.gmi_profile_read(st_ms, st_n, 1)
    L.gmi_profile_enable(0)
    near_ms = st_ms[1] / max(1, st_n[1])
    sig = S.cpu().numpy()
    pairs = pp_pairs(im, sig, k)
    clk = SM_MAX_MHZ
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * FP32_PER_SM_CLK / FP32_OPS_PER_PAIR * clk * 1e6 / 1e9
    achieved = pairs / (near_ms * 1e-3) / 1e9 if near_ms > 0 else None
    res["roofline"] = {"bound": "alu", "kernel": "near_kernel<4,4,3,truncated,per-point>", "launch_ms": near_ms,
                       "pairs_per_launch": pairs, "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                       "frac": achieved / peak if achieved else None,
                       "peak_basis": "FP32 pipe at the maximum SM clock %d MHz (%d SMs x %d / %d ops per pair)"
                                     % (clk, sms, FP32_PER_SM_CLK, FP32_OPS_PER_PAIR)}
    res["oracle"] = pp_oracle_rate(im, sig, k)
    res["workload"] = ("1024x1024x3 f32 from 262,144 jittered-grid points, sigma_i log-uniform in [%g, %g] px "
                       "(bound %g), truncated at %g sigma_i; forward_aniso draws sx_i, sy_i independently from "
                       "the same range, forward_cov adds rho_i uniform in [-0.9, 0.9] (bound: the largest sqrt of a "
                       "covariance eigenvalue); shared-sigma rows use sigma = %g with the same window; fwd_bwd through "
                       "the autograd ops (positions, values, sigmas), upstream N(0,1); *_exact rows: exact mode "
                       "(every point, k = 6)" % (lo, hi, hi, k, hi))
    return res

def bench_reconstruction(dev, side=768, factors=(2, 3, 4, 6, 8), sigma_scales=(0.2, 0.25, 0.35, 0.5, 0.7)):
    """Reconstruction quality (the paper's downsample-then-upsample study,
    section 3.2, on a smooth random field instead of ImageNet images): a field
    with up to 24 cycles across a side x side image is point-sampled at the
    centres of f x f blocks and brought back to full size by this method (best
    sigma of a small sweep, sigma = scale * f) and by torch's nearest, bilinear
    and bicubic resampling; mean L1 error against the full-resolution field."""
    import torch
    import torch.nn.functional as F
    import paper_2012_13257_b300 as gmi
    import workloads as wl
    rows = {}
    for f in factors:
        pts, vals, low, truth = wl.reconstruction_case(f, side)
        T = torch.as_tensor(truth, device=dev)
        P, V = torch.as_tensor(pts, device=dev), torch.as_tensor(vals, device=dev)
        errs = {}
        for sc in sigma_scales:
            out = gmi.interpolate(P, V, sc * f, side, side)
            errs[sc * f] = float((out - T).abs().mean())
        best = min(errs, key=errs.get)
        row = {"gmi": errs[best], "gmi_sigma": best, "gmi_by_sigma": errs}
        lowt = torch.as_tensor(low, device=dev).permute(2, 0, 1)[None]
        for mode in ("nearest", "bilinear", "bicubic"):
            kw = {} if mode == "nearest" else {"align_corners": False}
            up = F.interpolate(lowt, size=(side, side), mode=mode, **kw)[0].permute(1, 2, 0).clamp(0.0, 1.0)
            row[mode] = float((up - T).abs().mean())
        rows["x%d" % f] = row
    return {"metric": "mean L1 error vs the full-resolution field (lower is better)", "side": side,
            "factors": rows, "workload": "smooth random field (32 sinusoids, up to 24 cycles per image, 3 "
            "channels) point-sampled at block centres; torch resampling with align_corners=False"}


def bench_point_optimization(dev, side=256, n=4096, sigma=2.0, iters=200, lr=0.05):
    """Optimising the point positions by gradient descent (section 3.3) on a
    synthetic image: n uniformly random points carry the field's colours at
    their starting positions; Adam moves them to minimise the L1 error of the
    interpolated image, forward and backward through the autograd op."""
    import torch
    import paper_2012_13257_b300 as gmi
    import workloads as wl
    rng = np.random.default_rng(8)
    params = wl.field_params(rng, 3, max_cycles=8.0)
    yy, xx = np.meshgrid(np.arange(side) + 0.5, np.arange(side) + 0.5, indexing="ij")
    target = torch.as_tensor(wl.eval_field(params, np.stack([xx.ravel(), yy.ravel()], 1), float(side))
                             .reshape(side, side, 3), device=dev)
    p0 = wl.uniform_points(rng, n, side, side)
    mu = torch.as_tensor(p0, device=dev).clone().requires_grad_(True)
    vals = torch.as_tensor(wl.eval_field(params, p0, float(side)), device=dev)
    opt = torch.optim.Adam([mu], lr=lr)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(iters):
        opt.zero_grad(set_to_none=True)
        loss = (gmi.gmi_interpolate(mu, vals, sigma, side, side) - target).abs().mean()
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    moved = float((mu.detach() - torch.as_tensor(p0, device=dev)).norm(dim=1).mean())
    return {"loss_start": float(losses[0]), "loss_end": float(losses[-1]), "iters": iters,
            "iters_per_s": iters / t, "mean_displacement_px": moved, "sigma": sigma, "points": n,
            "workload": "%dx%dx3 smooth field, %d uniform points, colours fixed at their start, "
                        "Adam lr %g on positions, L1 loss" % (side, side, n, lr)}


def bench_serving(dev, n_requests=10000, rate=2000.0, n_templates=128):
    """Open-loop serving: Poisson arrivals at `rate`, sides log-uniform in
    [64, 2048], N = U[0.1, 1] H W, uniform or clustered, sigma U[0.5, 2];
    payloads cycle through `n_templates` pre-generated pinned requests.
    Latency = completion - scheduled arrival.  Compared with plain
    per-request launches (copy in, forward, copy out, one at a time)."""
    import threading
    import torch
    import paper_2012_13257_b300 as gmi
    import workloads as wl
    stream_spec = wl.serving_stream(n_requests=n_requests, rate=rate)
    tmpl = [r.materialise() for r in stream_spec[:n_templates]]
    hP = [torch.as_tensor(t.points).pin_memory() for t in tmpl]
    hV = [torch.as_tensor(t.values).pin_memory() for t in tmpl]
    hO = [torch.empty((t.H, t.W, 3), dtype=torch.float32).pin_memory() for t in tmpl]

    dP = dV = dO = None

    def run_server(device=False):
        srv = gmi.Server(budget_bytes=40 << 30, max_batch_images=64, max_batch_pixels=1 << 25, n_streams=2)
        if device:
            submit = lambda j, t: srv.submit_device(dP[j], dV[j], t.sigma, t.H, t.W, dO[j])
        else:
            submit = lambda j, t: srv.submit(hP[j], hV[j], t.sigma, t.H, t.W, hO[j])
        # warm-up (graph capture for both slots)
        for j in range(4):
            srv.wait(submit(j, tmpl[j]))
        sched, ids, sub = [], [], []
        lat = [0.0] * n_requests
        t0 = time.perf_counter()
        done_ev = threading.Event()

        def waiter():
            for r in range(n_requests):
                while len(ids) <= r:
                    time.sleep(0.0002)
                lat[r] = (sub[r] - sched[r]) + srv.wait(ids[r])
            done_ev.set()
        th = threading.Thread(target=waiter)
        th.start()
        for r, spec in enumerate(stream_spec):
            t_sched = t0 + spec.t_arrival
            while True:
                now = time.perf_counter()
                if now >= t_sched:
                    break
                time.sleep(min(0.0005, t_sched - now))
            j = r % n_templates
            t = tmpl[j]
            sched.append(t_sched)
            sub.append(time.perf_counter())
            ids.append(submit(j, t))
        done_ev.wait()
        th.join()
        wall = time.perf_counter() - t0
        st = srv.counters()
        srv.close()
        return lat, wall, st

    def run_plain():
        s = torch.cuda.Stream(dev)
        dP = [torch.empty_like(p, device=dev) for p in hP]
        dV = [torch.empty_like(v, device=dev) for v in hV]
        dO = [torch.empty_like(o, device=dev) for o in hO]
        lat = []
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            for r, spec in enumerate(stream_spec):
                t_sched = t0 + spec.t_arrival
                now = time.perf_counter()
                if now < t_sched:
                    time.sleep(t_sched - now)
                j = r % n_templates
                t = tmpl[j]
                dP[j].copy_(hP[j], non_blocking=True)
                dV[j].copy_(hV[j], non_blocking=True)
                gmi.interpolate(dP[j], dV[j], t.sigma, t.H, t.W, out=dO[j])
                hO[j].copy_(dO[j], non_blocking=True)
                s.synchronize()
                lat.append(time.perf_counter() - t_sched)
        return lat, time.perf_counter() - t0

    def run_saturated(n):
        """All n requests offered at once: the server against plain
        per-request launches (copy in, forward, copy out, synchronise)."""
        srv = gmi.Server(budget_bytes=40 << 30, max_batch_images=64, max_batch_pixels=1 << 25, n_streams=2)
        for j in range(4):
            srv.wait(srv.submit(hP[j], hV[j], tmpl[j].sigma, tmpl[j].H, tmpl[j].W, hO[j]))
        t0 = time.perf_counter()
        rids = [srv.submit(hP[r % n_templates], hV[r % n_templates], tmpl[r % n_templates].sigma,
                           tmpl[r % n_templates].H, tmpl[r % n_templates].W, hO[r % n_templates]) for r in range(n)]
        for rid in rids:
            srv.wait(rid)
        t_srv = time.perf_counter() - t0
        launches = srv.stats()["launches"]
        srv.close()
        s = torch.cuda.Stream(dev)
        dP = [torch.empty_like(p, device=dev) for p in hP]
        dV = [torch.empty_like(v, device=dev) for v in hV]
        dO = [torch.empty_like(o, device=dev) for o in hO]
        with torch.cuda.stream(s):
            t0 = time.perf_counter()
            for r in range(n):
                j = r % n_templates
                t = tmpl[j]
                dP[j].copy_(hP[j], non_blocking=True)
                dV[j].copy_(hV[j], non_blocking=True)
                gmi.interpolate(dP[j], dV[j], t.sigma, t.H, t.W, out=dO[j])
                hO[j].copy_(dO[j], non_blocking=True)
                s.synchronize()
            t_plain = time.perf_counter() - t0
        pxn = sum(tmpl[r % n_templates].H * tmpl[r % n_templates].W for r in range(n))
        return {"requests": n, "value": pxn / t_srv / 1e6, "plain_value": pxn / t_plain / 1e6,
                "speedup_vs_plain": t_plain / t_srv, "launches": launches - 4, "unit": "Mpix/s"}

    px = sum(tmpl[r % n_templates].H * tmpl[r % n_templates].W for r in range(n_requests))
    lat_s, wall_s, st = run_server()
    lat_p, wall_p = run_plain()
    sat = run_saturated(2000)
    # the same stream with the payloads already on the device (no copies)
    dP = [p.to(dev) for p in hP]
    dV = [v.to(dev) for v in hV]
    dO = [torch.empty((t.H, t.W, 3), dtype=torch.float32, device=dev) for t in tmpl]
    lat_d, wall_d, st_d = run_server(device=True)
    q = lambda v, p: float(np.percentile(np.asarray(v) * 1e3, p))
    return {"p50_ms": q(lat_s, 50), "p99_ms": q(lat_s, 99), "value": px / wall_s / 1e6, "unit": "Mpix/s",
            "wall_s": wall_s, "launches": st["launches"], "max_in_flight": st["max_in_flight"],
            "requests": n_requests,
            "device_resident": {"p50_ms": q(lat_d, 50), "p99_ms": q(lat_d, 99), "value": px / wall_d / 1e6,
                                "launches": st_d["launches"], "max_in_flight": st_d["max_in_flight"]},
            "plain_p50_ms": q(lat_p, 50), "plain_p99_ms": q(lat_p, 99), "plain_value": px / wall_p / 1e6,
            "plain_wall_s": wall_p, "offered_req_s": rate, "saturated": sat,
            "workload": "%d requests, Poisson %.0f req/s, sides log-uniform [64,2048], N=U[0.1,1]HW, "
                        "uniform/clustered, sigma U[0.5,2]; payloads cycle %d pinned templates; 40 GB budget, "
                        "2 batch slots; latency from scheduled arrival; 'device_resident': the same stream with the "
                        "payloads already on the device (gmi_server_submit_device, no copies); 'saturated': the "
                        "first 2000 requests offered at once, wall-clock throughput" % (n_requests, rate, n_templates)}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, per step a bounded
    pixel sample of the headline workload."""
    if rank != 0:
        return
    import oracle
    import workloads as wl
    im = wl.upsample_1024()
    rng = np.random.default_rng(7)
    per_step = 1024
    for _ in range(args.warmup):
        oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=rng.integers(0, im.H * im.W, 64))
    t = 0.0
    for _ in range(args.steps):
        pix = rng.integers(0, im.H * im.W, per_step)
        t0 = time.perf_counter()
        oracle.forward(im.points, im.values, im.H, im.W, im.sigma, pixels=pix)
        t += time.perf_counter() - t0
    v = per_step * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_pixels_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d random pixels per step of the %dx%d image" % (per_step, im.H, im.W)},
            "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_2012_13257_b300 as gmi
    from paper_2012_13257_b300 import _lib
    import workloads as wl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    D = Dist(world, dev)
    L = _lib.load()

    im = wl.upsample_1024()
    P = torch.as_tensor(im.points, device=dev)
    V = torch.as_tensor(im.values, device=dev)
    out = torch.empty((im.H, im.W, im.C), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if args.only:
        stream = torch.cuda.current_stream(dev)
        fn = {"batched": lambda: bench_batched(dev, args.steps, args.warmup, flush, stream,
                                               autotune=not args.no_autotune),
              "fwd_bwd": lambda: bench_fwd_bwd(dev, args.steps, args.warmup, flush, stream),
              "serving": lambda: bench_serving(dev),
              "reconstruction": lambda: bench_reconstruction(dev),
              "point_optimization": lambda: bench_point_optimization(dev),
              "per_point_sigma": lambda: bench_per_point_sigma(dev, args.steps, args.warmup, flush, stream)}[args.only]
        if rank == 0:
            print(json.dumps({args.only: fn()}), flush=True)
        D.close()
        return
    stream = torch.cuda.current_stream(dev)

    def step():
        # the public call with graph replay: one host launch per forward
        gmi.interpolate(P, V, im.sigma, im.H, im.W, out=out, graph=True)

    def step_plain():
        gmi.interpolate(P, V, im.sigma, im.H, im.W, out=out)

    for _ in range(max(3, args.warmup)):
        step()
        step_plain()
    torch.cuda.synchronize()

    # ---- headline: device-resident inputs, per-step events, L2 flushed between
    # steps; the steps are enqueued behind a device spin, so that no step waits
    # for the host inside its events (the spin precedes the first start event)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    D.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    spin = prequeue(args.steps + 1)
    flush.zero_()
    step()   # one more warm-up step in the queue, so no timed step starts the queued run
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    queue_ok = queued_in_time(spin)
    torch.cuda.synchronize()
    if not queue_ok:
        # the host fell behind the spin: once more, with a spin four times as long
        spin = prequeue(args.steps + 1, 1.6e-3)
        flush.zero_()
        step()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
        queue_ok = queued_in_time(spin)
        torch.cuda.synchronize()
    clk = clocks.stop()
    D.barrier()
    ms_steps = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_total = D.max(sum(ms_steps))

    # ---- the same steps as plain launches (seven host calls per forward)
    tp = timed_steps(step_plain, args.steps, flush, stream)
    plain = {"value": replica_throughput(im.H * im.W, args.steps, world, D.max(sum(tp))), "unit": "Mpix/s",
             "ms_per_step": D.max(sum(tp)) / args.steps,
             "note": "gmi.interpolate without graph replay; host-launch bound when the host is slow"}

    # ---- per-stage times (events around each stage on the launching stream),
    # in a separate pass: the steps are queued behind a short device spin so
    # that no stage waits for the host inside its events
    L.gmi_profile_enable(1)
    L.gmi_profile_read(None, None, 1)
    torch.cuda._sleep(int(args.steps * 400e-6 * SM_MAX_MHZ * 1e6))
    for k in range(args.steps):
        flush.zero_()
        step_plain()
    torch.cuda.synchronize()
    stage_ms = (ctypes.c_double * 4)()
    stage_n = (ctypes.c_int * 4)()
    L.gmi_profile_read(stage_ms, stage_n, 1)
    L.gmi_profile_enable(0)
    ms_per_step = t_total / args.steps
    value = replica_throughput(im.H * im.W, args.steps, world, t_total)

    # ---- e2e: pinned host buffers through the host-buffer C-ABI call
    # (gmi_forward_host: uploads, kernels and download, one graph per step),
    # copies inside the timed region
    hP = torch.as_tensor(im.points).pin_memory()
    hV = torch.as_tensor(im.values).pin_memory()
    hO = torch.empty((im.H, im.W, im.C), dtype=torch.float32).pin_memory()
    def host_step():
        gmi.interpolate_host(hP, hV, im.sigma, im.H, im.W, out=hO, graph=True)
    for _ in range(3):
        host_step()
    torch.cuda.synchronize()
    D.barrier()
    # queued behind a device spin like the headline steps, so that the host's
    # work for a call (argument checks, the graph lookup and launch) overlaps
    # the device's previous steps instead of idling the device inside the
    # step's events; every step still uploads its inputs and downloads its image
    eq = {}
    e_ms = timed_steps(host_step, args.steps, flush, stream, queued=True, info=eq)
    e_total = D.max(sum(e_ms))
    # the same calls issued one by one as the host gets to them (the host's
    # per-call time then lands inside the steps)
    D.barrier()
    hp_total = D.max(sum(timed_steps(host_step, args.steps, flush, stream)))
    e2e = {"value": replica_throughput(im.H * im.W, args.steps, world, e_total), "unit": "Mpix/s",
           "h2d_bytes_per_step": int(hP.numel() * 4 + hV.numel() * 4),
           "d2h_bytes_per_step": int(hO.numel() * 4),
           "ms_per_step": e_total / args.steps, "queue_ok": eq.get("queue_ok"),
           "host_paced": {"value": replica_throughput(im.H * im.W, args.steps, world, hp_total),
                          "ms_per_step": hp_total / args.steps}}
    e2e_pipe = e2e_pipelined(gmi, im, hP, hV, args.steps, D, world)
    e2e["breakdown"] = e2e_breakdown(gmi, im, hP, hV, hO, args.steps, flush, stream)

    # ---- roofline of the dominant kernel (near-field gather), timed live above
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    near_ms = stage_ms[1] / max(1, stage_n[1])
    pairs = algorithmic_pairs(im) if rank == 0 else 0
    rates = gmi.measure_unit_rates() if rank == 0 else None
    clk_mhz = clk.get("sm_mhz") or SM_MAX_MHZ
    # per-pair peaks of the two units the pair work uses; the FP32 pipe binds
    fp32_gpair = sms * FP32_PER_SM_CLK / FP32_OPS_PER_PAIR * clk_mhz * 1e6 / 1e9
    sfu_gpair = sms * SFU_PER_SM_CLK * clk_mhz * 1e6 / 1e9
    peak_gpair = min(fp32_gpair, sfu_gpair)
    achieved = pairs / (near_ms * 1e-3) / 1e9 if near_ms > 0 else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_gpair, "unit": "Gpair/s",
            "frac": (achieved / peak_gpair) if achieved else None,
            "traffic": near_kernel_traffic(),
            "kernel": "near_staged_kernel<4,4,3,exact>", "launch_ms": near_ms, "pairs_per_launch": pairs,
            "peak_basis": "FP32 pipe: %d SMs x %d FMA/clk / %d FP32 ops per algorithmic pair x %.0f MHz "
                          "(SM clock sampled during the timed steps); the SFU allows %.0f Gpair/s "
                          "(%d ex2/clk, one per pair); per-clock rates from the unit counts, checked by "
                          "unit_rates_measured (results per SM per clock)" %
                          (sms, FP32_PER_SM_CLK, FP32_OPS_PER_PAIR, clk_mhz, sfu_gpair, SFU_PER_SM_CLK),
            "unit_rates_measured": rates,
            "frac_fma_strict": (pairs * (im.C + 1) / (near_ms * 1e-3) /
                                (sms * FP32_PER_SM_CLK * clk_mhz * 1e6)) if near_ms > 0 else None}
    stages = {name: (stage_ms[i] / stage_n[i] if stage_n[i] else None) for i, name in enumerate(_lib.STAGES)}

    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": im.N, "H": im.H, "W": im.W, "C": im.C,
                       "sigma": im.sigma, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between steps (256 MB write), not timed"},
            "roofline": roof, "e2e": e2e, "gpu_launches": LAUNCHES_PER_FORWARD * args.steps, "clocks": clk,
            "stage_ms": stages, "plain_launch": plain, "e2e_pipelined": e2e_pipe,
            "step_ms": step_stats(ms_steps), "queue_ok": queue_ok}
    if rank == 0 and not args.no_extras:
        extras = {}
        for name, fn in (("batched", lambda: bench_batched(dev, args.steps, args.warmup, flush, stream)),
                         ("fwd_bwd", lambda: bench_fwd_bwd(dev, args.steps, args.warmup, flush, stream)),
                         ("serving", lambda: bench_serving(dev)),
                         ("reconstruction", lambda: bench_reconstruction(dev)),
                         ("point_optimization", lambda: bench_point_optimization(dev)),
                         ("per_point_sigma", lambda: bench_per_point_sigma(dev, args.steps, args.warmup, flush,
                                                                           stream))):
            try:
                extras[name] = fn()
            except Exception as e:   # a failed extra must not hide the headline
                extras[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        # the long objects first (with the full details of the metric's own
        # workloads); the metric's batched, served and fwd+bwd figures close
        # the line in a compact form
        for name in ("per_point_sigma", "reconstruction", "point_optimization"):
            line[name] = extras[name]
        line["details"] = {k: extras[k] for k in ("batched", "serving", "fwd_bwd")}
    D.barrier()
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(im)
    if rank == 0 and not args.no_extras:
        line["batched"] = summary(extras["batched"], ["value", "plain_per_image_value", "speedup_vs_plain",
                                                      "ms_per_step", "queue_ok"],
                                  roofline=["frac", "frac_step", "achieved", "launch_ms", "pairs_per_launch"])
        line["serving"] = summary(extras["serving"], ["p50_ms", "p99_ms", "plain_p50_ms", "plain_p99_ms", "value",
                                                      "plain_value", "launches", "max_in_flight"],
                                  saturated=["value", "plain_value", "speedup_vs_plain"],
                                  device_resident=["p50_ms", "p99_ms", "value"])
        line["fwd_bwd"] = summary(extras["fwd_bwd"], ["value", "ms_per_step", "list_batched_autograd_value",
                                                      "per_image_autograd_value", "backward_ms"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    D.close()


if __name__ == "__main__":
    main()
