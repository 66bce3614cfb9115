#!/usr/bin/env python
"""Training throughput of the GSta hot path on one GB300.

Workload (synthetic stand-in for the paper's Mip-NeRF 360 scenes): 1,000,000
Gaussians sampled on a sphere + ground plane + 20 boxes, SH degree 3, 200
cameras on a hemisphere at 1237x822, targets rendered from a 1.5M-Gaussian
ground-truth set. A step is one training iteration of Algorithm 1: the
freeze-map action and subset-PSNR check at their cadence, projection, sort,
compositing, loss, backward with frozen Gaussians skipped, masked Adam.

The model is first trained (untimed) through the GSta schedule up to
iteration 4750 -- past warmup, a reset and an update -- so the timed
iterations run on the freeze map the method itself produced; warm-up and
timed iterations continue the same schedule.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 runs N independent replicas (one per GPU, launched with torchrun);
the path has no exchange step, so no collective is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="surface-1M-1237x822", n_init=1_000_000, n_gt=1_500_000, views=200, width=1237, height=822,
                tile=16, sh_degree=3)
METRIC = "train it/s (GSta freezing, 1M Gaussians, 1237x822)"
PEAKS_FALLBACK = dict(hbm_gbs=6800.0, sm_max_mhz=2070.0)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- CPU (oracle) leg


def oracle_sample_step(scene, frac: float, rng_seed: int = 0) -> dict:
    """One oracle training step on a bounded sample of the workload.

    The sample is a centred crop of one training view covering `frac` of its
    pixels, with the Gaussians visible in it: the oracle runs its full step
    there (projection, sort, compositing, loss, backward, Adam on those
    Gaussians). Culling and Adam of the Gaussians outside the crop are timed
    on a random `frac` share of them. The step time of the whole view is the
    sample's time divided by `frac`."""
    import numpy as np

    import oracle
    from paper_2504_06716_gb300 import synth

    cam = scene.cameras[scene.train_views[0]]
    W, H = cam.width, cam.height
    s = float(np.sqrt(frac))
    cw, ch = max(16, int(round(W * s))), max(16, int(round(H * s)))
    x0, y0 = (W - cw) // 2, (H - ch) // 2
    crop = synth.Camera(cw, ch, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, cam.R, cam.t, cam.campos)
    ocam = oracle.make_cam(crop)
    true_frac = cw * ch / float(W * H)
    P = scene.init
    rng = np.random.default_rng(rng_seed)
    cache = scene.__dict__.setdefault("_crop_vis", {})
    if (cw, ch) not in cache:  # which Gaussians the crop sees (setup, untimed)
        cache[(cw, ch)] = np.nonzero(oracle.project(P, ocam)["radius"] > 0)[0]
    vis = cache[(cw, ch)]
    sub = np.ascontiguousarray(P[vis])
    others = np.setdiff1d(np.arange(P.shape[0]), vis)
    pick = rng.choice(others, size=max(1, int(len(others) * true_frac)), replace=False)
    gt = rng.uniform(0, 1, (3, ch, cw))
    M = np.zeros_like(sub)
    V = np.zeros_like(sub)
    t0 = time.perf_counter()
    res = oracle.loss_and_grad(sub, ocam, gt)
    oracle.adam(sub, res["G"], M, V, None, np.full(6, 1e-3), step=1)
    oracle.project(np.ascontiguousarray(P[pick]), ocam)
    Po = np.ascontiguousarray(P[pick])
    oracle.adam(Po, np.zeros_like(Po), np.zeros_like(Po), np.zeros_like(Po), None, np.full(6, 1e-3), step=1)
    dt = time.perf_counter() - t0
    return dict(seconds=dt, frac=true_frac, crop=(cw, ch), gaussians=int(len(vis)), step_s=dt / true_frac)


def cpu_baseline(scene, single_frac: float = 0.3) -> dict:
    """The oracle on the host's cores: one whole step of the workload on every
    core the oracle uses (its loops over Gaussians, pixels and tiles are
    parallel), and beside it one core on a centred crop of single_frac of the
    view, its time divided by that share."""
    import oracle

    cores = oracle.max_threads()
    try:
        oracle.set_threads(cores)
        full = oracle_sample_step(scene, 1.0)
        oracle.set_threads(1)
        one = oracle_sample_step(scene, single_frac, 1)
    finally:
        oracle.set_threads(cores)
    return dict(value=1.0 / full["step_s"], unit="it/s", cores=cores, kind="oracle",
                sample=(f"one whole oracle step of the workload (a training view, {full['gaussians']} visible "
                        f"Gaussians, Adam on them and culling of the rest) on {cores} threads, {full['seconds']:.1f} s"),
                single_thread=dict(value=1.0 / one["step_s"], unit="it/s", cores=1,
                                   sample=(f"one oracle step on a centred {one['crop'][0]}x{one['crop'][1]} crop "
                                           f"({one['frac']:.3f} of the view, {one['gaussians']} visible Gaussians) "
                                           f"plus culling and Adam of the same share of the others, "
                                           f"{one['seconds']:.1f} s on 1 thread, divided by the share (extrapolated)")))


def reference_arm(args):
    """The oracle as the reference implementation, on every host core it uses:
    W untimed and K timed steps. A step is one whole oracle step of the
    workload when K + W of them fit the time budget; otherwise a centred crop
    of the view sized to fit (the line states the fraction, and the rate is
    the crop's time divided by its share)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2504_06716_gb300 import synth

    scene = synth.surface_scene(WORKLOAD["n_init"], 10, WORKLOAD["views"], WORKLOAD["width"], WORKLOAD["height"])
    cores = oracle.max_threads()
    budget = 150.0
    first = oracle_sample_step(scene, 1.0, 0)  # the first warm-up step, whole
    frac = min(1.0, max(0.01, budget / max(1, args.steps + args.warmup - 1) / max(first["seconds"], 1e-3)))
    for i in range(1, args.warmup):
        oracle_sample_step(scene, frac, i)
    t0 = time.perf_counter()
    samples = [oracle_sample_step(scene, frac, 1000 + i) for i in range(args.steps)]
    wall = time.perf_counter() - t0
    true_frac = samples[0]["frac"]
    ms = 1000.0 * wall / args.steps
    its = true_frac / (wall / args.steps)
    sample = (f"each step: one whole oracle step of the workload on {cores} threads" if true_frac >= 1.0 else
              f"each step: the oracle on a centred crop of {true_frac:.4f} of a view on {cores} threads; the rate "
              f"divides the crop's time by that share")
    line = dict(impl="reference", metric=METRIC, value=its, unit="it/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", sample_fraction=true_frac,
                config=dict(workload=WORKLOAD["workload"], gaussians=WORKLOAD["n_init"],
                            resolution=f"{WORKLOAD['width']}x{WORKLOAD['height']}", sh_degree=3),
                cpu_baseline=dict(value=its, unit="it/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=its, unit="it/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- replicas


class Replicas:
    """N independent replicas of the step, one process per GPU (torchrun sets
    WORLD_SIZE / RANK / LOCAL_RANK). The training step has no exchange step,
    so nothing on the data path is collective: only the timing is combined --
    a barrier on both sides of the timed region, the slowest rank's time, and
    the units every rank processed. ``backend`` is "nccl" for the GPU arm and
    "gloo" on the CPU; with WORLD_SIZE 1 no process group is made."""

    def __init__(self, backend: str = "nccl", device=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.backend = backend
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist

            kw = {} if device is None else dict(device_id=device)
            dist.init_process_group(backend, **kw)
            self.dist = dist

    @property
    def printer(self) -> bool:
        """Rank 0 alone prints the result line."""
        return self.rank == 0

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def slowest_ms(self, ms: float) -> float:
        """The largest of the ranks' timed-region durations."""
        if self.dist is None:
            return ms
        import torch

        t = torch.tensor([ms], dtype=torch.float64, device="cuda" if self.backend == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def rate(self, units_per_rank: int, ms: float) -> float:
        """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
        return units_per_rank * self.world / (ms / 1000.0)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


# --------------------------------------------------------------------------- GPU arm


def gpu_arm(args):
    import torch

    from paper_2504_06716_gb300 import lib, pipeline, synth
    from paper_2504_06716_gb300.schedule import GStaConfig
    from paper_2504_06716_gb300.train import Trainer

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    reps = Replicas("nccl", torch.device("cuda", local))
    world, rank = reps.world, reps.rank
    lib.load()

    W_, H_ = WORKLOAD["width"], WORKLOAD["height"]
    scene = synth.surface_scene(WORKLOAD["n_init"], WORKLOAD["n_gt"], WORKLOAD["views"], W_, H_)
    if args.views < WORKLOAD["views"]:  # smaller profiling case: fewer targets on the device
        keep = set(scene.train_views[:args.views])
        scene.train_views = sorted(keep)
        scene.test_views = scene.test_views[:2]
        scene.subset_views = scene.train_views[:2]
    tr = Trainer(scene, GStaConfig(), tile=WORKLOAD["tile"])
    m = tr.model
    # untimed pre-training through the schedule (warmup, calibration, reset, first updates)
    while tr.k < args.start_iter:
        tr.iteration(allow_early_stop=False)
    tuning = None
    if not args.no_autotune:  # rasteriser tile size and launch shapes for this state (autotune.py)
        tr.autotune()
        tuning = dict(tile=tr.tuning.tile, fwd_ppt_batch=list(tr.tuning.fwd), bwd_ppt_batch=list(tr.tuning.bwd),
                      per_tile_ms={str(t): dict(project_sort=round(r["project_sort_ms"], 4),
                                                fwd=[*r["best_fwd"], round(min(r["fwd_ms"].values()), 4)],
                                                bwd=[*r["best_bwd"], round(min(r["bwd_ms"].values()), 4)],
                                                total=round(r["total_ms"], 4))
                                   for t, r in tr.tuning.table.items()})
    for _ in range(args.warmup):
        tr.iteration(allow_early_stop=False)
    torch.cuda.synchronize()
    if lib.gs_get_device_error():
        raise RuntimeError("device error flags set during pre-training")

    stream = torch.cuda.current_stream()
    # dominant kernel (rasteriser backward) timed live inside the timed region:
    # gs_train_step records a pair of events around it on the step's stream
    raster_ev = []
    orig_train_step = m.train_step

    def train_step_timed(view, gt, lrs, stream=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()  # creates the events; gs_train_step records them again in place
        e1.record()
        st = m._step_struct(view)
        st.bwd_events[0], st.bwd_events[1] = e0.cuda_event, e1.cuda_event
        orig_train_step(view, gt, lrs, stream)
        st.bwd_events[0] = st.bwd_events[1] = None
        raster_ev.append((e0, e1, tr.order[tr.k]))

    m.train_step = train_step_timed
    active_before = int(m.n_active.item())
    n_before = m.n
    k_start = tr.k
    reps.barrier()
    torch.cuda.synchronize()
    launches0 = lib.gs_launch_count()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        t0.record(stream)
        for _ in range(args.steps):
            tr.iteration(allow_early_stop=False)
        t1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = lib.gs_launch_count() - launches0
    ms = reps.slowest_ms(t0.elapsed_time(t1))
    reps.barrier()
    m.train_step = orig_train_step
    active_after = int(m.n_active.item())
    flags = lib.gs_get_device_error()
    its = reps.rate(args.steps, ms)

    # ---- per-stage split (fwd / bwd ms) on the same state, untimed above ----
    stages = stage_split(tr, 20)

    # ---- plain 3DGS on the same state: all Gaussians active ----
    plain = plain_rate(tr, max(50, min(args.steps, 300)))

    # ---- roofline of the dominant kernel ----
    peaks, peak_kind = _peaks()
    rb_ms = [a.elapsed_time(b) for a, b, _ in raster_ev]
    rb_mean = sum(rb_ms) / len(rb_ms)
    pc = pair_counts(tr, [v for _, _, v in raster_ev])
    clk_summary = clk.summary()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * 128 * sm_max * 1e6 / 1e12  # FP32 lane-instructions per second, in T/s
    ops = OPS_BLENDED_ACTIVE * pc[0] + OPS_BLENDED_FROZEN * pc[1] + OPS_SKIPPED * pc[2]
    achieved = ops / (rb_mean / 1e3) / 1e12
    roofline = dict(bound="alu", kernel="k_raster_bwd", achieved=achieved, peak=alu_peak, unit="TFLOP/s",
                    frac=achieved / alu_peak, traffic=raster_bwd_traffic(),
                    work_per_unit=f"FP32 lane-instructions per (pixel, splat) pair the backward walks: each"
                                  f" pixel's list up to its last contributor or to just behind the tile's last"
                                  f" unfrozen entry (the frozen splats behind it are skipped): {OPS_BLENDED_ACTIVE}"
                                  f" blended by an unfrozen splat,"
                                  f" {OPS_BLENDED_FROZEN} by a frozen one, {OPS_SKIPPED} skipped; per launch"
                                  f" {pc[0]:.3e} / {pc[1]:.3e} / {pc[2]:.3e} pairs (gs_raster_pair_counts,"
                                  f" freeze map at the end of the timed region)",
                    peak_source=f"{sms} SMs (device) x 128 FP32 lanes x {sm_max:.0f} MHz (max SM clock, "
                                + ("measured peaks file)" if peak_kind == "measured" else
                                   "fallback figure: no measured peaks file)"),
                    mean_launch_ms=rb_mean)
    adam = stages.get("adam_roofline")
    project = stages.get("project_roofline")
    adam_all = plain.get("adam_roofline")

    # ---- end to end through the public API with host buffers ----
    e2e = e2e_rate(tr, max(30, min(args.steps, 200)))

    config = dict(workload=WORKLOAD["workload"], gaussians=WORKLOAD["n_init"], resolution=f"{W_}x{H_}", sh_degree=3,
                  tile=tr.view.cam.tile, raster_tuning=tuning, views=WORKLOAD["views"], densify=tr.cfg.densify,
                  gaussians_start=n_before, gaussians_end=tr.model.n, start_iter=k_start,
                  active_gaussians_start=active_before, active_gaussians_end=active_after,
                  thresholds_eps0=list(tr.eps0), l2="working set (P, G, m, v = 1 GB) larger than L2; no flush",
                  parallelism=f"replicas x{world}" if world > 1 else "single GPU")
    periodic = periodic_costs(tr)
    amortized_ms = ms / args.steps + periodic["amortized_ms_per_step"]
    periodic.update(ms_per_step=amortized_ms, its=1e3 / amortized_ms,
                    note="the timed iterations plus the periodic steps at their cadence (timed separately)")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene)

    ttp = None
    if world == 1 and not args.no_time_to_psnr:
        del tr, m
        torch.cuda.empty_cache()
        ttp = {"noiseless": time_to_psnr(scene), "target_noise_0.03": time_to_psnr(scene, 0.03)}

    batched = None
    if world == 1 and not args.no_batch:
        batched = batch_leg()

    if reps.printer:
        line = dict(metric=METRIC, value=its, unit="it/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                    data="synthetic",
                    config=config,
                    fwd_ms=stages["fwd_ms"], bwd_ms=stages["bwd_ms"], stage_ms=stages["stage_ms"],
                    plain_its=plain["its"], plain_stage_ms=plain["stage_ms"], gsta_speedup_vs_plain=its / world /
                    plain["its"],
                    roofline=roofline, roofline_adam=adam, roofline_adam_all_active=adam_all,
                    roofline_project=project, cpu_baseline=cpu, e2e=e2e, gpu_launches=launches,
                    clocks=clk_summary, device_flags=flags, amortized=periodic, time_to_psnr=ttp,
                    batched_scenes=batched)
        print(json.dumps(line), flush=True)
    reps.close()


# DRAM traffic of the dominant kernel per launch, from one ncu capture of this
# benchmark's own timed launches (dram__bytes_read.sum + dram__bytes_write.sum,
# averaged over the captured launches; profiles/k_raster_bwd_traffic_surface-1M-1237x822.md
# gives the command). Valid only for the kernel sources it was taken on: the
# digest of those files is compared at run time and traffic is reported as null
# once they have changed.
RASTER_BWD_TRAFFIC = dict(bytes_per_launch=86249472,
                          sources_sha256="bc6c9ed3d5d8c517458d919f3c4d49d3f942f36aafcd9879d92b9a0f869007bb")
RASTER_BWD_SOURCES = ("paper_2504_06716_gb300/csrc/render.cu", "paper_2504_06716_gb300/csrc/common.cuh")
# The same for Adam and the projection (profiles/k_adam_traffic_surface-1M-1237x822.md,
# profiles/k_project_fwd_traffic_surface-1M-1237x822.md):
# DRAM bytes per launch of three captured launches, with the launch's units
# (active Gaussians; the projection's algorithmic bytes), so that a run on
# another state scales the traffic by its own units.
ADAM_TRAFFIC = dict(bytes_per_launch=54777856, active=52186,
                    sources_sha256="9d8ebeb61c1b3774cceebad5438ced7db05608feaa78eef00845ec0860717c55")
ADAM_SOURCES = ("paper_2504_06716_gb300/csrc/optim.cu", "paper_2504_06716_gb300/csrc/common.cuh")
PROJECT_TRAFFIC = dict(bytes_per_launch=280659627, algorithmic_bytes=252735533,
                       sources_sha256="ebe0ce4ab160cf25a187e3a33c2d647e92ac4bb162f39343f6b5a945f363c0aa")
PROJECT_SOURCES = ("paper_2504_06716_gb300/csrc/project.cu", "paper_2504_06716_gb300/csrc/common.cuh")


def sources_digest(paths) -> str:
    import hashlib

    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for p in paths:
        with open(os.path.join(root, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def raster_bwd_traffic():
    t = RASTER_BWD_TRAFFIC
    if t["bytes_per_launch"] is None or t["sources_sha256"] != sources_digest(RASTER_BWD_SOURCES):
        return None
    return t["bytes_per_launch"]


def adam_traffic(active: int):
    """Captured Adam DRAM bytes per launch scaled to `active` Gaussians (null
    once the kernel's sources differ from the captured ones)."""
    t = ADAM_TRAFFIC
    if t["sources_sha256"] != sources_digest(ADAM_SOURCES):
        return None
    return round(t["bytes_per_launch"] * active / t["active"])


def project_traffic(algorithmic_bytes: float):
    t = PROJECT_TRAFFIC
    if t["sources_sha256"] != sources_digest(PROJECT_SOURCES):
        return None
    return round(t["bytes_per_launch"] * algorithmic_bytes / t["algorithmic_bytes"])


# Algorithmic FP32 work of the rasteriser backward per (pixel, splat) pair, counted
# from its formula (an FMA as two). Every pair: offset (2), exponent (8), exp and
# opacity (3), alpha floor/cap tests (3) = 16, all a skipped pair costs. A blended
# pair adds the transmittance recovery (2) and the colour-behind sum (dL/dC . c: 5,
# times alpha and T into the sum: 3) = 26, all a frozen splat's pair costs (no
# gradient, Sec. 3.2.4); an unfrozen splat's pair adds dL/dalpha (6), the colour
# gradient (7), the opacity and exponent moments (8) and its share of the conic
# and mean gradients formed from those moments (6) = 53. The pairs counted are the
# ones the resuming backward walks: each pixel's list up to its last contributor or
# to just behind the tile's last unfrozen entry, whichever comes first.
OPS_SKIPPED, OPS_BLENDED_FROZEN, OPS_BLENDED_ACTIVE = 16, 26, 53


def pair_counts(tr, views) -> list[float]:
    """(blended by an unfrozen splat, blended by a frozen splat, skipped) pairs
    per launch, averaged over the views of the timed launches (re-rendered
    after timing, on the final freeze map)."""
    import torch

    from paper_2504_06716_gb300 import lib

    m, view = tr.model, tr.view
    counts = torch.zeros(3, dtype=torch.int64, device=m.P.device)
    sample = views[:: max(1, len(views) // 16)]
    for v in sample:
        m.retarget(view, tr.cams[v])
        m.rasterize(view)
        lib.gs_raster_pair_counts(m.splats, view.vals, view.ranges, view.cam, view.n_last, m.frozen, counts)
    return [float(c) / len(sample) for c in counts.cpu().tolist()]


# Algorithmic bytes of the projection per Gaussian: a culled one reads its
# mean, scale, rotation and opacity (three 16-byte vectors) and writes a zero
# splat record (48 B); a visible one also reads its 48 SH coefficients
# (240 B in all) and writes its 48-byte record.
PROJECT_BYTES_CULLED = 48 + 48
PROJECT_BYTES_VISIBLE = 240 + 48


def stage_split(tr, n) -> dict:
    import torch

    from paper_2504_06716_gb300 import lib

    m, view = tr.model, tr.view
    names = ["project", "sort", "render", "loss", "raster_bwd", "project_bwd", "adam"]
    acc = {k: 0.0 for k in names}
    lrs = list(tr.lrs)
    proj_bytes = 0
    for i in range(n):
        v = tr.order[tr.k + i]
        m.retarget(view, tr.cams[v])
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        # the device waits ~0.5 ms while the host enqueues the whole sequence, so
        # each event pair brackets its kernel alone (no host launch gap inside)
        torch.cuda._sleep(1_000_000)
        ev[0].record()
        lib.gs_project(m.P, m.n, m.sh_degree, view.cam, m.splats)
        ev[1].record()
        lib.gs_sort(m.splats, m.n, view.cam, view.sort_ws, view.capacity, view.vals, view.ranges, view.count)
        ev[2].record()
        m.render_fwd(view)
        ev[3].record()
        m.loss(view, tr.targets[v])
        ev[4].record()
        m.raster_bwd(view)
        ev[5].record()
        lib.gs_project_bwd(m.P, m.n, m.sh_degree, view.cam, m.splats, m.act, m.n_active, m.grad2d, m.G, m.acc_xyz,
                           m.acc_rgb, m.cnt)
        ev[6].record()
        m.adam(lrs)
        ev[7].record()
        torch.cuda.synchronize()
        for j, k in enumerate(names):
            acc[k] += ev[j].elapsed_time(ev[j + 1])
        n_vis = int((m.splats[:m.n, 10].contiguous().view(torch.int32) > 0).sum().item())
        proj_bytes += n_vis * PROJECT_BYTES_VISIBLE + (m.n - n_vis) * PROJECT_BYTES_CULLED
    st = {k: v / n for k, v in acc.items()}
    peaks, kind = _peaks()
    proj_gbs = proj_bytes / n / (st["project"] / 1e3) / 1e9
    n_act = int(m.n_active.item())
    adam_bytes = n_act * 15 * 16 * 7  # read P, G, m, v and write P, m, v: 15 16-byte vectors each
    adam_gbs = adam_bytes / (st["adam"] / 1e3) / 1e9
    return dict(stage_ms=st, fwd_ms=st["project"] + st["sort"] + st["render"],
                bwd_ms=st["loss"] + st["raster_bwd"] + st["project_bwd"],
                adam_roofline=dict(bound="hbm", kernel="k_adam", achieved=adam_gbs, peak=peaks["hbm_gbs"],
                                   unit="GB/s", frac=adam_gbs / peaks["hbm_gbs"], traffic=adam_traffic(n_act),
                                   bytes_per_active_gaussian=15 * 16 * 7, active=n_act, peak_source=kind),
                project_roofline=dict(bound="hbm", kernel="k_project_fwd", achieved=proj_gbs, peak=peaks["hbm_gbs"],
                                      unit="GB/s", frac=proj_gbs / peaks["hbm_gbs"],
                                      traffic=project_traffic(proj_bytes / n),
                                      bytes_per_gaussian=dict(visible=PROJECT_BYTES_VISIBLE,
                                                              culled=PROJECT_BYTES_CULLED),
                                      gaussians=m.n, bytes_per_launch=round(proj_bytes / n), peak_source=kind))


def plain_rate(tr, n) -> dict:
    """Plain 3DGS iterations (no freezing) from the current state."""
    import torch

    m = tr.model
    saved = (m.frozen.clone(), m.act.clone(), m.n_active.clone())
    m.freeze_update(0.0, 0.0, 1)
    for i in range(5):
        v = tr.order[i]
        m.retarget(tr.view, tr.cams[v])
        m.train_step(tr.view, tr.targets[v], tr.lrs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(n):
        v = tr.order[i]
        m.retarget(tr.view, tr.cams[v])
        m.train_step(tr.view, tr.targets[v], tr.lrs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sp = stage_split(tr, 10)
    m.frozen.copy_(saved[0])
    m.act.copy_(saved[1])
    m.n_active.copy_(saved[2])
    return dict(its=n / (ms / 1e3), stage_ms=sp["stage_ms"], adam_roofline=sp["adam_roofline"])


def e2e_rate(tr, n) -> dict:
    """Same iterations through the public API with host buffers: each step copies
    its target image from pinned host memory and reads the loss back."""
    import torch

    from paper_2504_06716_gb300.pipeline import TargetFeeder

    m, view = tr.model, tr.view
    views = [tr.order[i] for i in range(n)]
    host = {v: tr.targets[v].cpu().pin_memory() for v in set(views)}
    feeder = TargetFeeder(tuple(tr.targets[views[0]].shape))
    loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
    done = torch.cuda.Event()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    feeder.prefetch(host[views[0]])
    for i, v in enumerate(views):
        gt = feeder.take()
        m.retarget(view, tr.cams[v])
        m.train_step(view, gt, tr.lrs)
        feeder.release()
        if i + 1 < n:
            feeder.prefetch(host[views[i + 1]])  # the next upload overlaps this step
        loss_host.copy_(view.loss, non_blocking=True)
        done.record()
        done.synchronize()  # the step's loss is on the host
    dt = time.perf_counter() - t0
    return dict(value=n / dt, unit="it/s", h2d_bytes_per_step=int(feeder.bufs[0].numel() * 4), d2h_bytes_per_step=4,
                note="host-pinned target upload (the next step's overlapping the current one, two device buffers) "
                     "and loss read-back every step; freeze map as in the timed region")


def _reach(evals, target):
    """(wall seconds, iteration) of the first evaluation at or above target, or None."""
    for e in evals:
        if e["heldout_psnr"] >= target:
            return e["wall_s"], e["k"]
    return None


def time_to_psnr(scene, target_noise: float = 0.0) -> dict:
    """Held-out PSNR against training wall time for plain 3DGS and for GSta
    (its freeze rule, early stop and schedule), trained from the same
    initialisation, views and seeds with densification, each after its own
    launch-shape autotuning. The target is plain 3DGS's final held-out PSNR
    minus 0.1 dB; held-out PSNR is evaluated every 1000 iterations, and its
    evaluations are not counted as training time. target_noise > 0 adds
    seeded per-pixel noise of that standard deviation to every target image
    (a captured image's sensor noise), which bounds the reachable PSNR as the
    paper's real scenes do."""
    import torch

    from paper_2504_06716_gb300 import train

    runs = {}
    for arm in ("plain", "gsta"):
        args = train.parser().parse_args(["--arm", arm, "--autotune", "--eval-every", "1000", "--target-noise",
                                          str(target_noise)])
        runs[arm] = train.run(args, scene)
        torch.cuda.synchronize()
    plain, gsta = runs["plain"], runs["gsta"]
    target = plain["final_heldout_psnr"] - 0.1
    out = dict(target_noise=target_noise, target_db=target,
               rule="held-out PSNR (every 8th view) >= plain 3DGS final - 0.1 dB, checked every 1000 iterations; "
                    "training wall time, held-out evaluations excluded")
    for arm, r in runs.items():
        hit = _reach(r["evals"] + [dict(k=r["iters"], wall_s=r["train_s"], heldout_psnr=r["final_heldout_psnr"])],
                     target)
        stop = [e[0] for e in r["events"] if e[1] == "early_stop"]
        out[arm] = dict(final_db=r["final_heldout_psnr"], train_s=r["train_s"], iters=r["iters"],
                        s_to_target=None if hit is None else hit[0], iter_at_target=None if hit is None else hit[1],
                        early_stop_iter=stop[0] if stop else None, gaussians_end=r["n_final"],
                        curve=[[e["k"], round(e["wall_s"], 2), round(e["heldout_psnr"], 3)] for e in r["evals"]])
    eq = _reach(plain["evals"], gsta["final_heldout_psnr"])
    out["gsta_within_0.1db_of_plain_final"] = gsta["final_heldout_psnr"] >= target
    out["train_time_ratio_plain_over_gsta"] = plain["train_s"] / gsta["train_s"]
    out["equal_quality"] = dict(db=gsta["final_heldout_psnr"], gsta_s=gsta["train_s"],
                                plain_s=None if eq is None else eq[0], plain_iter=None if eq is None else eq[1])
    return out


def batch_leg(steps: int = 40, warmup: int = 8, pretrain: int = 300) -> dict:
    """Several scenes per step (the batched workload): 8 scenes of 50K to 2M
    Gaussians (5.72M in all), 4 views of each at 800x800 per step, one
    persistent compositing and one persistent backward launch over the 32
    (scene, view) jobs, each step replayed from a CUDA graph; tile size and
    launch shapes from the batch's own autotuner; CUDA events over `steps`
    replayed steps after `pretrain` + `warmup` steps."""
    import torch

    from paper_2504_06716_gb300 import batch
    from paper_2504_06716_gb300.schedule import GStaConfig

    t0 = time.perf_counter()
    bt = batch.BatchTrainer(batch.make_scenes(), GStaConfig())
    setup_s = time.perf_counter() - t0
    tuning = batch.tune(bt)
    for _ in range(pretrain):
        bt.step("graph")
    r = batch.measure(bt, steps, warmup, "graph")
    out = dict(workload="8 scenes of 50K-2M Gaussians (5.72M), 4 views each at 800x800 per step",
               ms_per_step=r["ms_per_step"], gaussian_views_per_s=r["gaussian_views_per_s"],
               launches_per_step=r["launches_per_step"], steps=steps, start_step=pretrain + warmup,
               tuning=dict(tile=tuning["tile"], fwd_ppt_batch=list(tuning["fwd"]), bwd_ppt_batch=list(tuning["bwd"])),
               setup_s=setup_s, timing="CUDA events around the replayed steps on the launching stream")
    del bt
    torch.cuda.empty_cache()
    return out


def periodic_costs(tr) -> dict:
    """Milliseconds of the work GSta does only every so many iterations,
    measured on the bench state at the end (they change it): a densification
    step (every 100 iterations in the window), a freeze-map update (every 250)
    and the subset-PSNR check of Eq. 7 (every 1000)."""
    import torch

    from paper_2504_06716_gb300.schedule import FREEZE_UPDATE

    def wall(fn, reps=1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0) / reps

    k = tr.k
    psnr = wall(lambda: tr.psnr_of(tr.scene.subset_views), 2)
    ex, er = tr.thresholds(k)
    freeze = wall(lambda: tr.model.freeze_update(ex, er, FREEZE_UPDATE), 3)
    den = wall(lambda: tr._densify(k), 1)
    return dict(densify_ms=den, densify_every=tr.cfg.den_every, freeze_update_ms=freeze, freeze_every=tr.cfg.every,
                psnr_check_ms=psnr, psnr_every=tr.cfg.psnr_every,
                amortized_ms_per_step=den / tr.cfg.den_every + freeze / tr.cfg.every + psnr / tr.cfg.psnr_every)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gsta", "reference"], default="gsta")
    ap.add_argument("--start-iter", type=int, default=4750)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep 16-pixel tiles and default launch shapes")
    ap.add_argument("--no-batch", action="store_true", help="skip the several-scene step (about a minute)")
    ap.add_argument("--no-time-to-psnr", action="store_true",
                    help="skip the four full training runs of the time-to-PSNR comparison (about three minutes)")
    ap.add_argument("--views", type=int, default=WORKLOAD["views"],
                    help="train on the first N training views only (smaller device footprint for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
