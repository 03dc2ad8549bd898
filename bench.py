#!/usr/bin/env python
"""Benchmark of the layered UTR reconstruction on synthetic seeded workloads.

A step is one ``recon_run`` over the whole workload: every direction through the
FFT / per-layer CTF filter / inverse FFT stage and the layered backprojection, with
the images already resident in HBM.  The metric is voxel x direction updates per
second (U = V * D per step).  One JSON line is printed by rank 0.

``--impl reference`` times the FP64 CPU oracle instead (a bounded sample of the
same workload per step, on the host cores).

Multi-GPU: the reconstruction has no exchange step on one GPU's worth of work, so
``--gpus N`` (under torchrun) runs N independent replicas, one seeded tomogram per
rank, and reports the aggregate (weak scaling)."""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel×direction updates/s at stated rel-L2 vs FP64 oracle; % HBM roofline"
UNIT = "updates/s"

WORKLOAD_TEXT = {
    "mid": ("mid-size plain method: 256^3 grid (0.1 nm voxels), 360 single-axis directions over 180 deg, "
            "256x256 float32 images, 300 keV electrons (lambda 1.97 pm), Nz=32 depth layers, defocus 1 um, "
            "Cs 2.7 mm, sigma 0.07, eps 0.1; 2e4 Gaussian pseudo-atoms (s 0.1 nm, weights U[1,8]); "
            "multislice images with 100 e/px Poisson noise"),
    "small": ("small plain method: 64^3 grid (1 nm voxels), 90 single-axis directions over 180 deg, 64x64 "
              "float32 images, lambda 0.1 nm, Nz=8 depth layers, R_n ~ U[100,120] nm, sigma 0.01, eps 0.01; "
              "20 uniform balls (r U[2,8] vox, delta U[1e-6,1e-5]); multislice images, 1e4 photons/px"),
    "learned": ("learned-filter scan: 512^3 grid (0.1 nm voxels), 720 single-axis directions over 180 deg, "
                "512x512 float32 images, lambda 1.97 pm, Nz=64 layers, R_n ~ U[0.5,1.5] um, Cs 2.7 mm, sigma "
                "0.07, eps 0.1; 1.6e5 Gaussian pseudo-atoms; 100 e/px (--filter mlp: the trained network)"),
    "slab": ("arbitrary geometry, large slab: 1024x1024x256 grid (0.05 nm voxels), 1500 Haar-random directions "
             "within 60 deg of the slab normal, 1024x1024 float32 images, lambda 1.97 pm, Nz=64 layers, R 1 um, "
             "Cs 2.7 mm, sampling-density weighting; 2e5 Gaussian pseudo-atoms filling the slab; 50 e/px"),
    "batch": ("batched: 48 tomograms of uneven sizes (64^3-256^3 grids, 64^2-256^2 images, 60-360 single-axis "
              "directions, Nz 4-32), balls and blobs, soft X-ray and electron physics, one graph replay"),
}
# stack precision each workload is specified with
DEFAULT_STACK = {"mid": "f32", "small": "f32", "learned": "bf16", "slab": "bf16", "batch": "bf16"}

# DRAM traffic per launch (bytes) from ncu captures, keyed by kernel and workload and
# valid only for the kernel source they were taken on (sha256 of the .cu file).  The column
# kernels' entries were re-stamped once, after a change to stage_a.cu that touched only the row
# kernel (its FFT call now asks the engine for twiddle powers, a template branch the column
# kernels do not take): their code is the captured code.
NCU_TRAFFIC: dict = {
    # mid (float32): one 40-direction launch each, scaled by 120/40 to the bench's blocks (the
    # backprojection's volume read-modify-write does not scale; its figure overstates it)
    ("k_cols", "mid", "f32"): {"bytes_per_launch": (21.171456e6 + 612.15744e6) * 3, "l2_hit_pct": 3.8,
                               "src": "12ea9f939a270171"},
    ("k_backproject", "mid", "f32"): {"bytes_per_launch": (617.094656e6 + 59.883008e6) * 3, "l2_hit_pct": 51.1,
                                      # 171.8 M warp instructions for 40 x 256^3 updates
                                      "warp_inst_per_update": 171823104 / (40 * 256 ** 3),
                                      "src": "b7ee0b8780a4373d"},
    # slab (bf16 stack): the column kernel from one 3-direction sub-block launch (the bench's
    # launch size); the TMA-staged backprojection from a 6-direction launch, its reads scaled
    # by 56/6 to the bench's 56-direction blocks (the stack boxes grow with the directions),
    # plus the volume read of an accumulating block and the volume write (1.07 GB each)
    ("k_cols", "slab", "bf16"): {"bytes_per_launch": 55.945984e6 + 1.550934e9, "l2_hit_pct": 8.4,
                                 "src": "12ea9f939a270171"},
    ("k_backproject", "slab", "bf16"): {"bytes_per_launch": 3.059654e9 * 56 / 6 + 1.073742e9 + 1.055155e9,
                                        "l2_hit_pct": 56.2,
                                        # 1.553 G warp instructions for 6 x 1024^2 x 256 updates
                                        "warp_inst_per_update": 1553227094 / (6 * 1024 * 1024 * 256),
                                        "src": "f76a56888e3e5455"},
}


# The roof that binds each stage-A kernel (ncu evidence in profiles/): FP32 arithmetic for the
# column FFT and filter, the L1 / shared-memory pipe for the row stage; the forward row FFTs
# are small and memory-bound.  The backprojection's depends on the kernel that ran.
KERNEL_BOUND = {"k_rows_fwd": "hbm", "k_cols": "alu (FP32)", "k_rows_inv": "l1/shared-memory pipe"}
ISSUE_PEAK = 152 * 4 * 2.07e9  # warp instructions per second


def ncu_traffic(kernel: str, workload: str, stack: str, filt: str):
    """The captured entry for this kernel and workload, or None.  The stage-A captures are of
    the Tikhonov filter's kernels; another filter is another kernel instantiation."""
    if kernel != "k_backproject" and filt != "tikhonov":
        return None
    return NCU_TRAFFIC.get((kernel, workload, stack))


def _src_hash(name: str) -> str:
    p = os.path.join(ROOT, "paper_2206_09151_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"]}, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ----------------------------------------------------------------------------- workload
def workload(name: str, rank: int = 0, dirs: int | None = None):
    from paper_2206_09151_gb300 import phantoms as ph
    cfg = ph.config_workload(name, scale_dirs=dirs)
    cfg["seed"] = cfg["seed"] + 100 * rank
    return cfg


def make_images(cfg, device):
    import torch

    from paper_2206_09151_gb300 import phantoms as ph
    return ph.make_images(cfg, device=device, dtype=torch.float32)


# volumes above this many voxels are compared with the oracle on a random voxel sample
FULL_VOLUME_LIMIT = 1 << 24


def sample_voxels(cfg):
    """None (the full volume) for volumes up to 2^24 voxels, else 2^18 seeded random voxels."""
    V = int(np.prod(cfg["grid"]))
    if V <= FULL_VOLUME_LIMIT:
        return None
    rng = np.random.default_rng(cfg["seed"] + 99)
    nx, ny, nz = cfg["grid"]
    n = 1 << 18
    return rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)


def oracle_sample(cfg, images_np, dirs, mlp=None, voxels=None, workers: int = 1, layer_interp: str = "nearest"):
    """FP64 oracle on the directions ``dirs`` alone (a D = len(dirs) scan), at ``voxels`` or
    over the full volume, in ``workers`` processes; ``mlp`` = (weights, nsr) selects the
    learned regulariser (with ``views``, the divisor of its eps); ``layer_interp`` the
    nearest layer or the blend of the two bracketing ones."""
    import oracle as O
    kw = dict(lam=cfg["lam"], delta=cfg["delta"], defocus=cfg["defocus"][dirs], nz_layers=cfg["nz_layers"],
              grid=cfg["grid"], sigma=cfg["sigma"], cs=cfg["cs"], voxels=voxels, workers=workers,
              density=cfg.get("ramp", "single_axis") == "density")
    if cfg.get("filter") == "pair":
        return O.recon(images_np[dirs], cfg["rot"][dirs], eps=cfg["eps"], filt=O.FILTER_PAIR,
                       layer_interp=O.LAYER_LINEAR if layer_interp == "linear" else O.LAYER_NEAREST, **kw)
    if mlp is not None:
        return O.learned.recon_learned(images_np[dirs], cfg["rot"][dirs], mlp[0].astype(np.float64), nsr=mlp[1],
                                       views=mlp[2],
                                       **kw)
    return O.recon(images_np[dirs], cfg["rot"][dirs], eps=cfg["eps"],
                   layer_interp=O.LAYER_LINEAR if layer_interp == "linear" else O.LAYER_NEAREST, **kw)


# ----------------------------------------------------------------------------- reference arm
def host_cpu() -> tuple[int, str]:
    """Host cores the oracle's process pool uses, and the CPU model."""
    cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                             timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return cores, model


def oracle_timed(cfg, images_np, dirs, workers, mlp=None, voxels=None, layer_interp: str = "nearest"):
    """The FP64 oracle on the directions ``dirs`` (a scan of its own) over ``voxels``,
    spread over ``workers`` spawned processes; returns (result, wall seconds)."""
    t0 = time.perf_counter()
    ref = oracle_sample(cfg, images_np, dirs, mlp, voxels, workers, layer_interp)
    return ref, time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import torch
    if args.workload == "batch":  # the oracle on one member of the batch
        from paper_2206_09151_gb300 import phantoms as ph
        cfg = ph.batch_workloads()[0]
    else:
        cfg = workload(args.workload)
    cores, model = host_cpu()
    vox = sample_voxels(cfg)
    V = int(np.prod(cfg["grid"])) if vox is None else vox[0].size
    D = cfg["n_dir"]
    # one direction per step; the warm-up steps and then the timed steps each run as one
    # batch of directions spread over the host cores
    order = [(s * 97) % D for s in range(args.warmup + args.steps)]
    need = sorted(set(order))
    sub = dict(cfg, rot=cfg["rot"][need], defocus=cfg["defocus"][need])
    images = np.zeros((D, cfg["nv"], cfg["nu"]), np.float32)
    images[need] = make_images(sub, "cpu").numpy()  # only the sampled views are simulated
    warm, timed = order[:args.warmup], order[args.warmup:]
    oracle_timed(cfg, images, warm, min(cores, len(warm)), voxels=vox)
    _, t = oracle_timed(cfg, images, timed, min(cores, len(timed)), voxels=vox)
    value = V * len(timed) / t
    where = "the full volume" if vox is None else f"{V} random voxels"
    sample = (f"{len(timed)} directions (one per step) over {where} of the {'x'.join(map(str, cfg['grid']))} grid"
              + (" (first tomogram of the batch)" if args.workload == "batch" else "")
              + f", FP64 numpy oracle in {min(cores, len(timed))} spawned processes on {cores} host cores ({model});"
              f" each direction's FFT / per-layer filter work is done in full, the backprojection on the voxel set")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / len(timed),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(cores, len(timed)), "host_cores": cores,
                             "cpu_model": model, "kind": "oracle", "sample": sample, "seconds": t},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    del torch
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- replicas
def max_over_ranks(value: float, device=None) -> float:
    """The largest ``value`` over the ranks of the default process group (the slowest
    replica's time); the value itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_step: float, steps: int, world: int, total_ms_max: float) -> float:
    """Whole-job throughput of ``world`` independent replicas, each doing ``units_per_step``
    per step, timed by the slowest one."""
    return world * units_per_step * steps / (total_ms_max / 1e3)


# ----------------------------------------------------------------------------- our arm
KERNELS = ["k_rows_fwd", "k_cols", "k_rows_inv", "k_backproject"]


def algorithmic_bytes(cfg, r, stack_bytes: int, dir_counts: list[int]) -> list[float]:
    """Bytes each kernel must move per run (inputs read once, outputs written once)."""
    nu, nv, nzl = cfg["nu"], cfg["nv"], cfg["nz_layers"]
    half = r.padded // 2 + 1
    V = int(np.prod(cfg["grid"]))
    out = [0.0, 0.0, 0.0, 0.0]
    for b, nb in enumerate(dir_counts):
        spec = nb * nv * half * 8
        inter = nb * nzl * nv * half * 8
        stack = nb * nzl * (nv + 2) * (nu + 2) * stack_bytes
        out[0] += nb * nv * nu * 4 + spec
        out[1] += spec + inter
        out[2] += inter + stack
        out[3] += stack + V * (4 if b == 0 else 8)
    return out


# FP32 peak of the column-filter kernel's roofline: 152 SMs x 128 FP32 lanes x 2 flops (FMA)
# x 2070 MHz maximum SM clock.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12


def cols_flops(cfg, r, dir_counts: list[int]) -> float:
    """FP32 work of the column kernel per run: a length-P complex FFT counted as
    5 P log2 P flops, one forward and Nz inverse transforms per half-spectrum column,
    and the real per-layer filter applied to every complex coefficient (2 flops)."""
    P, nzl = r.padded, cfg["nz_layers"]
    half = P // 2 + 1
    fft = 5.0 * P * math.log2(P)
    return float(sum(dir_counts)) * half * ((1 + nzl) * fft + nzl * 2.0 * P)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2206_09151_gb300 import _abi
    from paper_2206_09151_gb300.build import build
    from paper_2206_09151_gb300.recon import Reconstructor
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    cfg = workload(args.workload, rank, args.dirs)
    if args.filter == "pair":
        # the opposite-pair form needs every view's opposite: the same number of single-axis
        # views spread over 360 degrees instead of 180
        from paper_2206_09151_gb300 import phantoms as ph
        cfg["rot"] = ph.single_axis_rotations(cfg["n_dir"], span=2 * np.pi)
        cfg["filter"] = "pair"
    images = make_images(cfg, dev)
    torch.cuda.synchronize()
    V = int(np.prod(cfg["grid"]))
    D = cfg["n_dir"]
    U = V * D
    filt_kw = {"filter": "pair"} if args.filter == "pair" else {}
    mlp = None
    if args.filter == "mlp":
        # the trained regulariser; its per-view eps divided by the D views the volume averages
        from paper_2206_09151_gb300.train_regulariser import load_weights
        mlp = (load_weights(), float(cfg["photons"]) ** -0.5, float(D))
        filt_kw = dict(filter="mlp", mlp_weights=mlp[0], nsr=mlp[1], mlp_views=mlp[2])
    r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                      defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
                      cs=cfg["cs"], stack_dtype=args.stack, dir_block=args.dir_block, stage_block=args.stage_block,
                      bp_kernel=args.bp_kernel, ramp=cfg["ramp"], layer_interp=args.layer_interp, device=dev,
                      **filt_kw)
    vol = r.new_volume()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(args.warmup):
        r.run(images, vol)
    torch.cuda.synchronize()

    _abi.recon_profile_enable(r.plan, True)
    kern_ms = [0.0] * 4
    kern_n = [0] * 4
    sampler = ClockSampler(gpu_index(local))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush, outside the timed span
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.run(images, vol, stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ms, n = _abi.recon_profile_read(r.plan)
        for q in range(4):
            kern_ms[q] += ms[q]
            kern_n[q] += n[q]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    _abi.recon_profile_enable(r.plan, False)
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = aggregate_rate(U, args.steps, world, total_ms)

    # end to end through the public API: pinned host images in (recon_run_host, which uploads
    # each direction block on a stream of its own while the previous block is reconstructed),
    # volume out, every step
    host_img = images.cpu().pin_memory()
    host_vol = torch.empty(vol.shape, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r.run_host(host_img, vol, stream)
        host_vol.copy_(vol, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if s >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms), dev)
    e2e_value = aggregate_rate(U, args.steps, world, e2e_total)

    # roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    db, nb = r.dir_block, r.n_blocks
    counts = [min(db, D - b * db) for b in range(nb)]
    algo = algorithmic_bytes(cfg, r, 2 if args.stack == "bf16" else 4, counts)
    kernels = {}
    bp_src = "backproject_tma.cu" if r.bp_kernel_used == "tma" else "backproject.cu"
    for q, name in enumerate(KERNELS):
        per_launch_ms = kern_ms[q] / max(kern_n[q], 1)
        gbs = algo[q] / (kern_ms[q] / args.steps / 1e3) / 1e9 if kern_ms[q] > 0 else None
        tr = ncu_traffic(name, args.workload, args.stack, args.filter)
        src = bp_src if q == 3 else "stage_a.cu"
        valid = tr is not None and tr["src"] == _src_hash(src)
        kernels[name] = {"launches": kern_n[q], "ms_per_launch": per_launch_ms,
                         "share": kern_ms[q] / max(sum(kern_ms), 1e-12), "algorithmic_GBps": gbs,
                         "algorithmic_bytes_per_launch": algo[q] * args.steps / max(kern_n[q], 1),
                         "ncu_dram_bytes_per_launch": tr["bytes_per_launch"] if valid else None,
                         "bound": KERNEL_BOUND[name] if q < 3 else
                         ("issue (FMA/ALU pipes)" if r.bp_kernel_used == "tma" else "l1 (gathers)")}
        if valid and per_launch_ms > 0:
            # the captured bytes at the bench's launch time, against the measured HBM peak
            kernels[name]["ncu_dram_frac"] = tr["bytes_per_launch"] / (per_launch_ms / 1e3) / 1e9 / peaks["hbm_gbs"]
            kernels[name]["ncu_l2_hit_pct"] = tr.get("l2_hit_pct")
            if "warp_inst_per_update" in tr and kern_ms[q] > 0:
                # issue roofline: warp instructions per update (ncu) x updates/s, against
                # 152 SMs x 4 schedulers x 2070 MHz
                ups = V * D * args.steps / (kern_ms[q] / 1e3)
                kernels[name]["issue_frac"] = tr["warp_inst_per_update"] * ups / ISSUE_PEAK
    flops = cols_flops(cfg, r, counts)
    kernels["k_cols"]["algorithmic_TFLOPs"] = (flops / (kern_ms[1] / args.steps / 1e3) / 1e12
                                               if kern_ms[1] > 0 else None)
    dom = max(range(4), key=lambda q: kern_ms[q])
    dom_name = KERNELS[dom]
    src = bp_src if dom == 3 else "stage_a.cu"
    tr = ncu_traffic(dom_name, args.workload, args.stack, args.filter)
    traffic = tr["bytes_per_launch"] if tr and tr["src"] == _src_hash(src) else None
    launches = max(kern_n[dom], 1)
    common = {"kernel": dom_name, "traffic": traffic,
              "algorithmic_bytes_per_launch": algo[dom] * args.steps / launches, "launches": kern_n[dom],
              "ms_per_launch": kern_ms[dom] / launches,
              "units_per_launch": (V * D if dom == 3 else D) * args.steps / launches}
    if dom == 1:
        # the column kernel is bound by FP32 arithmetic (FFTs and the per-layer filter):
        # its flops over its summed launch time, against the FP32 peak of the SM count and clock
        achieved = flops * args.steps / (kern_ms[dom] / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS,
                    "peak_source": "FP32: 152 SMs x 128 lanes x 2 flops x 2070 MHz",
                    "algorithmic_flops_per_launch": flops * args.steps / launches, **common}
    else:
        # bytes of all launches over their summed time (a launch is a block or a sub-block)
        achieved = algo[dom] * args.steps / (kern_ms[dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else
                    "fallback 6.8 TB/s", **common}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.stack, "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload] + (f" [first {D} directions only]" if args.dirs else "")
                       + (" [the views spread over 360 degrees for the opposite-pair filter]"
                          if args.filter == "pair" else ""),
                       "stack": args.stack, "filter": args.filter, "dir_block": db,
                       "stage_block": r.stage_block, "bp_kernel": args.bp_kernel,
                       "bp_kernel_used": r.bp_kernel_used, "layer_interp": args.layer_interp,
                       "blocks": nb, "padded_fft": r.padded, "updates_per_step": U,
                       "l2": "flushed between timed steps (256 MiB write outside the timed span)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "api": "recon_run_host (pinned host images, upload overlapped)",
                    "h2d_bytes_per_step": images.numel() * 4,
                    "d2h_bytes_per_step": vol.numel() * 4},
            "gpu_launches": sum(kern_n) + (2 * kern_n[0] if args.filter == "mlp" else 0), "roofline": roofline, "kernels": kernels, "clocks": clocks}

    if rank == 0 and world == 1 and args.filter == "mlp":
        # learned against analytic regulariser on the same GPU: speed, and the error of each
        # against the phantom (pseudo-atoms sampled at the voxel centres) over the field of view
        from paper_2206_09151_gb300 import phantoms as ph
        from paper_2206_09151_gb300.layer_study import phantom_volume
        truth = phantom_volume(ph.make_phantom(cfg), cfg["grid"], dev)
        nx, ny, nz = cfg["grid"]
        if cfg["ramp"] == "single_axis":
            xx = torch.arange(nx, device=dev, dtype=torch.float64) - (nx - 1) / 2
            zz = torch.arange(nz, device=dev, dtype=torch.float64) - (nz - 1) / 2
            fov = ((xx[None, :] ** 2 + zz[:, None] ** 2) <= (0.5 * min(nx, nz) - 2) ** 2)[:, None, :].expand(nz, ny, nx)
        else:
            fov = torch.ones((nz, ny, nx), dtype=torch.bool, device=dev)
        compare = {}
        for name, kw in (("learned", filt_kw), ("tikhonov eps=%g" % cfg["eps"], {})):
            rr = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                               defocus=cfg["defocus"], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
                               cs=cfg["cs"], stack_dtype=args.stack, dir_block=args.dir_block, ramp=cfg["ramp"],
                               device=dev, **kw)
            vv = rr.new_volume()
            rr.run(images, vv)
            torch.cuda.synchronize()
            ts = []
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rr.run(images, vv, stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            err = float(torch.linalg.norm((vv.double() - truth)[fov]) / torch.linalg.norm(truth[fov]))
            compare[name] = {"ms_per_step": min(ts), "rel_l2_vs_phantom": err}
            rr.close()
            del vv
        line["learned_vs_analytic"] = dict(compare, nsr=mlp[1], mlp_views=D,
                                           weights="paper_2206_09151_gb300/data/regulariser.npz")
        del truth
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample (a few directions spread over the host cores), beside
        # the same sample reconstructed on the GPU: the stated accuracy and the CPU rate
        cores, model = host_cpu()
        n_sel = args.cpu_dirs if args.cpu_dirs else cores
        sel = [int(x) for x in np.linspace(0, D - 1, n_sel).round()]
        img_np = images.cpu().numpy()
        vox = sample_voxels(cfg)
        workers = min(cores, len(sel))
        ref, dt = oracle_timed(cfg, img_np, sel, workers, mlp, vox, args.layer_interp)
        rs = Reconstructor(cfg["rot"][sel], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                           defocus=cfg["defocus"][sel], nz_layers=cfg["nz_layers"], sigma=cfg["sigma"],
                           eps=cfg["eps"], cs=cfg["cs"], stack_dtype=args.stack, ramp=cfg["ramp"], device=dev,
                           bp_kernel=args.bp_kernel, layer_interp=args.layer_interp, **filt_kw)
        got = rs.run(images[sel].contiguous())
        rs.close()
        if vox is None:
            got = got.cpu().numpy()
            n_vox, where = V, "the full volume"
        else:
            got = got[tuple(torch.as_tensor(x, device=dev) for x in vox[::-1])].cpu().numpy()
            n_vox, where = vox[0].size, f"{vox[0].size} random voxels"
        rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        sample = (f"{len(sel)} of {D} directions (a scan of their own) over {where} ({len(sel) * n_vox:.3e} updates),"
                  f" FP64 numpy oracle in {workers} spawned processes on {cores} host cores ({model}); each "
                  f"direction's FFT / per-layer filter work is done in full")
        line["cpu_baseline"] = {"value": len(sel) * n_vox / dt, "unit": UNIT, "cores": workers, "host_cores": cores,
                                "cpu_model": model, "kind": "oracle", "sample": sample, "seconds": dt}
        line["accuracy"] = {"rel_l2_vs_fp64_oracle": rel, "sample": sample,
                            "target": 1e-5 if args.stack == "f32" else 3e-3}
    if rank == 0:
        print(json.dumps(line))
    r.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """48 uneven tomograms (``phantoms.batch_workloads``) reconstructed together: stage A per
    tomogram and one persistent backprojection per round, the whole step captured once as a
    CUDA graph and replayed.  ``value`` is the voxel x direction updates of all 48 per second."""
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2206_09151_gb300 import phantoms as ph
    from paper_2206_09151_gb300.build import build
    from paper_2206_09151_gb300.recon import Batch, Reconstructor
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    cfgs = ph.batch_workloads(seed=4001 + 100 * rank)
    images = [make_images(c, dev) for c in cfgs]
    recons = [Reconstructor(c["rot"], c["nu"], c["nv"], c["grid"], lam=c["lam"], delta=c["delta"],
                            defocus=c["defocus"], nz_layers=c["nz_layers"], sigma=c["sigma"], eps=c["eps"],
                            cs=c["cs"], stack_dtype=args.stack, device=dev, allocate=False) for c in cfgs]
    tuned = None
    if args.dir_block <= 0:  # the round size from the autotuner (timed before the measured region)
        from paper_2206_09151_gb300.autotune import tune_batch_round
        tuned = tune_batch_round(recons, images, candidates=(16, 32, 64), repeats=1)
    dbb = args.dir_block if args.dir_block > 0 else tuned["dir_block"]
    b = Batch(recons, dir_block=dbb)
    vols = [r.new_volume() for r in recons]
    U = sum(int(np.prod(c["grid"])) * c["n_dir"] for c in cfgs)
    rounds = max((c["n_dir"] + dbb - 1) // dbb for c in cfgs)
    # kernels per replay: per round, stage A (3 launches) for every tomogram still active,
    # and one persistent backprojection
    launches = sum(3 * sum(1 for c in cfgs if rr * dbb < c["n_dir"]) + 1 for rr in range(rounds))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        b.run(images, vols, graph=True)  # the first run captures, the others replay
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index(local))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(images, vols, graph=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = aggregate_rate(U, args.steps, world, total_ms)
    # end to end: pinned host images in through recon_batch_run_host (round r + 1 uploads
    # while round r runs), volumes out, every step
    host_img = [im.cpu().pin_memory() for im in images]
    host_vol = [torch.empty(v.shape, dtype=torch.float32).pin_memory() for v in vols]
    e2e_ms = []
    for st in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run_host(host_img, vols, stream=stream)
        for h, v in zip(host_vol, vols):
            h.copy_(v, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if st >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = aggregate_rate(U, args.steps, world, max_over_ranks(sum(e2e_ms), dev))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.stack, "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT["batch"], "tomograms": len(cfgs), "round_directions": dbb,
                       "round_tuning_ms": tuned["ms"] if tuned else None,
                       "rounds": rounds, "updates_per_step": U, "stack": args.stack,
                       "l2": "flushed between timed steps (256 MiB write outside the timed span)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "api": "recon_batch_run_host (pinned host images, upload "
                    "overlapped)", "h2d_bytes_per_step": sum(im.numel() * 4 for im in images),
                    "d2h_bytes_per_step": sum(v.numel() * 4 for v in vols)},
            "gpu_launches": launches * args.steps,
            "roofline": None,
            "roofline_note": "the graph replay has no per-kernel events; the kernels are those of the single "
                             "runs, whose rooflines the mid workload reports",
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    b.close()
    for r in recons:
        r.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_fourier(args):
    """The two 3D-Fourier forms on one GPU: Eq. 12's swapped order (``--form swap``: the CT step
    with the Ewald placement, then one 3D CTF inversion) and the Fourier-gridding UTR
    (``--form grid``: the bracket per view splatted onto the Ewald paraboloids, S_eps^-1, one
    inverse 3D FFT).  A step is one whole reconstruction; the swap's 3D inversion alone (the
    cost of every further (sigma, eps)) is reported beside it."""
    import torch
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("--form swap / grid runs on one GPU")
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2206_09151_gb300.build import build
    from paper_2206_09151_gb300.recon import Reconstructor
    build()
    cfg = workload(args.workload, 0, args.dirs)
    images = make_images(cfg, dev)
    torch.cuda.synchronize()
    V = int(np.prod(cfg["grid"]))
    D = cfg["n_dir"]
    U = V * D
    R = float(np.mean(cfg["defocus"]))  # Eq. 12 needs one defocus for every view
    r = Reconstructor(cfg["rot"], cfg["nu"], cfg["nv"], cfg["grid"], lam=cfg["lam"], delta=cfg["delta"],
                      defocus=np.full(D, R), nz_layers=cfg["nz_layers"], sigma=cfg["sigma"], eps=cfg["eps"],
                      cs=cfg["cs"], stack_dtype="f32", ramp=cfg["ramp"],
                      filter="pair" if args.form == "swap" else "tikhonov", device=dev)
    vol = r.new_volume()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    nsr = float(cfg["photons"]) ** -0.5 if args.form == "grid" else 0.0

    def step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        if args.form == "swap":
            ws = r.swap_ct(images)
            e1.record(stream)
            r.swap_phase(ws, cfg["sigma"], cfg["eps"], vol)
        else:
            r.grid_run(images, nsr, vol)
            e1.record(stream)
        e2.record(stream)  # e1 -> e2: the swap's 3D inversion inside the step
        e2.synchronize()
        return e0.elapsed_time(e2), e1.elapsed_time(e2)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    sampler = ClockSampler(gpu_index(0))
    sampler.start()
    time.sleep(0.3)
    ms, tail_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        a, b = step()
        ms.append(a)
        tail_ms.append(b)
    clocks = sampler.stop()
    ms_step = sum(ms) / args.steps
    # the swap's 3D inversion alone, timed on its own (the per-(sigma, eps) cost)
    phase_ms = None
    if args.form == "swap":
        ws = r.swap_ct(images)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r.swap_phase(ws, cfg["sigma"], cfg["eps"], vol)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        phase_ms = sum(ts) / len(ts)
        del ws
    # end to end: pinned host images in, volume out
    host_img = images.cpu().pin_memory()
    host_vol = torch.empty(vol.shape, dtype=torch.float32).pin_memory()
    dimg = torch.empty_like(images)
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dimg.copy_(host_img, non_blocking=True)
        if args.form == "swap":
            r.swap_phase(r.swap_ct(dimg), cfg["sigma"], cfg["eps"], vol)
        else:
            r.grid_run(dimg, nsr, vol)
        host_vol.copy_(vol, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e.append(e0.elapsed_time(e1))
    # launches per step: the layered CT step twice (cos and sin volumes) or the per-view
    # spectra and splats, plus the 3D passes
    P3 = [1 << int(np.ceil(np.log2(2 * n))) for n in cfg["grid"]]
    fft3 = sum(1 for q in P3 if q > 1)
    sub = max(r.stage_block, 1)
    nsub = sum(-(-min(r.dir_block, D - b * r.dir_block) // sub) for b in range(r.n_blocks))
    dens = 2 if cfg["ramp"] == "density" else 0  # the sampling density, once per call
    if args.form == "swap":
        launches = dens + 2 * (3 * nsub + r.n_blocks) + 1 + fft3 + (1 + fft3 + 1)
        # the inversion: the phase kernel reads Z and writes the work grid, each 3D pass reads
        # and writes it, the crop reads the kept voxels and writes the volume
        cells = float(np.prod(P3))
        algo = cells * 8 * 2 + fft3 * cells * 8 * 2 + V * 12
        peaks, peak_src = load_peaks()
        achieved = algo / (phase_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "kernel": "swap_phase (k_swap_phase, k_fft3_lines x3, "
                    "k_crop_real)", "traffic": None, "algorithmic_bytes_per_launch": algo, "launches": 1,
                    "ms_per_launch": phase_ms, "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)"}
    else:
        gsub = -(-D // max(1, min(D, (1 << 30) // (cfg["nv"] * (r.padded // 2 + 1) * 8 + (r.padded // 2 + 1)
                                                   * r.padded * 8))))
        launches = dens + 3 * gsub + 2 + fft3 + 1
        roofline = None
    line = {"metric": METRIC, "value": U / (ms_step / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload] + (f" [first {D} directions only]" if args.dirs else ""),
                       "form": {"swap": "Eq. 12 swapped order (one defocus for every view: the workload's mean)",
                                "grid": "Fourier-gridding UTR with the NSR noise filter"}[args.form],
                       "padded_grid": P3, "updates_per_step": U,
                       "l2": "flushed between timed steps (256 MiB write outside the timed span)",
                       "parallelism": "replicas x1"},
            "e2e": {"value": U / (sum(e2e) / len(e2e) / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": images.numel() * 4, "d2h_bytes_per_step": vol.numel() * 4},
            "gpu_launches": launches * args.steps, "roofline": roofline, "clocks": clocks,
            "accuracy": {"note": "parity against the FP64 oracle in tests/test_fourier_gpu.py (1e-5 rel-L2; 1e-3 "
                                 "with the noise filter)"}}
    if args.form == "swap":
        line["swap_ct_ms"] = ms_step - sum(tail_ms) / args.steps
        line["swap_phase_ms"] = phase_ms
    else:
        line["roofline_note"] = ("one call; its per-view splat (8 float atomics per accumulator and sample) and "
                                 "3D passes are broken down by the launch list in profiles/")
    print(json.dumps(line))
    r.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOAD_TEXT), default="slab",
                    help="slab (the default) is the largest single-GPU workload")
    ap.add_argument("--stack", choices=["f32", "bf16"], default=None,
                    help="layer-stack precision (default: the workload's, f32 for mid/small, bf16 otherwise)")
    ap.add_argument("--filter", choices=["tikhonov", "mlp", "pair"], default="tikhonov",
                    help="mlp: the trained learned regulariser (data/regulariser.npz), reported beside the "
                         "analytic one; pair: the opposite-pair form of Eq. 10/11 on a single-axis workload, its "
                         "views spread over 360 degrees")
    ap.add_argument("--dir-block", type=int, default=0)
    ap.add_argument("--stage-block", type=int, default=0, help="directions per FFT/filter sub-block, 0 = auto")
    ap.add_argument("--bp-kernel", choices=["auto", "direct", "staged", "tma"], default="auto",
                    help="backprojection variant (tma: the TMA-staged kernel for any geometry)")
    ap.add_argument("--form", choices=["layered", "swap", "grid"], default="layered",
                    help="swap: Eq. 12's CT step and 3D CTF inversion; grid: the Fourier-gridding UTR")
    ap.add_argument("--layer-interp", choices=["nearest", "linear"], default="nearest",
                    help="a voxel's layer: the one containing its depth, or the blend of the two bracketing ones")
    ap.add_argument("--dirs", type=int, default=None, help="first N directions only (small profiling cases)")
    ap.add_argument("--cpu-dirs", type=int, default=None, help="oracle directions of the CPU baseline "
                    "(default: one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    if args.stack is None:
        args.stack = DEFAULT_STACK[args.workload]
    if args.layer_interp == "linear" and args.filter == "mlp":
        ap.error("--layer-interp linear is measured with the analytic filter")
    if args.filter == "pair" and (args.workload not in ("mid", "small") or args.form != "layered"
                                  or args.impl != "ours"):
        ap.error("--filter pair runs the layered form on a single-axis workload (mid or small)")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.form != "layered":
        return run_fourier(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
