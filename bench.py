#!/usr/bin/env python
"""Benchmark of batched hard-binned Shannon / Tsallis MI on one GB300 (or N replicas).

Workload (one step): a 256 x 256 x 256 uint16 12-bit head-like phantom pair,
256 bins, 4096 random 9-parameter transforms (translation U(+-15 mm),
rotation U(+-20 deg), scale U(0.85, 1.15)) x q in {0.5, 1, 1.5, 2}, evaluated
by one persistent, graph-replayed launch.  Metric: voxels x transforms per
second.  Each rank evaluates its own 4096 transforms (weak scaling, no
collective on the data path).

Also reported: the same metric end to end through the C ABI with host
buffers (e2e), the one-transform-per-launch plain form, the Parzen MI+gradient
throughput (192 x 192 x 128 float32, 64 bins, q in {1, 0.7, 1.3}), the
roofline of the main kernel and the CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MI evals/sec (voxels·transforms/s) at 256³, batched vs plain; MI+grad/s; % of roofline"
SHAPE = (256, 256, 256)
BINS = 256
DEPTH = 12
N_T = 4096
QS = [0.5, 1.0, 1.5, 2.0]
# algorithmic integer operations per voxel x transform of the hard path, one per coordinate multiply-add
# (3), stage lerp (7) and binning (2), plus the weight extraction, gather address and increment (8): 20,
# counted over the voxels inside each transform's overlap (those outside cost no per-voxel work).  This
# is the roofline's numerator.  The kernel's own tally (each lerp 4 operations: two products, the
# rounding add and the shift; 9 address and 6 index/weight operations: 50) is reported beside it.
ALG_OPS_PER_VOXT = 20
DESIGN_OPS_PER_VOXT = 50
# Counters of one ncu capture of k_batched on this workload (see profiles/), reported only while the
# kernel source and the selected configuration are the ones measured: DRAM bytes of one full launch
# (4096 transforms), and from a one-wave capture the issue and L1TEX utilisation and the
# shared-memory wavefronts per shared atomic instruction.
K_BATCHED_NCU = {"source_sha16": "a052ba2f01e56eb8", "config": [10, 2, 4],
                 "dram_bytes_per_launch": 181408323840 + 61779200, "issue_active": 0.815,
                 "l1tex_throughput": 0.695, "smem_wavefronts_per_atomic": 333607686 / 71766929,
                 "smem_atomic_wavefronts_per_sm_cycle": 333607686 / 152 / 11992171.03,
                 "profile": "profiles/k_batched_rows_quad_256cubed_256bins.md"}
# algorithmic FP32 operations per voxel x transform of the Parzen MI + gradient at 3 q values:
# forward 31 (trilinear 14, bin coordinate 1, B-spline weights 12, 4 increments),
# adjoint 89 (trilinear value and gradient 23, bin coordinate 1, B-spline derivatives 8, 3 q x 19)
PARZEN_OPS_PER_VOXT = 120
# Counters of the Parzen forward (k_parzen_hist) from one ncu capture of the 50-pose call (see profiles/),
# reported while the kernel source is the one measured: shared-atomic instructions and wavefronts, SM
# cycles elapsed per launch, and the DRAM bytes read and written by the forward and the adjoint
K_PARZEN_NCU = {"source_sha16": "c75922c23d63e0fa", "atom_inst": 52167744, "atom_wavefronts": 242402137,
                "sm_cycles_elapsed": 2143008.79, "time_ms": 1.0395,
                "dram_bytes_per_call": 416319232 + 4436224 + 26225664,
                "profile": "profiles/parzen_fwd_adj_192x192x128_64bins.md"}
PARZEN_SHAPE = (128, 192, 192)
PARZEN_SPACING = (1.0, 1.0, 1.2)
PARZEN_BINS = 64
PARZEN_QS = [1.0, 0.7, 1.3]
PARZEN_N = 50


def workload_config():
    return {"workload": "batched hard-binned MI, 256x256x256 uint16 12-bit head-like pair, 256 bins, "
                        "4096 transforms x 4 q per step, one persistent graph-replayed launch",
            "volume": list(SHAPE[::-1]), "bits": DEPTH, "bins": BINS, "transforms_per_step": N_T, "q": QS,
            "transform_dist": "t U(+-15 mm), r U(+-20 deg), s U(0.85, 1.15)",
            "l2": "flushed (256 MiB write) between timed steps"}


def kernel_source_sha16(name="mi_hard.cu"):
    import hashlib

    p = os.path.join(ROOT, "paper_1909_10690_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampler over the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        load = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": float(np.median([r[0] for r in load])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


def rank_transforms(rank):
    """The transforms one rank evaluates per step: a seed of its own, so ranks share no
    work and add up (weak scaling; no collective on the data path)."""
    from paper_1909_10690_gb300 import phantoms

    return phantoms.random_transforms(N_T, seed=31 + rank)


def max_over_ranks(x, world):
    """Largest value of a host scalar over all ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as tdist

    t = torch.tensor([float(x)], dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, units_per_rank_step, seconds):
    """Units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_rank_step / seconds


def oracle_rate(f, m, prm, cores):
    """Oracle vox.T/s on the given transforms (all host cores, parallel across transforms)."""
    import oracle

    t0 = time.perf_counter()
    oracle.mi_eval(f, m, BINS, prm, QS, fixed_depth=DEPTH, moving_depth=DEPTH, nthreads=cores)
    dt = time.perf_counter() - t0
    return len(prm) * f.size / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1909_10690_gb300 import phantoms

    cores = os.cpu_count() or 1
    f, m = phantoms.head_pair(shape=SHAPE, spacing=(1, 1, 1), seed=30)
    prm = rank_transforms(0)
    per_step = cores  # one transform per core per step: a bounded sample of the step's 4096
    for w in range(args.warmup):
        oracle_rate(f, m, prm[w * per_step:(w + 1) * per_step], cores)
    total_t, total_units = 0.0, 0
    for s in range(args.steps):
        sel = prm[(s * per_step) % N_T:(s * per_step) % N_T + per_step]
        _, dt = oracle_rate(f, m, sel, cores)
        total_t += dt
        total_units += len(sel) * f.size
    value = total_units / total_t
    line = {"metric": METRIC, "value": value, "unit": "voxel*transforms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "impl": "reference", "config": workload_config(), "ranks": world,
            "cpu_baseline": {"value": value, "unit": "voxel*transforms/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of the step's {N_T} transforms per step (256^3, 256 bins, 4 q)"},
            "e2e": {"value": value, "unit": "voxel*transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import phantoms

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()

    f, m = phantoms.head_pair(shape=SHAPE, spacing=(1, 1, 1), seed=30)
    prm = rank_transforms(rank)
    stream = torch.cuda.Stream(device=dev)
    ctx = mi.Context(f, m, bins=BINS, fixed_depth=DEPTH, moving_depth=DEPTH, path="batched", device=local_rank)
    ctx.set_stream(stream)
    T_dev = torch.from_numpy(prm).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    nvox = int(np.prod(SHAPE))
    for _ in range(args.warmup):
        ctx.eval(T_dev, QS)
    variant = ctx.selected_variant(N_T)
    # the voxels the kernel processes: each transform's overlap (rows are clipped to it exactly, so a fixed
    # voxel outside costs no per-voxel work); the metric's value counts every fixed voxel
    overlap = float(ctx.eval(T_dev, QS, with_entropies=True)[2].sum().item())
    # --- device-resident timed region -------------------------------------------
    clocks = Clocks(local_rank)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kern_ms, launches = [], 0
    barrier()
    clocks.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev0[k].record(stream)
        out = ctx.eval(T_dev, QS)
        ev1[k].record(stream)
        km, nl = ctx.last_kernel_ms()
        kern_ms.append(km)
        launches += nl
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world)
    assert torch.isfinite(out).all()
    value = whole_job_rate(world, args.steps, N_T * nvox, total_s)
    # --- roofline of the main kernel ----------------------------------------------
    pk, src = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    sms = props.multi_processor_count
    alu_peak = sms * 128 * sm_mhz * 1e6 / 1e12  # int32 lane-ops/s, Tops/s
    kms = float(np.mean(kern_ms))
    units_per_s = overlap / (kms / 1e3)  # overlap voxel x transforms per second
    achieved = ALG_OPS_PER_VOXT * units_per_s / 1e12
    design = DESIGN_OPS_PER_VOXT * units_per_s / 1e12
    cfg = ctx.selected_config(N_T)
    ncu = K_BATCHED_NCU
    ncu_ok = ncu["source_sha16"] == kernel_source_sha16() and ncu["config"] == [cfg["variant"], cfg["tile_rows"],
                                                                                  cfg["tile_slabs"]]
    traffic = ncu["dram_bytes_per_launch"] if ncu_ok else None
    # one shared atomic per voxel x transform; the peak is one conflict-free 32-lane shared-memory
    # wavefront per clock per SM
    atom_peak = sms * 32 * sm_mhz * 1e6
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s", "frac": achieved / alu_peak,
                "traffic": traffic, "kernel": "k_batched", "kernel_ms": kms,
                "ops_per_voxel_transform": ALG_OPS_PER_VOXT,
                "units_per_launch": overlap, "overlap_fraction": overlap / (N_T * nvox),
                "units_note": "overlap voxel x transforms: the voxels the kernel processes",
                "peak_source": f"{sms} SMs x 128 int32 lanes x {sm_mhz:.0f} MHz ({src} clock)",
                "algorithmic_bytes": int(nvox * 1 + nvox * 2),
                "algorithmic_bytes_note": "both volumes once per launch: uint8 fixed bins and the uint16 moving volume",
                "design_count": {"ops_per_voxel_transform": DESIGN_OPS_PER_VOXT, "achieved": design,
                                 "frac": design / alu_peak},
                "shared_atomics": {"achieved_per_s": units_per_s, "peak_per_s": atom_peak,
                                   "frac": units_per_s / atom_peak,
                                   "peak_source": f"{sms} SMs x 32 lanes (one wavefront) x {sm_mhz:.0f} MHz"}}
    if ncu_ok:
        roofline["hbm"] = {"achieved_gbs": traffic / (kms / 1e3) / 1e9, "peak_gbs": float(pk["hbm_gbs"]),
                           "frac": traffic / (kms / 1e3) / 1e9 / float(pk["hbm_gbs"]), "peak_source": src}
        roofline["ncu"] = {k: ncu[k] for k in ("issue_active", "l1tex_throughput", "smem_wavefronts_per_atomic",
                                               "smem_atomic_wavefronts_per_sm_cycle", "profile")}
    # --- end to end through the C ABI with host buffers ----------------------------
    prm_pinned = torch.from_numpy(prm).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = ctx.eval(prm_pinned, QS)  # host in, host out
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    assert np.isfinite(res).all()
    e2e = {"value": whole_job_rate(world, args.steps, N_T * nvox, e2e_s), "unit": "voxel*transforms/s",
           "h2d_bytes_per_step": N_T * 48 + N_T * 8, "d2h_bytes_per_step": N_T * len(QS) * 8 + 8}
    extra = {}
    if rank == 0 and not args.skip_extras:
        # --- plain form: one transform per launch, host sync each time --------------
        pctx = mi.Context(f, m, bins=BINS, fixed_depth=DEPTH, moving_depth=DEPTH, path="plain", device=local_rank)
        pctx.set_stream(stream)
        n_plain = 64
        for i in range(3):
            pctx.eval(T_dev[i:i + 1], QS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(n_plain):
            pctx.eval(T_dev[i:i + 1], QS)
        plain_s = time.perf_counter() - t0
        plain_rate = n_plain * nvox / plain_s
        extra["plain"] = {"value": plain_rate, "unit": "voxel*transforms/s", "transforms": n_plain,
                          "form": "one transform per call: memset + histogram kernel + entropy kernel + D2H sync",
                          "batched_over_plain": value / world / plain_rate}
        del pctx
        # --- differentiable form: Parzen MI + gradient --------------------------------
        fp, mp = phantoms.head_pair(shape=PARZEN_SHAPE, spacing=PARZEN_SPACING, seed=50, dtype=np.float32)
        zctx = mi.Context(fp, mp, bins=PARZEN_BINS, kernel="parzen", fixed_spacing=PARZEN_SPACING,
                          moving_spacing=PARZEN_SPACING, device=local_rank)
        zctx.set_stream(stream)
        pp = torch.from_numpy(phantoms.random_transforms(PARZEN_N, seed=51, t_mm=10, r_deg=15,
                                                         s_range=(0.9, 1.1))).to(dev)
        for _ in range(3):
            zctx.grad(pp, PARZEN_QS)
        zk = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            zctx.grad(pp, PARZEN_QS)
            zk.append(zctx.last_kernel_ms()[0])
        z_s = time.perf_counter() - t0
        pv = int(np.prod(PARZEN_SHAPE))
        zms = float(np.mean(zk))
        z_over = float(zctx.eval(pp, PARZEN_QS, with_entropies=True)[2].sum().item())  # voxels processed
        z_ach = PARZEN_OPS_PER_VOXT * z_over / (zms / 1e3) / 1e12
        extra["mi_grad"] = {"value": args.steps * PARZEN_N / z_s, "unit": "(MI+grad over 9 params, 3 q)/s",
                            "voxel_transforms_per_s": args.steps * PARZEN_N * pv / z_s,
                            "kernel_ms_per_call": zms, "poses_per_call": PARZEN_N,
                            "volume": list(PARZEN_SHAPE[::-1]), "bins": PARZEN_BINS, "q": PARZEN_QS,
                            "roofline": {"bound": "alu", "achieved": z_ach, "peak": alu_peak, "unit": "Tops/s",
                                         "frac": z_ach / alu_peak, "traffic": None,
                                         "kernel": "k_parzen_hist + k_parzen_cells + k_parzen_adj",
                                         "units_per_call": z_over, "overlap_fraction": z_over / (PARZEN_N * pv),
                                         "note": "FP32 lane-ops per overlap voxel x transform over the whole "
                                                 "MI+grad call"}}
        pn = K_PARZEN_NCU
        if pn["source_sha16"] == kernel_source_sha16("mi_parzen.cu"):
            extra["mi_grad"]["roofline"]["traffic"] = pn["dram_bytes_per_call"]
            extra["mi_grad"]["roofline"]["traffic_note"] = "DRAM bytes of k_parzen_hist + k_parzen_adj per call (ncu)"
            extra["mi_grad"]["roofline"]["algorithmic_bytes"] = int(pv * 1 + pv * 4)
            # the forward's binding unit: the shared-memory pipe, one wavefront per clock per SM
            extra["mi_grad"]["forward_shared_atomics"] = {
                "wavefronts_per_sm_cycle": pn["atom_wavefronts"] / sms / pn["sm_cycles_elapsed"],
                "lane_atomics_per_s": pn["atom_inst"] * 32 / (pn["time_ms"] / 1e3),
                "lane_atomics_peak_per_s": atom_peak, "wavefronts_per_instruction": pn["atom_wavefronts"] / pn["atom_inst"],
                "profile": pn["profile"]}
        del zctx
    line = {"metric": METRIC, "value": value, "unit": "voxel*transforms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": dict(workload_config(), hist_variant=variant, parallelism=f"replicas x{world}",
                           selected=ctx.selected_config(N_T)),
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    line.update(extra)
    if rank == 0 and not args.skip_cpu:
        cores = os.cpu_count() or 1
        # about 10 s of oracle work on this machine's cores: 28 transforms a core (~45 ms each at 256^3)
        sample = prm[:min(len(prm), 28 * cores)]
        rate, dt = oracle_rate(f, m, sample, cores)
        line["cpu_baseline"] = {"value": rate, "unit": "voxel*transforms/s", "cores": cores, "kind": "oracle",
                                "sample": f"{len(sample)} of the 4096 transforms (256^3, 256 bins, 4 q), {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_profile(args):
    """Only the batched 256^3 evaluation of ``args.profile`` transforms with a fixed histogram
    variant (no autotuning), for ncu captures of the main kernel on a small case."""
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import phantoms

    f, m = phantoms.head_pair(shape=SHAPE, spacing=(1, 1, 1), seed=30)
    prm = torch.from_numpy(phantoms.random_transforms(args.profile, seed=31)).cuda()
    ctx = mi.Context(f, m, bins=BINS, fixed_depth=DEPTH, moving_depth=DEPTH, path="batched",
                     hist_variant=args.variant, autotune=False, block_threads=args.threads,
                     tile_rows=args.tile_rows, tile_slabs=args.slabs)
    for _ in range(args.warmup):
        ctx.eval(prm, QS)
    ms = []
    for _ in range(args.steps):
        ctx.eval(prm, QS)
        ms.append(ctx.last_kernel_ms()[0])
    nvox = int(np.prod(SHAPE))
    print(json.dumps({"profile": "batched", "transforms": args.profile, "variant": args.variant, "threads": args.threads,
                      "tile_rows": args.tile_rows, "slabs": args.slabs, "kernel_ms": ms,
                      "voxel_transforms_per_s": args.profile * nvox / (np.mean(ms) / 1e3)}))


def run_profile_parzen(args):
    """Only the Parzen MI + gradient of ``args.profile_parzen`` poses on the 192x192x128 pair, for ncu."""
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import phantoms

    fp, mp = phantoms.head_pair(shape=PARZEN_SHAPE, spacing=PARZEN_SPACING, seed=50, dtype=np.float32)
    ctx = mi.Context(fp, mp, bins=PARZEN_BINS, kernel="parzen", fixed_spacing=PARZEN_SPACING,
                     moving_spacing=PARZEN_SPACING)
    pp = torch.from_numpy(phantoms.random_transforms(args.profile_parzen, seed=51, t_mm=10, r_deg=15,
                                                     s_range=(0.9, 1.1))).cuda()
    for _ in range(args.warmup):
        ctx.grad(pp, PARZEN_QS)
    ms = []
    for _ in range(args.steps):
        ctx.grad(pp, PARZEN_QS)
        ms.append(ctx.last_kernel_ms()[0])
    print(json.dumps({"profile": "parzen", "poses": args.profile_parzen, "kernel_ms": ms}))


def run_maps(args):
    """The Methodology's parameter-space maps of the 256x256x160 12-bit head-like pair (64 bins, Shannon and
    Tsallis q = 1.5) through the batched path, args.maps^3 points each: translations over +-25 mm, unit-ball
    rotations over +-0.3 per versor component (the Results' rotation maps; up to 2 asin(0.52) = 63 deg), and
    zero-centred scales over +-0.2; the pair has no motion, so the true pose is each grid's centre.  Then the
    ascent analysis of the Results on each Shannon map, and where the maximum lies (off the grid's lattice
    every rotation and scale interpolates, which smooths the moving volume's noise: the Discussion's
    interpolation effects).  One JSON line per family."""
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import maps, phantoms

    sp = (1.0, 1.0, 1.2)
    f, m = phantoms.head_pair(shape=(160, 256, 256), spacing=sp, seed=60, motion=(0, 0, 0, 0, 0, 0, 1, 1, 1))
    n = args.maps
    c = (n - 1) // 2
    for family, lo, hi, opts in (("translation", -25, 25, {}), ("rotation", -0.3, 0.3, {"rotation": "versor"}),
                                 ("scale", -0.2, 0.2, {"scale": "offset"})):
        ctx = mi.Context(f, m, bins=64, fixed_depth=12, moving_depth=12, fixed_spacing=sp, moving_spacing=sp,
                         path="batched", **opts)
        # warm-up on the same map: the autotuner keys on the call's size class (below 152, below 608 or
        # more transforms on 152 SMs) and the graph cache on its exact count, so a smaller warm-up grid
        # leaves the map's 32 768-transform chunks untuned and its last, shorter chunk without a graph
        maps.param_map(ctx, family, lo, hi, n, q=[1.0, 1.5])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mp = maps.param_map(ctx, family, lo, hi, n, q=[1.0, 1.5])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t1 = time.perf_counter()
        frac = maps.capture_fraction(mp[..., 0], (c, c, c))
        _, maxima = maps.ascent_sinks(mp[..., 0])
        da = time.perf_counter() - t1
        peak = np.unravel_index(np.argmax(mp[..., 0]), mp.shape[:3])
        print(json.dumps({"maps": family, "grid": [n, n, n], "range": [lo, hi], "transforms": n ** 3,
                          "voxels": int(f.size), "seconds": dt, "voxel_transforms_per_s": n ** 3 * f.size / dt,
                          "peak_at_centre": bool(peak == (c, c, c)),
                          "peak_offset_steps": [int(x) - c for x in peak],
                          "mi_peak_minus_centre": float(mp[..., 0].max() - mp[c, c, c, 0]),
                          "capture_fraction_shannon": frac, "local_maxima_shannon": int(len(maxima)),
                          "ascent_analysis_seconds": da}), flush=True)
        del ctx


def run_uneven(args):
    """The uneven batch: 48 pairs from 96^3 to 320x320x200 (half uint8, half uint16 12-bit; 32, 64 or 128
    bins each) with 256 transforms per pair, all 12 288 in one batched call (one persistent launch over
    every pair, q = 1, 0.5, 1.5, 2); then the Parzen MI and gradient of the 8 largest pairs, each at its own
    bin count, 64 poses each, in one multi-pair call (q = 1, 0.7, 1.3).  The pairs' volumes and textures
    (several GB) are larger than L2.  Device time by CUDA events around each call, after ``args.warmup``
    untimed calls; one JSON line per part."""
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import phantoms

    specs = phantoms.uneven_specs(48, seed=5)
    vols = [phantoms.head_pair(shape=s["shape"], spacing=(1, 1, 1), depth=s["depth"], seed=s["seed"], dtype=s["dtype"])
            for s in specs]
    nvox = np.array([int(np.prod(s["shape"])) for s in specs])
    n_per = 256
    prm = phantoms.random_transforms(n_per * len(specs), seed=61)
    pair_of = np.repeat(np.arange(len(specs), dtype=np.int32), n_per)
    perm = np.random.default_rng(62).permutation(len(prm))
    prm, pair_of = prm[perm], pair_of[perm]

    def timed(call):
        for _ in range(args.warmup):
            call()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            ev[0].record()
            call()
            ev[1].record()
            torch.cuda.synchronize()
            ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ms)), ms

    ctx = mi.Context(pairs=[dict(fixed=f, moving=m, bins=s["bins"], fixed_depth=s["depth"], moving_depth=s["depth"])
                            for s, (f, m) in zip(specs, vols)])
    ctx.set_stream(torch.cuda.current_stream())  # the stream the timing events are recorded on
    d_pof, d_prm = torch.from_numpy(pair_of).cuda(), torch.from_numpy(prm).cuda()
    qs = [1.0, 0.5, 1.5, 2.0]
    med, ms = timed(lambda: ctx.batch_eval(d_pof, d_prm, qs))
    work = float(nvox[pair_of].sum())
    print(json.dumps({"uneven": "hard", "pairs": len(specs), "transforms": len(prm), "q": qs,
                      "voxel_transforms": work, "ms": med, "ms_all": ms, "kernel_ms": ctx.last_kernel_ms()[0],
                      "voxel_transforms_per_s": work / (med * 1e-3), "selected": ctx.selected_config(len(prm))}),
          flush=True)
    del ctx
    big = np.argsort(nvox)[-8:]
    pctx = mi.Context(pairs=[dict(fixed=vols[p][0], moving=vols[p][1], bins=specs[p]["bins"],
                                  fixed_depth=specs[p]["depth"], moving_depth=specs[p]["depth"]) for p in big],
                      kernel="parzen")
    pctx.set_stream(torch.cuda.current_stream())
    psel = np.concatenate([np.nonzero(pair_of == p)[0][:64] for p in big])
    pof = torch.from_numpy(np.repeat(np.arange(len(big), dtype=np.int32), 64)).cuda()
    pprm = torch.from_numpy(prm[psel]).cuda()
    qz = [1.0, 0.7, 1.3]
    med, ms = timed(lambda: pctx.batch_grad(pof, pprm, qz, allow_empty=True))
    work = float(64 * nvox[big].sum())
    print(json.dumps({"uneven": "parzen", "pairs": [int(p) for p in big], "bins": [specs[p]["bins"] for p in big],
                      "poses": len(psel), "q": qz, "ms": med, "ms_all": ms, "kernel_ms": pctx.last_kernel_ms()[0],
                      "launches": pctx.last_kernel_ms()[1], "poses_per_s": len(psel) / (med * 1e-3),
                      "voxel_transforms_per_s": work / (med * 1e-3)}), flush=True)


def run_parzen_bins(args):
    """The Parzen MI + gradient per bin count: 64 poses (the uneven batch's transform distribution) on a
    256x256x160 uint16 12-bit head-like pair at 32, 64, 96 and 128 bins, q = 1, 0.7, 1.3; device time of
    the call's kernels, median of ``args.steps`` after ``args.warmup``.  One JSON line per bin count."""
    import torch

    import paper_1909_10690_gb300 as mi
    from paper_1909_10690_gb300 import phantoms

    f, m = phantoms.head_pair(shape=(160, 256, 256), spacing=(1, 1, 1), seed=7)
    prm = torch.from_numpy(phantoms.random_transforms(64, seed=61)).cuda()
    for B in (32, 64, 96, 128):
        ctx = mi.Context(f, m, bins=B, kernel="parzen", fixed_depth=12, moving_depth=12)
        for _ in range(args.warmup):
            ctx.grad(prm, PARZEN_QS, allow_empty=True)
        ms = []
        for _ in range(args.steps):
            ctx.grad(prm, PARZEN_QS, allow_empty=True)
            ms.append(ctx.last_kernel_ms()[0])
        med = float(np.median(ms))
        print(json.dumps({"parzen_bins": B, "poses": 64, "volume": [256, 256, 160], "q": PARZEN_QS,
                          "kernel_ms": med, "voxel_transforms_per_s": 64 * f.size / (med * 1e-3)}), flush=True)
        del ctx


def relaunch_ranks():
    """``--gpus N`` run by hand (no WORLD_SIZE in the environment): start the N ranks on this node with
    torch.distributed.run, one per GPU, each running this script with the same arguments."""
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ap = argparse.ArgumentParser(add_help=False)
    ap.add_argument("--gpus", type=int, default=1)
    n = ap.parse_known_args()[0].gpus
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-extras", action="store_true", help="skip the plain and Parzen lines")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile", type=int, default=0, help="profile mode: batched kernel only, on this many transforms")
    ap.add_argument("--variant", type=int, default=9, help="histogram variant in profile mode (MI_HV_*)")
    ap.add_argument("--threads", type=int, default=1024, help="CTA size in profile mode (512 or 1024)")
    ap.add_argument("--tile-rows", type=int, default=1, help="fixed rows per warp step in profile mode (1, 2, 4)")
    ap.add_argument("--slabs", type=int, default=4, help="slabs per sweep in profile mode (1..16)")
    ap.add_argument("--profile-parzen", type=int, default=0, help="profile mode: Parzen MI + gradient of this many poses")
    ap.add_argument("--maps", type=int, default=0,
                    help="time N^3 translation, rotation and scale maps of the head-like pair")
    ap.add_argument("--uneven", action="store_true",
                    help="time the 48-pair uneven batch (hard) and the Parzen MI + gradient of its 8 largest pairs")
    ap.add_argument("--parzen-bins", action="store_true",
                    help="time the Parzen MI + gradient at 32, 64, 96 and 128 bins")
    args = ap.parse_args()
    if args.parzen_bins:
        run_parzen_bins(args)
        return
    if args.maps:
        run_maps(args)
        return
    if args.uneven:
        run_uneven(args)
        return
    if args.profile:
        run_profile(args)
        return
    if args.profile_parzen:
        run_profile_parzen(args)
        return
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_ranks())
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("gloo")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
