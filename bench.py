#!/usr/bin/env python
"""Throughput of the photon generation + propagation path on GB300.

Metric: traced photon bunches (rays) per second, batched FP32 path, against
the plain FP64 GPU path, at oracle tolerance.  One step = one call of the
whole path (yield, generation, refracted propagation with absorption, hit
test, sort, per-telescope counts and sums) over the 2e7-step 1 TeV vertical
gamma shower (5-layer atmosphere, spherical Earth, absorption, bunch size 5,
10 x 10 telescopes at 100 m).  Inputs are synthetic and seeded; the
segment array (1.28 GB) is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank traces its own shower (weak scaling) with
no data-path collective; the timed region is bracketed by barriers and the
maximum over ranks is reported.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "traced photons/s, 1 GB300: batched FP32 vs plain FP64 at oracle tolerance"
UNIT = "rays/s"

# Algorithmic operations per unit of work on the FMA/ALU pipes, counted
# from the kernel source (trace_kernels.cu, ray.cuh): per quadrature node of
# the refracted spherical integrand, per altitude cell (node placement and
# accumulation), per ray traced in full outside the nodes (Philox rounds,
# cone, emission point, vacuum line and landing point in FP32 pairs, arrival
# time, absorption, hit search), and per ray that the first pass shows to
# land clear of every telescope (Philox rounds, cone, emission point and
# altitude in binary32, the displacement bound and the clearance lookup:
# skip_ray and clear_miss).  MUFU ops (ex2, rsqrt, rcp, sin, cos) counted apart.
OPS_NODE = 39
MUFU_NODE = 5
NODES_PER_CELL = 3
OPS_CELL = 8
OPS_RAY = 680
MUFU_RAY = 12
OPS_SKIPPED_RAY = 255
MUFU_SKIPPED_RAY = 7
FP32_LANES_PER_SM = 128
MUFU_LANES_PER_SM = 16


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        # nvidia-smi's start-up holds the driver for a few hundred ms: let it
        # reach its first sample before the timed region opens
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)
        time.sleep(0.2)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
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
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(n_steps):
    """DRAM bytes of one fused-kernel launch from the recorded ncu capture,
    scaled by steps, or None when the kernel sources changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_trace_fused_traffic.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    rec = {}
    for f in lines:
        if f[0] == "sha256":
            src = os.path.join(ROOT, "paper_2309_15861_gb300", "csrc", f[1])
            try:
                if hashlib.sha256(open(src, "rb").read()).hexdigest() != f[2]:
                    return None
            except OSError:
                return None
        else:
            rec[f[0]] = float(f[1])
    return rec["bytes_per_step"] * n_steps if "bytes_per_step" in rec else None


def _oracle_rate(w, budget_s, block, seed, threads):
    import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    n = len(w.segments)
    starts = rng.permutation(n // block)
    rays = 0
    t0 = time.perf_counter()
    blocks = 0
    for b in starts:
        lo = int(b) * block
        _, _, _, st = O.trace(w.segments[lo:lo + block], w.atmosphere, w.telescopes, w.params,
                              n_showers=w.n_showers, seg_base=lo, threads=threads)
        rays += st["rays"]
        blocks += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return rays, blocks, time.perf_counter() - t0


def cpu_baseline(w, budget_s=12.0, block=256, seed=0, single_s=0.0):
    """The FP64 oracle on contiguous blocks of the same workload (host cores;
    optionally also on one thread)."""
    n = len(w.segments)
    rays, blocks, dt = _oracle_rate(w, budget_s, block, seed, 0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": rays / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{blocks} random blocks of {block} consecutive steps ({blocks * block} of {n} "
                     f"steps, {rays} rays) of the same shower, {dt:.1f} s, FP64 oracle with OpenMP"}
    if single_s > 0:
        r1, b1, d1 = _oracle_rate(w, single_s, block, seed + 1, 1)
        out["single_thread"] = {"value": r1 / d1, "unit": UNIT, "sample": f"{b1} blocks, {r1} rays, {d1:.1f} s"}
    return out


def reference_arm(args, rank):
    """The oracle timed on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return 0
    w = make_workload(args.workload, args.n_segs, 0, args.scale)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(w, budget_s=per_step, seed=i)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "segments": len(w.segments), "telescopes": len(w.telescopes),
                       "bunch": w.params.bunch},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"],
                             "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = ("shower_1tev", "inclined", "batch", "adjoint")


def make_workload(name, n_segs, rank, scale):
    from paper_2309_15861_gb300 import inputs as I
    wk = I.default_workers()
    if name == "inclined":
        return I.workload_inclined(n=n_segs or 100_000_000, seed=1 + rank, workers=wk)
    if name == "batch":
        return I.batch_showers(256, seed=1 + rank, scale=scale, workers=wk)
    if name == "adjoint":
        return I.workload_shower_1tev(n=n_segs or 1_000_000, seed=1 + rank, workers=wk)
    return I.workload_shower_1tev(n=n_segs or 20_000_000, seed=1 + rank, workers=wk)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shower_1tev", choices=WORKLOADS,
                    help="shower_1tev: 2e7-step vertical 1 TeV shower (the default); inclined: 1e8 steps at "
                         "60 deg over 441 telescopes; batch: 256 showers with fluorescence (7.4e8 steps, "
                         "autotuned); adjoint: 1e6 steps, forward + adjoint per step")
    ap.add_argument("--n-segs", type=int, default=0)
    ap.add_argument("--scale", type=float, default=1.0, help="segment-count scale of the batch workload")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--propagator", default="exact", choices=["exact", "straight"],
                    help="exact: the refracted ray's deviation integrated (default); straight: the vacuum "
                         "line with first-order refraction corrections (Sec. 2's method, approximate)")
    ap.add_argument("--disp-B", type=float, default=0.0,
                    help="dispersion: n - 1 = delta(h) (1 + B/lambda^2)/(1 + B/400^2), B in nm^2 (0 = none)")
    ap.add_argument("--fl-beaming", action="store_true",
                    help="beam the fluorescence toward the array (Sec. 1.1.1); the batch workload's default is "
                         "isotropic emission")
    ap.add_argument("--fl-roulette", action="store_true",
                    help="fluorescence steps with fewer photons than a bunch emit one full bunch with "
                         "probability N/B (unbiased; with --fl-beaming this is what removes rays)")
    ap.add_argument("--cut-study", action="store_true",
                    help="also time the Cherenkov angular cut (array centre and per telescope, 6 deg) and "
                         "report its speedup and photon loss against the uncut step")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--cell-width", type=float, default=0.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return reference_arm(args, rank)

    import torch
    import paper_2309_15861_gb300 as G
    from paper_2309_15861_gb300 import build as B, inputs as I
    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    t_gen = time.perf_counter()
    w = make_workload(args.workload, args.n_segs, rank, args.scale)
    t_gen = time.perf_counter() - t_gen
    if args.disp_B > 0:
        w.atmosphere.disp_B = args.disp_B
        w.atmosphere.disp_lref = 400.0
    if args.fl_beaming:
        import dataclasses
        c, r = I.beam_cone(w.telescopes)
        w.params = dataclasses.replace(w.params, fl_beaming=1, beam_centre=c, beam_radius=r)
    if args.fl_roulette:
        import dataclasses
        w.params = dataclasses.replace(w.params, fl_roulette=1)
    ns = w.n_showers
    ctx = G.Context(local)
    extra = dict(use_graph=1, precision=args.precision, block=args.block, ctas_per_sm=args.ctas_per_sm,
                 cell_width=args.cell_width, propagator=1 if args.propagator == "straight" else 0)
    ctx.setup(w, **extra)
    dev = f"cuda:{local}"
    segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).to(dev)
    n = len(w.segments)
    cap = max(1 << 20, n // 4)
    hits = torch.empty(cap * 48, dtype=torch.uint8, device=dev)
    ng = ns * len(w.telescopes)
    counts = torch.zeros(ng, dtype=torch.int64, device=dev)
    sums = torch.zeros(ng, dtype=torch.float64, device=dev)

    tune = None
    if args.workload == "batch" and not args.no_tune:
        # a sample of the batch (every shower's share) picks block, CTAs, cell width and bunch <= 5
        n_sample = min(n, 4_000_000)
        tune = ctx.autotune(segs, n_sample, ns, hits, cap, bunch_max=w.params.bunch, reps=3)
        extra.update(block=tune["block"], ctas_per_sm=tune["ctas_per_sm"], cell_width=tune["cell_width"])
        w.params.bunch = tune["bunch"]
        ctx.set_params(w.params, **extra)

    code, nh, st = ctx.trace(segs, n, ns, hits, cap, counts, sums, raise_on_error=False)
    if code == G.ERR_HIT_CAPACITY:
        cap = int(nh * 1.25) + 1024
        hits = torch.empty(cap * 48, dtype=torch.uint8, device=dev)
        code, nh, st = ctx.trace(segs, n, ns, hits, cap, counts, sums)

    adj = None
    if args.workload == "adjoint":
        gen = torch.Generator(device=dev).manual_seed(7)
        gx = torch.randn(nh, generator=gen, device=dev)
        gy = torch.randn(nh, generator=gen, device=dev)
        gt = torch.randn(nh, generator=gen, device=dev)
        gY = torch.randn(ng, generator=gen, device=dev, dtype=torch.float64)
        adj = dict(gx=gx, gy=gy, gt=gt, gY=gY)

    def step():
        out = ctx.trace(segs, n, ns, hits, cap, counts, sums)
        if adj is not None:
            ctx.trace_adjoint(segs, n, ns, hits, out[1], **adj)
        return out

    for _ in range(args.warmup):
        step()
    # ---- timed region (device-resident inputs)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms, sms = [], []
    e0.record(s)
    for _ in range(args.steps):
        code, nh, st = step()
        a, b = ctx.last_timing()
        kms.append(a)
        sms.append(b)
    e1.record(s)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        r = torch.tensor([float(st["rays"])], device=dev)
        dist.all_reduce(r)
        rays_all = float(r.item())
    else:
        rays_all = float(st["rays"])
    ms_step = ms / args.steps
    value = rays_all * args.steps / (ms / 1e3)
    key_bits = (ng - 1).bit_length() + (n - 1).bit_length() + 16
    passes = (key_bits + 7) // 8
    # the fused kernel, plus the deferred-ray kernel on the default path
    deferred = args.precision == 0 and not (args.disp_B > 0 and (args.propagator == "straight" or args.fl_beaming
                                                                  or args.fl_roulette))
    # a call with the default queue runs in pieces of half the queue's entries
    piece = min(max(2 * n, 1 << 20), 1 << 28) // 2
    pieces = -(-n // piece) if deferred else 1
    launches_per_step = (2 if deferred else 1) * pieces + 5 * passes + 3 + (3 if adj is not None else 0)

    # ---- roofline of the dominant kernel (generation + propagation + hits)
    k_ms = statistics.mean(kms)
    # rays decided without the quadrature and landing: clear of every
    # telescope, escaping, or emitted below the observation level
    short = st["skipped"] + st["escaped"] + st["under"]
    full = st["rays"] - short
    ops = full * OPS_RAY + short * OPS_SKIPPED_RAY + st["cells"] * (OPS_CELL + NODES_PER_CELL * OPS_NODE)
    mufu = full * MUFU_RAY + short * MUFU_SKIPPED_RAY + st["cells"] * NODES_PER_CELL * MUFU_NODE
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_ops = n_sm * FP32_LANES_PER_SM * f_max
    achieved = ops / (k_ms / 1e3)
    traffic = recorded_traffic(n) if args.workload == "shower_1tev" else None
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s (FP32 pipe)",
            "frac": achieved / peak_ops, "traffic": traffic,
            "traffic_note": "DRAM bytes per launch: ncu capture of 2e6 steps scaled by steps "
                            "(profiles/k_trace_fused_traffic.txt); null if the kernel changed since",
            "kernel": "k_trace_fused + k_trace_deferred" if deferred else "k_trace_fused", "kernel_ms": k_ms, "sort_ms": statistics.mean(sms),
            "mufu_frac": (mufu / (k_ms / 1e3)) / (n_sm * MUFU_LANES_PER_SM * f_max),
            "ops_per_ray": ops / max(1, st["rays"]), "peak_basis": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                                                                 f"{f_max / 1e6:.0f} MHz (max SM clock)"}

    # ---- angular segment cut: the same step with the cut on
    cut = None
    if args.cut_study:
        import dataclasses
        base_sum, base_hits = float(sums.sum().item()), nh
        cut = []
        for mode in (1, 2):
            p2 = dataclasses.replace(w.params, cut_mode=mode, cut_deg=6.0, cut_centre=I.array_centre(w.telescopes))
            ctx.set_params(p2, **extra)
            for _ in range(3):
                ctx.trace(segs, n, ns, hits, cap, counts, sums)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            kc = max(5, args.steps // 4)
            c0.record(s)
            for _ in range(kc):
                code, nh_c, st_c = ctx.trace(segs, n, ns, hits, cap, counts, sums)
            c1.record(s)
            torch.cuda.synchronize()
            cms = c0.elapsed_time(c1) / kc
            cut.append({"mode": ["", "array centre", "each telescope"][mode], "deg": 6.0,
                        "segments_cut": int(st_c["cut"]), "rays": int(st_c["rays"]), "ms_per_step": cms,
                        "speedup": ms_step / cms, "hits_kept": nh_c / max(1, base_hits),
                        "photon_loss": 1.0 - float(sums.sum().item()) / base_sum if base_sum else None})
        ctx.set_params(w.params, **extra)

    # ---- plain FP64 GPU path on the same workload (at most its first 2e7 steps)
    fp64 = None
    if not args.no_fp64:
        n64 = min(n, 20_000_000)
        ctx.trace(segs, n64, ns, hits, cap, counts, sums, fp64=True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s)
        code, nh64, st64 = ctx.trace(segs, n64, ns, hits, cap, counts, sums, fp64=True)
        f1.record(s)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        v64 = st64["rays"] / (fms / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": fms, "segments": n64,
                "speedup_of_fp32": value / v64 if v64 else None}

    # ---- end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e and adj is None:
        pinned = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).pin_memory()
        hbuf = torch.empty(cap * 48, dtype=torch.uint8).pin_memory()
        cbuf = torch.zeros(ng, dtype=torch.int64).pin_memory()
        sbuf = torch.zeros(ng, dtype=torch.float64).pin_memory()
        seg_np = pinned.numpy().view(I.SEG_DTYPE)
        hits_np = hbuf.numpy().view(G.HIT_DTYPE)
        ctx.set_params(w.params, **{**extra, "use_graph": 0})
        ctx.trace_host(seg_np, ns, cap, hits_out=hits_np, counts_out=cbuf.numpy(), sums_out=sbuf.numpy())
        k2 = max(3, args.steps // 4)
        barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            code, hh, cc, ss, st2 = ctx.trace_host(seg_np, ns, cap, hits_out=hits_np, counts_out=cbuf.numpy(),
                                                   sums_out=sbuf.numpy())
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        e2e = {"value": st2["rays"] * k2 / wall, "unit": UNIT,
               "h2d_bytes_per_step": int(n * 64),
               "d2h_bytes_per_step": int(len(hh) * 48 + cbuf.numel() * 8 + sbuf.numel() * 8),
               "ms_per_step": wall * 1e3 / k2,
               "path": "clight_trace_host on pinned host buffers: the steps copied to the device every step "
                       "(2^22-step chunks on a copy stream, each launch waiting for its own chunk); hits, "
                       "counts and sums copied back every step"}
        ctx.set_params(w.params, **extra)
        del pinned, hbuf

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, single_s=4.0)

    if rank == 0:
        atm = "5-layer, spherical, absorbing"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "segments": n, "showers": ns, "rays_per_step": st["rays"],
                       "hits_per_step": nh, "telescopes": len(w.telescopes), "bunch": w.params.bunch,
                       "atmosphere": atm, "fluorescence": w.params.fluor_yield > 0,
                       "precision": ["float-pair", "fp64-guard"][args.precision], "graph": True,
                       "l2": f"inputs ({n * 64 / 1e9:.2f} GB) larger than L2; no flush",
                       "parallelism": f"replicas x{world}", "generation_s": round(t_gen, 1),
                       "fl_beaming": bool(args.fl_beaming), "fl_roulette": bool(args.fl_roulette),
                       "propagator": args.propagator,
                       "dispersion_B_nm2": args.disp_B,
                       "step": "trace + adjoint" if adj is not None else "trace"},
            "roofline": roof, "fp64_plain": fp64, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": ck, "gpu_launches": launches_per_step * args.steps,
            "stats": {k: int(v) for k, v in st.items()},
        }
        if tune is not None:
            line["autotune"] = tune
        if cut is not None:
            line["angular_cut"] = cut
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
