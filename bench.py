#!/usr/bin/env python
"""Throughput of the photon generation + propagation path on GB300.

Metric: traced photon bunches (rays) per second, batched FP32 path, against
the plain FP64 GPU path, at oracle tolerance.  One step = one call of the
whole path (yield, generation, refracted propagation with absorption, hit
test, sort, per-telescope counts and sums) over the default workload: 256
showers (energies log-uniform 10 GeV-10 TeV, 2e4 steps per 10 GeV, 7.92e8
steps in all, zenith 0-45 deg) with fluorescence (5 photons/MeV), a 5-layer
spherical absorbing atmosphere and 10 x 10 telescopes at 100 m, in one
persistent work-stealing launch sequence replayed as a CUDA graph, with the
bunch size (<= 5), launch shape and work chunk picked by the autotuner.
Inputs are synthetic and seeded; the step array (50.7 GB) is far larger
than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload batch|shower_1tev|inclined|adjoint] [--peaks]

Under torchrun (N > 1) every rank traces its own batch (weak scaling) with
no data-path collective; the timed region is bracketed by barriers and the
maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import dataclasses
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

METRIC = "traced photons/s, 1 GB300: batched FP32 vs plain FP64 at oracle tolerance"
UNIT = "rays/s"

# Algorithmic work per unit, as the measurement plan of the path states it
# (FP32-pipe operations): generation + Philox of a ray; a ray decided from
# its vacuum line (the line plus one clearance test); a ray traced in full
# (vacuum line and hit search); one node of the refracted-ray quadrature
# (3 per altitude cell).
OPS8D_GEN = 80
OPS8D_SKIPPED = OPS8D_GEN + 20 + 15
OPS8D_TRACED = OPS8D_GEN + 135
OPS8D_NODE = 30
NODES_PER_CELL = 3
# Operations counted from the kernel source (a second, larger figure: it
# includes the step set-up, the bunch bookkeeping and the pair arithmetic):
# per ray decided in the first pass, per ray traced in full outside the
# quadrature, per altitude cell and per node.
SRC_OPS_SKIPPED = 255
SRC_OPS_RAY = 680
SRC_OPS_CELL = 8
# Adjoint: a candidate ray (or hit) recomputes a traced ray -- generation and
# hit search (OPS8D_TRACED) and ~5 quadrature nodes -- in forward-mode dual
# numbers carrying the value and one tangent per parameter.
ADJ_NODES = 5
ADJ_OPS_PER_UNIT = OPS8D_TRACED + ADJ_NODES * OPS8D_NODE
SRC_OPS_NODE = 39


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


def recorded_traffic(workload, n_units):
    """DRAM bytes of one call's tracing kernels from the recorded ncu
    capture (profiles/<kernel>_<workload>_traffic.txt), scaled by the units
    of the record, or None when no record exists or a kernel source changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", f"tracing_{workload}_traffic.txt")
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
    return rec["bytes_per_step"] * n_units if "bytes_per_step" in rec else None


def traffic_record(workload):
    """The traffic record as written, whatever the sources now hold:
    {"bytes_per_step", "current"} (current = every source hash still
    matches), or None without a record."""
    path = os.path.join(ROOT, "profiles", f"tracing_{workload}_traffic.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    rec, current = {}, True
    for f in lines:
        if f[0] == "sha256":
            try:
                src = os.path.join(ROOT, "paper_2309_15861_gb300", "csrc", f[1])
                current &= hashlib.sha256(open(src, "rb").read()).hexdigest() == f[2]
            except OSError:
                current = False
        else:
            rec[f[0]] = float(f[1])
    if "bytes_per_step" not in rec:
        return None
    return {"bytes_per_step": rec["bytes_per_step"], "current": current,
            "file": f"profiles/tracing_{workload}_traffic.txt"}


# ------------------------------------------------------------------ oracle legs
def _oracle_blocks(w, budget_s, block, seed, threads, keep_hits=False):
    """The FP64 oracle on contiguous blocks of `block` steps drawn at random
    from the whole workload, until `budget_s` has passed."""
    import oracle as O
    O.build()
    rng = np.random.default_rng(seed)
    n = len(w.segments)
    starts = rng.permutation(max(1, n // block))
    rays = 0
    t0 = time.perf_counter()
    done = []
    hits = []
    for b in starts:
        lo = int(b) * block
        hi = min(n, lo + block)
        h, _, _, st = O.trace(w.segments[lo:hi], w.atmosphere, w.telescopes, w.params,
                              n_showers=w.n_showers, seg_base=lo, threads=threads)
        rays += st["rays"]
        done.append(lo)
        if keep_hits:
            hits.append(h)
        if time.perf_counter() - t0 > budget_s:
            break
    return rays, done, time.perf_counter() - t0, hits


def _block_of(w):
    # the batch's steps vary widely in cost (isotropic fluorescence): larger
    # blocks keep every host core busy
    return 4096 if w.n_showers > 1 else 256


def cpu_baseline(w, budget_s=12.0, seed=0, single_s=0.0, keep_hits=False):
    """The FP64 oracle on random blocks of the same workload (host cores;
    optionally also on one thread)."""
    n = len(w.segments)
    block = _block_of(w)
    rays, done, dt, hits = _oracle_blocks(w, budget_s, block, seed, 0, keep_hits)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": rays / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{len(done)} random blocks of {block} consecutive steps ({len(done) * block} of {n} "
                     f"steps, {rays} rays) of the same workload, {dt:.1f} s, FP64 oracle with OpenMP"}
    if single_s > 0:
        r1, d1, t1, _ = _oracle_blocks(w, single_s, block, seed + 1, 1)
        out["single_thread"] = {"value": r1 / t1, "unit": UNIT, "sample": f"{len(d1)} blocks, {r1} rays, {t1:.1f} s"}
    return out, done, block, hits


def oracle_error(gpu_hits, blocks, block, ref_hits, tels):
    """Per-output errors of the GPU hits against the oracle's on the blocks
    the CPU baseline traced: max |dx|, |dy| (m), |dt| (ns), relative weight
    and wavelength, direction cosines; hits present on one side only."""
    if not blocks:
        return None
    ref = np.concatenate(ref_hits) if ref_hits else np.zeros(0, dtype=gpu_hits.dtype)
    sel = np.isin(gpu_hits["seg"] // block, np.asarray(blocks, dtype=np.int64) // block)
    g = gpu_hits[sel]

    def key(h):
        return (h["seg"].astype(np.int64) * (1 << 20) + h["k"].astype(np.int64)) * 65536 + h["tel"].astype(np.int64)
    kg, kr = key(g), key(ref)
    common, ig, ir = np.intersect1d(kg, kr, return_indices=True)
    a, b = g[ig], ref[ir]
    R = tels["R"].astype(np.float64)
    only_ref = np.setdiff1d(np.arange(len(ref)), ir)
    edge = np.abs(ref["dperp"][only_ref] - R[ref["tel"][only_ref]]) < 0.01 if len(only_ref) else np.zeros(0, bool)

    def mx(v):
        return float(np.max(v)) if len(v) else 0.0
    return {"steps": int(len(blocks) * block), "hits_compared": int(len(common)),
            "only_oracle": int(len(only_ref)), "only_oracle_at_edge": int(edge.sum()),
            "only_gpu": int(len(g) - len(common)),
            "max_x_m": mx(np.abs(a["x_rel"] - b["x_rel"])), "max_y_m": mx(np.abs(a["y_rel"] - b["y_rel"])),
            "max_t_ns": mx(np.abs(a["t"] - b["t"])),
            "max_weight_rel": mx(np.abs(a["weight"] / b["weight"] - 1.0)),
            "max_lambda_rel": mx(np.abs(a["lambda"] / b["lambda"] - 1.0)),
            "max_dir": mx(np.maximum(np.abs(a["cx"] - b["cx"]), np.abs(a["cy"] - b["cy"]))),
            "bars": {"x_m": 0.01, "y_m": 0.01, "t_ns": 0.01}}


def reference_arm(args, rank):
    """The oracle timed on the host cores, on bounded samples of the workload."""
    if rank != 0:
        return 0
    w = make_workload(args.workload, args.n_segs, 0, args.scale)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    for i in range(args.warmup + args.steps):
        r, _, _, _ = cpu_baseline(w, budget_s=per_step, seed=i)
        if i >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "segments": len(w.segments), "showers": w.n_showers,
                       "telescopes": len(w.telescopes), "bunch": w.params.bunch},
            "cpu_baseline": {"kind": "oracle", "cores": vals[0]["cores"], "sample": vals[0]["sample"],
                             "value": v, "unit": UNIT},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


WORKLOADS = ("batch", "shower_1tev", "inclined", "adjoint")


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


def strided_sample(torch, segs_u8, n, m, blocks=64):
    """m steps (a multiple of 32 per block) in `blocks` blocks spread evenly over
    the n steps of a device step array: every shower of a batch contributes in
    proportion to its size."""
    if m >= n:
        return segs_u8, n
    b = max(32, (m // blocks) // 32 * 32)
    nb = min(blocks, max(1, n // b))
    v = segs_u8.view(n, 64)
    parts = [v[(i * (n - b)) // max(1, nb - 1):(i * (n - b)) // max(1, nb - 1) + b] for i in range(nb)]
    return torch.cat(parts).reshape(-1), nb * b


def timed_calls(torch, ctx, segs, n, ns, hits, cap, counts, sums, k, warm=1, fp64=False):
    """Median of k timed calls (CUDA events on the current stream) after `warm` calls."""
    s = torch.cuda.current_stream()
    st = None
    for _ in range(warm):
        _, _, st = ctx.trace(segs, n, ns, hits, cap, counts, sums, fp64=fp64)
    ts = []
    for _ in range(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _, _, st = ctx.trace(segs, n, ns, hits, cap, counts, sums, fp64=fp64)
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=WORKLOADS,
                    help="batch: 256 showers with fluorescence, 7.92e8 steps, autotuned (the default); "
                         "shower_1tev: one 2e7-step vertical 1 TeV shower; inclined: 1e8 steps at 60 deg over "
                         "441 telescopes; adjoint: 1e6 steps, forward + adjoint per step")
    ap.add_argument("--n-segs", type=int, default=0)
    ap.add_argument("--scale", type=float, default=1.0, help="segment-count scale of the batch workload")
    ap.add_argument("--peaks", action="store_true", help="only measure the pipe throughputs and print them")
    ap.add_argument("--no-peaks", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-guard", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--noalloc", action="store_true",
                    help="also time clight_trace_noalloc (unsorted hits, no allocation) on the same steps")
    ap.add_argument("--tune-sample", type=int, default=40_000_000)
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
    ap.add_argument("--work-chunk", type=int, default=0)
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
    if args.peaks:
        print(json.dumps({"pipe_rates": G.pipe_rates(local)}), flush=True)
        return 0
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
        c, r = I.beam_cone(w.telescopes)
        w.params = dataclasses.replace(w.params, fl_beaming=1, beam_centre=c, beam_radius=r)
    if args.fl_roulette:
        w.params = dataclasses.replace(w.params, fl_roulette=1)
    ns = w.n_showers
    ctx = G.Context(local)
    extra = dict(use_graph=1, precision=args.precision, block=args.block, ctas_per_sm=args.ctas_per_sm,
                 cell_width=args.cell_width, work_chunk=args.work_chunk,
                 propagator=1 if args.propagator == "straight" else 0)
    ctx.setup(w, **extra)
    dev = f"cuda:{local}"
    segs = torch.from_numpy(w.segments.view(np.uint8).reshape(-1)).to(dev)
    n = len(w.segments)
    cap = max(1 << 20, n // 4)
    hits = torch.empty(cap * 48, dtype=torch.uint8, device=dev)
    ng = ns * len(w.telescopes)
    counts = torch.zeros(ng, dtype=torch.int64, device=dev)
    sums = torch.zeros(ng, dtype=torch.float64, device=dev)

    # measured pipe throughputs (the roofline's denominators)
    pipes = None
    if not args.no_peaks:
        pipes = G.pipe_rates(local)

    tune = None
    if args.workload == "batch" and not args.no_tune:
        # a sample spread over every shower picks bunch (<= 5), launch shape, work chunk, cell width
        tune = ctx.autotune(segs, n, min(n, args.tune_sample), ns, hits, cap, bunch_max=w.params.bunch, reps=5)
        extra.update(block=tune["block"], ctas_per_sm=tune["ctas_per_sm"], cell_width=tune["cell_width"],
                     work_chunk=tune["work_chunk"])
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
    adj_ms = []

    def step():
        out = ctx.trace(segs, n, ns, hits, cap, counts, sums)
        if adj is not None:
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(torch.cuda.current_stream())
            ctx.trace_adjoint(segs, n, ns, hits, out[1], **adj)
            a1.record(torch.cuda.current_stream())
            a1.synchronize()
            adj_ms.append(a0.elapsed_time(a1))
        return out

    for _ in range(args.warmup):
        step()
    adj_ms.clear()
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
    deferred = st["deferred"] > 0 or (args.precision == 0 and args.disp_B == 0)
    # a call with the default queue runs in pieces of half the queue's entries
    piece = min(max(2 * n, 1 << 20), 1 << 28) // 2
    pieces = -(-n // piece) if deferred else 1
    launches_per_step = (2 if deferred else 1) * pieces + 5 * passes + 3 + (3 if adj is not None else 0)

    # ---- roofline of the dominant kernels (generation + propagation + hits)
    k_ms = statistics.mean(kms)
    k_s = k_ms / 1e3
    skipped = st["skipped"]
    decided = st["rays"] - skipped
    nodes = st["cells"] * NODES_PER_CELL
    ops8 = skipped * OPS8D_SKIPPED + decided * OPS8D_TRACED + nodes * OPS8D_NODE
    # rays the first pass decided (two-pass path) or the in-place kernel skipped
    short = st["rays"] - st["deferred"] if st["deferred"] else skipped + st["escaped"] + st["under"]
    ops_src = (short * SRC_OPS_SKIPPED + (st["rays"] - short) * SRC_OPS_RAY +
               st["cells"] * (SRC_OPS_CELL + NODES_PER_CELL * SRC_OPS_NODE))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    if pipes is not None and pipes["ffma_per_s"] > 0:
        # the measured FP32-FMA rate, scaled from the probe's clock to the
        # median SM clock sampled during the timed region
        f_run = (ck or {}).get("sm_mhz") or pipes["ffma_mhz"]
        peak = pipes["ffma_per_s"] * f_run / pipes["ffma_mhz"]
        peak_basis = (f"measured: FP32 FMA probe {pipes['ffma_per_s'] / 1e12:.2f} Tops/s at "
                      f"{pipes['ffma_mhz']:.0f} MHz ({pipes['ffma_per_s'] / (n_sm * pipes['ffma_mhz'] * 1e6):.1f} "
                      f"per SM per clock), scaled to {f_run:.0f} MHz")
    else:
        peak = n_sm * 128 * 2070e6
        peak_basis = f"nominal: {n_sm} SMs x 128 FP32 lanes x 2070 MHz"
    traffic = recorded_traffic(w.name, n) if args.precision == 0 else None
    trec = traffic_record(w.name) if args.precision == 0 else None
    roof = {"bound": "alu", "achieved": ops8 / k_s / 1e12, "peak": peak / 1e12, "unit": "Tops/s (FP32 pipe)",
            "frac": ops8 / k_s / peak, "traffic": traffic,
            "kernel": "k_classify + k_trace_deferred" if deferred else "k_trace_fused",
            "kernel_ms": k_ms, "sort_ms": statistics.mean(sms),
            "work": f"per-unit work of the measurement plan: {OPS8D_SKIPPED} ops per ray decided from its vacuum "
                    f"line ({skipped}), {OPS8D_TRACED} per other ray ({decided}), {OPS8D_NODE} per quadrature "
                    f"node ({nodes}); {ops8 / max(1, st['rays']):.1f} ops per ray",
            "peak_basis": peak_basis,
            "source_counted": {"achieved": ops_src / k_s / 1e12, "frac": ops_src / k_s / peak,
                               "ops_per_ray": ops_src / max(1, st["rays"])},
            "step_skipped_uncredited": {"frac": (ops8 - st.get("step_skipped", 0) * OPS8D_SKIPPED) / k_s / peak,
                                        "note": "the same per-unit work with the rays decided per step (never "
                                                "drawn) credited nothing"},
            "hbm": {"achieved_gbs": (n * 64 + nh * 48) / k_s / 1e9,
                    "note": "algorithmic bytes: the 64-byte steps read once and the 48-byte hits written"}}
    if trec is not None:
        # the last capture's figure; `traffic` above is null unless it was
        # taken from the sources that now run
        roof["traffic_record"] = trec
    if pipes is not None and pipes["mufu_ex2_per_s"] > 0:
        roof["pipes_measured"] = {k: pipes[k] for k in ("ffma_per_s", "mufu_ex2_per_s", "dfma_per_s", "imad_per_s",
                                                        "lop3_per_s", "ffma_mhz")}

    # ---- the adjoint's own kernels
    adjoint = None
    if adj is not None and adj_ms:
        info = ctx.last_adjoint()
        n_par = len(w.atmosphere.c) + 2
        units = info["candidates"] + info["hits"]
        work = units * ADJ_OPS_PER_UNIT * (1 + n_par)
        adjoint = {"ms_per_step": statistics.mean(adj_ms), "hits": info["hits"], "candidates": info["candidates"],
                   "phases_ms": {"candidate_pass": info["candidate_ms"], "candidate_sort": info["sort_ms"],
                                 "tangent_kernels": info["tangent_ms"]},
                   "note": "candidate pass + sort + tangent kernels + fixed-order sum, CUDA events (last call)"}
        if pipes is not None and info["tangent_ms"] > 0:
            adjoint["roofline"] = {
                "bound": "alu", "kernel": "k_adjoint_soft + k_adjoint_hits",
                "achieved": work / (info["tangent_ms"] * 1e-3) / 1e12, "peak": peak / 1e12,
                "unit": "Tops/s (FP32 pipe)", "frac": work / (info["tangent_ms"] * 1e-3) / peak,
                "work": f"{ADJ_OPS_PER_UNIT} ops per candidate ray or hit (a traced ray, {ADJ_NODES} quadrature nodes) "
                        f"x (1 + {n_par}) for the value and {n_par} tangents; {units} units"}

    # ---- angular segment cut: the same step with the cut on
    cut = None
    if args.cut_study:
        base_sum, base_hits = float(sums.sum().item()), nh
        cut = []
        for mode in (1, 2):
            p2 = dataclasses.replace(w.params, cut_mode=mode, cut_deg=6.0, cut_centre=I.array_centre(w.telescopes))
            ctx.set_params(p2, **extra)
            kc = max(5, args.steps // 4)
            cms, st_c = timed_calls(torch, ctx, segs, n, ns, hits, cap, counts, sums, kc, warm=3)
            cut.append({"mode": ["", "array centre", "each telescope"][mode], "deg": 6.0,
                        "segments_cut": int(st_c["cut"]), "rays": int(st_c["rays"]), "ms_per_step": cms,
                        "speedup": ms_step / cms, "hits_kept": st_c["hits"] / max(1, base_hits),
                        "photon_loss": 1.0 - float(sums.sum().item()) / base_sum if base_sum else None})
        ctx.set_params(w.params, **extra)

    # the GPU's hits of the timed call, for the comparison with the oracle
    gpu_hits = hits[: nh * 48].cpu().numpy().view(G.HIT_DTYPE).copy() if rank == 0 and not args.no_cpu else None

    # ---- plain FP64 GPU path, and the FP32 path on the same steps with and
    # without the skip of rays that provably land clear of every telescope
    fp64 = None
    if not args.no_fp64:
        sub, n64 = strided_sample(torch, segs, n, 20_000_000)
        f64_ms, st64 = timed_calls(torch, ctx, sub, n64, ns, hits, cap, counts, sums, 1, warm=1, fp64=True)
        v64 = st64["rays"] / (f64_ms / 1e3)
        ctx.set_params(w.params, **{**extra, "use_graph": 0, "trace_all": 1})
        all_ms, st_all = timed_calls(torch, ctx, sub, n64, ns, hits, cap, counts, sums, 3, warm=1)
        ctx.set_params(w.params, **{**extra, "use_graph": 0})
        d_ms, st_d = timed_calls(torch, ctx, sub, n64, ns, hits, cap, counts, sums, 3, warm=1)
        ctx.set_params(w.params, **extra)
        v_all = st_all["rays"] / (all_ms / 1e3)
        v_d = st_d["rays"] / (d_ms / 1e3)
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": f64_ms, "segments": n64,
                "sample": f"{n64} steps in 64 blocks spread over the workload",
                "speedup_of_fp32": value / v64 if v64 else None,
                "fp32_same_steps": {"value": v_d, "ms_per_step": d_ms, "speedup": v_d / v64},
                "fp32_trace_all_same_steps": {"value": v_all, "ms_per_step": all_ms, "speedup": v_all / v64,
                                              "note": "every ray traced in full: the same algorithm as the "
                                                      "FP64 path, so this ratio is the precision's share"},
                "split": {"precision": v_all / v64, "algorithm": v_d / v_all}}

    # ---- FP64 at the precise steps (the literal precision pattern), same workload
    guard = None
    if not args.no_guard and args.precision == 0:
        ctx.set_params(w.params, **{**extra, "precision": 1, "use_graph": 0})
        g_ms, st_g = timed_calls(torch, ctx, segs, n, ns, hits, cap, counts, sums, 2, warm=1)
        ctx.set_params(w.params, **extra)
        guard = {"value": st_g["rays"] / (g_ms / 1e3), "unit": UNIT, "ms_per_step": g_ms,
                 "note": "binary64 at the altitude-from-position and horizontal-distance steps instead of FP32 "
                         "pairs (in-place kernel); same hits within tolerance"}

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

    # ---- the 2e7-step 1 TeV shower as a secondary figure
    secondary = None
    if args.workload == "batch" and not args.no_secondary:
        w1 = make_workload("shower_1tev", 0, rank, 1.0)
        ctx.setup(w1, use_graph=1)
        s1 = torch.from_numpy(w1.segments.view(np.uint8).reshape(-1)).to(dev)
        n1 = len(w1.segments)
        c1 = torch.zeros(len(w1.telescopes), dtype=torch.int64, device=dev)
        u1 = torch.zeros(len(w1.telescopes), dtype=torch.float64, device=dev)
        ms1, st1 = timed_calls(torch, ctx, s1, n1, 1, hits, cap, c1, u1, 10, warm=3)
        k1, _ = ctx.last_timing()
        secondary = {"workload": w1.name, "value": st1["rays"] / (ms1 / 1e3), "unit": UNIT, "ms_per_step": ms1,
                     "kernel_ms": k1, "rays": st1["rays"], "skipped": st1["skipped"], "deferred": st1["deferred"]}
        del s1

    # ---- the entry point that allocates nothing (in-place kernel, unsorted hits)
    noalloc = None
    if args.noalloc:
        s0 = torch.cuda.current_stream()
        for _ in range(2):
            code_n, nh_n, st_n = ctx.trace_noalloc(segs, n, ns, hits, cap, counts, raise_on_error=False)
        na_ms = []
        for _ in range(max(3, args.steps // 4)):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(s0)
            code_n, nh_n, st_n = ctx.trace_noalloc(segs, n, ns, hits, cap, counts, raise_on_error=False)
            a1.record(s0)
            torch.cuda.synchronize()
            na_ms.append(a0.elapsed_time(a1))
        m_na = statistics.median(na_ms)
        noalloc = {"status": int(code_n), "ms_per_step": m_na, "value": st_n["rays"] / (m_na / 1e3), "unit": UNIT,
                   "hits": int(nh_n), "note": "clight_trace_noalloc: static scratch, unsorted hits, per-group counts"}

    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, blocks, blk, ref_hits = cpu_baseline(w, single_s=4.0, keep_hits=True)
        err = oracle_error(gpu_hits, blocks, blk, ref_hits, w.telescopes)

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
                       "propagator": args.propagator, "dispersion_B_nm2": args.disp_B,
                       "step": "trace + adjoint" if adj is not None else "trace"},
            "rays_fully_traced_per_s": st["deferred"] * args.steps / (ms / 1e3),
            "skip_fraction": st["skipped"] / max(1, st["rays"]),
            "roofline": roof, "fp64_plain": fp64, "fp64_guard": guard, "e2e": e2e, "cpu_baseline": cpu,
            "oracle_error": err, "clocks": ck, "gpu_launches": launches_per_step * args.steps,
            "stats": {k: int(v) for k, v in st.items()},
        }
        if tune is not None:
            line["autotune"] = tune
        if secondary is not None:
            line["secondary"] = secondary
        if adjoint is not None:
            line["adjoint"] = adjoint
        if cut is not None:
            line["angular_cut"] = cut
        if noalloc is not None:
            line["noalloc"] = noalloc
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
