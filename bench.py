#!/usr/bin/env python
"""Benchmark of the baryon pasting hot path on the full-scale light-cone.

Workload (one step, the headline): 5e8 particles in a 5x5 deg^2 light-cone to z = 3 (60%
from 2e5 truncated-NFW halos with dN/dlnM ~ M^-0.9 on 1e12-1e15 h^-1 Msun, 40% field),
4096^2 maps.  A step solves the ICM model of the 2e5 halos, assigns the particle signals,
pastes them (pair list, radix sort, tensor-core deposit, partial-tile reduction), pastes the
halos' projected profiles onto their own 4096^2 maps (second stream) and finalises both map
pairs.  On N GPUs (torchrun) the same sky is shared: particles and halos are partitioned by
index, each rank fills full map planes and one all-reduce sums them (strong scaling).

Side sections on one GPU: the 4e6-particle 2x2 deg^2 cone, the 1000-halo HP catalogue,
the surrogate against the plain solve, smoothing lengths, the power spectrum, batched HP
and the all-sky HP map.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a bounded,
representative sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pasted particles/s (PP), halos/s (HP), frac of HBM roofline; surrogate vs solve"
UNIT = "particles/s"
WORKLOAD = ("PP full-scale: 5e8 particles (SoA FP32 positions, velocities, smoothing lengths, "
            "int32 halo id) in a 5x5 deg^2 light-cone z 0.05-3, 2e5 halos (dN/dlnM ~ M^-0.9 on "
            "1e12-1e15 h^-1 Msun; 60% halo / 40% field particles), 4096^2 y and kSZ maps; plus HP "
            "of the 2e5 halos on 4096^2 maps")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# the oracle's sample of the full-scale cone: a seeded subset of the halos with all of their
# particles, and the same share of the field particles (inputs.lightcone_device(sample=...))
REF_SAMPLE = (1.0e-3, 1.0e-3)


def config(args, world):
    """The workload description shared by both arms (and every N)."""
    return {"workload": WORKLOAD, "particles": args.particles, "halos": args.halos,
            "maps": f"{args.npix}x{args.npix}", "pp_tile": 64,
            "deposit_kernel": "tcgen05 split-FP16 (power-of-two scaled operands, FP32 accumulation)",
            "l2": "inputs (16 GB of particles) far larger than L2; 256 MB written between "
                  "timed steps as well",
            "parallelism": "single sky, particles and halos partitioned by index, one map "
                           f"all-reduce (x{world})" if world > 1 else "one GPU"}


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (the step time a multi-rank job reports)."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def f16_peak(peaks, sustained=False):
    """FP16 dense peak (FP32 accumulation): the measured cuBLAS bf16 rate (the nominal FP16 and
    BF16 dense rates are equal); the burst rate for a kernel timed alone, the sustained one for
    a kernel timed inside a long step."""
    key = "bf16_tflops_sustained" if sustained and "bf16_tflops_sustained" in peaks else "bf16_tflops"
    return float(peaks.get(key, 1900.0))


def fp32_peak(peaks):
    """FP32 FMA peak: 152 SMs x 128 lanes x 2 flops x the maximum SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi samples of SM clock, utilisation and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,utilization.gpu,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
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
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 10:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        load = [r for r in rows if num(r[3]) >= 50] or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(num(r[1]) for r in load),
                "sm_max_mhz": max(num(r[2]) for r in rows), "reasons": reasons,
                "samples": len(rows), "samples_under_load": len(load)}


def phase_bandwidth(ph, n, n_pairs, nx, ny, hbm_peak):
    """Algorithmic bytes of the streaming phases over their live durations, and the
    fraction of the measured HBM copy bandwidth (GB/s)."""
    maps = 2 * nx * ny * 4  # one FP32 plane of y and of b
    bytes_ = {
        # particle SoA 8 x 4 B in, 32 B record out
        "assign": n * 64,
        # two reads of the 32 B records (count, emit), counts 4 B, offsets 8 B, pairs 8 B
        "pairs": n * (32 + 32 + 4 + 8) + n_pairs * 8,
        # per 8-bit pass: key read for the histogram, key + value read and written; key read
        # for the tile ranges (one pass for <= 256 tiles, two for 4096)
        "sort": n_pairs * (4 + 16) * (1 if nx * ny <= 256 * 64 * 64 else 2) + n_pairs * 4,
        # map and lo planes of y and b read and written, for the PP and the HP maps (both
        # finalised on the particle chain's stream)
        "finalize": 8 * maps,
    }
    out = {}
    for k, b in bytes_.items():
        ms = ph.get(k, 0.0)
        if ms > 0:
            gbs = b / (ms * 1e-3) / 1e9
            out[k] = {"bytes": b, "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)}
    return out


def deposit_work(rec, nx, ny, tile=64, sspan=0):
    """Algorithmic work of one deposit, computed with torch on the records' device, split
    between the tensor-core kernel and the small-particle kernel (particles whose clipped
    pixel box is at most `sspan` pixels wide; 0: none): flops = 2 per pixel update (one FMA)
    per map the particle touches (field particles carry no y) over every particle's clipped
    2h x 2h footprint; pixel updates; and the (tile, particle) pairs of the pair list (the
    tiles each footprint's pixel box touches)."""
    import torch

    ints = rec.view(torch.int32)
    w = {k: 0.0 for k in ("flops", "flops_tc", "updates", "pairs", "pairs_tc")}
    for a in range(0, rec.shape[0], 50_000_000):
        r = rec[a:a + 50_000_000]
        iv = ints[a:a + 50_000_000]
        px = iv[:, 6].double() + r[:, 0].double()
        py = iv[:, 7].double() + r[:, 1].double()
        hp = r[:, 2].double()
        i0, i1 = torch.floor(px - hp), torch.floor(px + hp)
        j0, j1 = torch.floor(py - hp), torch.floor(py + hp)
        ok = (iv[:, 5] != 2) & (i1 >= 0) & (i0 <= nx - 1) & (j1 >= 0) & (j0 <= ny - 1)
        ci0, ci1 = i0.clamp(0, nx - 1)[ok], i1.clamp(0, nx - 1)[ok]
        cj0, cj1 = j0.clamp(0, ny - 1)[ok], j1.clamp(0, ny - 1)[ok]
        upd = (ci1 - ci0 + 1) * (cj1 - cj0 + 1)
        fl = 2.0 * upd * torch.where(r[:, 3][ok] != 0, 2.0, 1.0).double()
        tp = ((torch.floor(ci1 / tile) - torch.floor(ci0 / tile) + 1) *
              (torch.floor(cj1 / tile) - torch.floor(cj0 / tile) + 1))
        big = torch.maximum(ci1 - ci0, cj1 - cj0) + 1 > sspan
        w["flops"] += float(fl.sum())
        w["flops_tc"] += float(fl[big].sum())
        w["updates"] += float(upd.sum())
        w["pairs"] += float(tp.sum())
        w["pairs_tc"] += float(tp[big].sum())
    w["pairs"], w["pairs_tc"] = int(w["pairs"]), int(w["pairs_tc"])
    return w


def small_span_auto(nx, ny, tile=64):
    """The small-particle span the library picks by default: 8 pixels on maps with at least
    4 tiles per SM, else 0 (every particle on the tensor cores)."""
    return 8 if -(-nx // tile) * -(-ny // tile) >= 4 * SM_COUNT else 0


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it was
    captured on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_counters.json")
    try:
        d = json.load(open(path))[kernel_key]
    except Exception:
        return None
    files = d["sources"] if "sources" in d else [d["source"]]
    try:
        src = b"".join(open(os.path.join(ROOT, "paper_2201_02632_gb300", "csrc", f), "rb").read()
                       for f in files)
    except OSError:
        return None
    if hashlib.sha256(src).hexdigest()[:16] != d.get("source_sha256_16"):
        return None
    return d.get("dram_bytes_per_launch_scaled")


def deposit_roofline(kernel, ph, work, peaks, traffic_key, sustained=False):
    """Roofline entry of the tensor-core deposit from its live CUDA-event duration and the
    algorithmic flops of the particles it deposits (against the FP16 tensor peak of
    measured: its MMAs take FP16 operands), plus the MMA work it issues; the small-particle
    kernel (FP32 ALU and shared memory) beside it."""
    dep_ms, small_ms = ph["deposit"], ph.get("deposit_small", 0.0)
    achieved = work["flops_tc"] / (dep_ms * 1e-3) / 1e12
    peak = f16_peak(peaks, sustained)
    # per (tile, particle) pair the kernel issues a 128 x 64 rank-1 update in three
    # split-FP16 products
    mma = work["pairs_tc"] * 128 * 64 * 2 * 3
    out = {"kernel": kernel, "bound": "tensor", "achieved": achieved, "peak": peak,
           "unit": "TFLOP/s", "frac": achieved / peak, "traffic": ncu_traffic(traffic_key),
           "deposit_ms": dep_ms, "algorithmic_flops_per_launch": work["flops_tc"],
           "pixel_updates_all": work["updates"], "tile_pairs": work["pairs_tc"],
           "mma_flops_issued_per_launch": mma,
           "mma_tflops_issued": mma / (dep_ms * 1e-3) / 1e12,
           "frac_fp32_alu_peak": achieved / fp32_peak(peaks),
           "peak_note": ("of measured: bf16 " + ("sustained" if sustained else "burst") +
                         f" {peak:.1f} TFLOP/s (nominal FP16 and BF16 dense rates are equal)")}
    if small_ms > 0:
        fs = work["flops"] - work["flops_tc"]
        out["small"] = {"kernel": "k_deposit_small", "bound": "alu", "ms": small_ms,
                        "algorithmic_flops_per_launch": fs,
                        "tile_pairs": work["pairs"] - work["pairs_tc"],
                        "achieved": fs / (small_ms * 1e-3) / 1e12, "peak": fp32_peak(peaks),
                        "unit": "TFLOP/s",
                        "frac": fs / (small_ms * 1e-3) / 1e12 / fp32_peak(peaks)}
    return out


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample_step(sample_lc, threads):
    """One step of the FP64 oracle on the sample cone: solve of the halos its particles
    reference, assign + deposit of its particles, HP of those halos.  Returns (seconds,
    particles, detail)."""
    import oracle as O

    parts = {k: v.cpu().numpy() for k, v in sample_lc.parts.items()}
    cat, gm = sample_lc.halos, sample_lc.geom
    g = O.geom(gm.nx, gm.ny, gm.theta0_x, gm.theta0_y, gm.dtheta)
    hk = np.unique(parts["hid"][parts["hid"] >= 0])
    t0 = time.perf_counter()
    mo = O.solve_referenced(cat.M, cat.c, cat.z, hk, nthreads=threads)
    t1 = time.perf_counter()
    a = O.pp_assign(parts, sample_lc.Mp, cat.pos, mo, g, nthreads=threads)
    O.pp_deposit(a, g, nthreads=threads)
    t2 = time.perf_counter()
    O.hp_map(cat.thx[hk], cat.thy[hk], cat.vlos[hk], mo[hk], g, rtol=1e-8, nthreads=threads)
    t3 = time.perf_counter()
    n = parts["x"].size
    det = {"particles": int(n), "halos_solved": int(hk.size), "solve_s": round(t1 - t0, 3),
           "assign_deposit_s": round(t2 - t1, 3), "hp_s": round(t3 - t2, 3)}
    return t3 - t0, n, det


def sample_cone(args):
    from paper_2201_02632_gb300 import inputs as I

    return I.lightcone_device(n_part=args.particles, n_halo=args.halos, npix=args.npix,
                              device="cpu", sample=REF_SAMPLE)


def sample_text(lc):
    s = lc.info["sample"]
    return (f"seeded sample of the full-scale cone: {s['halos_kept']} of the {lc.halos.M.size} "
            f"halos (each kept with probability {s['halo_keep']}) with all of their particles "
            f"and {s['field_keep']} of the field particles, {s['particles']} particles in all, "
            "with the full cone's particle mass and smoothing lengths; per step the FP64 oracle "
            "solves the sampled halos, assigns and deposits the sampled particles and pastes "
            "the sampled halos on the 4096^2 maps; value = sampled particles / measured step time")


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    lc = sample_cone(args)
    threads = os.cpu_count() or 1
    times, det = [], None
    for k in range(args.warmup + args.steps):
        t, n, det = oracle_sample_step(lc, threads)
        if k >= args.warmup:
            times.append(t)
    t_step = statistics.mean(times)
    v = n / t_step
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
           "higher_is_better": True, "scaling": "strong" if args.gpus > 1 else "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(args, args.gpus),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample_text(lc), "detail": det},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ headline (GPU)
def headline(api, args, dev, rank, world, peaks):
    """The full-scale cone, one sky over `world` ranks.  Returns the line's fields."""
    import torch

    from paper_2201_02632_gb300 import inputs as I
    from paper_2201_02632_gb300 import shard

    t0 = time.perf_counter()
    lc = I.lightcone_device(n_part=args.particles, n_halo=args.halos, npix=args.npix, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    n_all = lc.parts["x"].numel()
    lo, hi = shard.shard_range(n_all, rank, world)
    if world > 1:
        for k in list(lc.parts):
            lc.parts[k] = lc.parts[k][lo:hi].clone()
        torch.cuda.empty_cache()
    n = hi - lo
    cat = lc.halos
    nh = cat.M.size
    hlo, hhi = shard.shard_range(nh, rank, world)
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    keys = list(lc.parts.keys())

    # pinned host copies of this rank's inputs: the end-to-end leg uploads them every step
    t0 = time.perf_counter()
    h_parts = []
    for k in keys:
        h = torch.empty(lc.parts[k].shape, dtype=lc.parts[k].dtype, pin_memory=True)
        h.copy_(lc.parts[k])
        h_parts.append(h)
    h_halo = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
              (cat.M, cat.c, cat.z, cat.pos, cat.thx[hlo:hhi], cat.thy[hlo:hhi],
               cat.vlos[hlo:hhi])]
    h_in = h_parts + h_halo
    d_in = [lc.parts[k] for k in keys] + [t.to(dev) for t in h_halo]
    pin_s = time.perf_counter() - t0
    del lc.parts
    h2d_bytes = sum(t.numel() * t.element_size() for t in h_in)

    ctx = api.Context()
    comp = torch.cuda.current_stream()
    hp_stream = torch.cuda.Stream()
    ctx_hp = api.Context(stream=hp_stream)
    hp_pool = concurrent.futures.ThreadPoolExecutor(1)
    rec = torch.empty((n, api.ASSIGNED_STRIDE), dtype=torch.float32, device=dev)

    def new_maps():
        buf = shard.map_planes(8, 1, g.ny, g.nx, dev)  # PP y, b, ylo, blo; HP y, b, ylo, blo
        return buf, api.Maps(buf[0], buf[1], buf[2], buf[3]), api.Maps(buf[4], buf[5], buf[6],
                                                                         buf[7])

    buf, pp, hp = new_maps()
    out_host = [torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory() for _ in range(4)]
    d2h_bytes = sum(t.numel() * t.element_size() for t in out_host)
    sub = (lambda m: m) if world == 1 else (lambda m: m[:, hlo:hhi].contiguous())

    def step(ins=None, maps=None):
        """One pass of the hot path over this rank's share (ins: device inputs, maps: the
        (buffer, PP maps, HP maps) to fill)."""
        ins = d_in if ins is None else ins
        mbuf, mpp, mhp = (buf, pp, hp) if maps is None else maps
        parts = dict(zip(keys, ins[:len(keys)]))
        M, c, z, pos, thx, thy, vl = ins[len(keys):]
        mbuf.zero_()
        model, status = ctx.solve_halos(M, c, z, raise_on_noconv=False)
        solved = torch.cuda.Event()
        solved.record(comp)

        def halo_paste():
            with torch.cuda.stream(hp_stream):
                hp_stream.wait_event(solved)
                ctx_hp.paste_halos(thx, thy, vl, sub(model), sub(status), g, mhp)
                done = torch.cuda.Event()
                done.record(hp_stream)
                return done

        fut = hp_pool.submit(halo_paste)
        ctx.assign_particles(parts, lc.Mp, pos, model, status, g, out=rec)
        ctx.paste_particles(rec, g, mpp)
        comp.wait_event(fut.result())
        shard.reduce_maps(mbuf, world)
        ctx.finalize(g, mpp)
        ctx.finalize(g, mhp)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    work = deposit_work(rec, g.nx, g.ny, sspan=small_span_auto(g.nx, g.ny))
    ctx.set_timing(True)
    ctx.phase_times()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", 0)))
    barrier()
    if rank == 0:
        sampler.start()
    launches0 = ctx.kernel_launches() + ctx_hp.kernel_launches()
    step_ms, phases = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        phases.append(ctx.phase_times())  # synchronises the stream
        step_ms.append(e0.elapsed_time(e1))
    barrier()
    launches = ctx.kernel_launches() + ctx_hp.kernel_launches() - launches0
    clocks = sampler.stop() if rank == 0 else None
    ctx.set_timing(False)
    t_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)

    # end to end through the public API: this step's inputs uploaded from pinned host memory,
    # the finalised maps read back; serial (copy, step, copy back) ...
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for hsrc, ddst in zip(h_in, d_in):
            ddst.copy_(hsrc, non_blocking=True)
        step()
        for hdst, dsrc in zip(out_host, (pp.y[0], pp.b[0], hp.y[0], hp.b[0])):
            hdst.copy_(dsrc, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    t_e2e_serial = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, dev)

    # ... and pipelined as a production loop runs it: an upload stream copies step k + 1's
    # inputs and a download stream reads step k - 1's maps while step k computes (inputs and
    # maps double-buffered); every step's uploads, compute and downloads lie inside the timed
    # region, which runs from the first upload to the last download
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ins2 = [d_in, [torch.empty_like(t) for t in d_in]]
    maps2 = [(buf, pp, hp), new_maps()]
    outs2 = [out_host, [torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory()
                        for _ in range(4)]]
    ev = lambda: torch.cuda.Event(enable_timing=False)
    in_ready = [ev() for _ in range(args.steps)]
    done = [ev() for _ in range(args.steps)]
    drained = [ev() for _ in range(args.steps)]

    def upload(k):
        with torch.cuda.stream(up):
            if k >= 2:
                up.wait_event(done[k - 2])  # step k - 2 no longer reads this input set
            for hsrc, ddst in zip(h_in, ins2[k % 2]):
                ddst.copy_(hsrc, non_blocking=True)
            in_ready[k].record(up)

    barrier()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0e.record(up)
    upload(0)
    for k in range(args.steps):
        b = k % 2
        if k + 1 < args.steps:
            upload(k + 1)  # queued before step k's host-synchronising calls
        comp.wait_event(in_ready[k])
        if k >= 2:
            comp.wait_event(drained[k - 2])  # those maps have been read back
        step(ins2[b], maps2[b])
        done[k].record(comp)
        with torch.cuda.stream(down):
            down.wait_event(done[k])
            _, m_pp, m_hp = maps2[b]
            for hdst, dsrc in zip(outs2[b], (m_pp.y[0], m_pp.b[0], m_hp.y[0], m_hp.b[0])):
                hdst.copy_(dsrc, non_blocking=True)
            drained[k].record(down)
    down.wait_event(drained[args.steps - 1])
    t1e.record(down)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(t0e.elapsed_time(t1e) / args.steps, world, dev)
    del ins2, maps2

    mean_ph = {k: round(sum(p[k] for p in phases) / len(phases), 4) for k in phases[0]}
    hbm = float(peaks.get("hbm_gbs", 6780.4))
    res = {
        "value": n_all / (t_step * 1e-3), "ms_per_step": t_step,
        "phase_ms": mean_ph,
        "phase_note": "the particle chain's phases on the main stream (solve .. finalize); the "
                      "halo paste runs on a second stream beside it",
        "phase_hbm": phase_bandwidth(mean_ph, n, work["pairs"], g.nx, g.ny, hbm),
        "roofline": deposit_roofline("k_deposit_tc", mean_ph, work, peaks,
                                     "k_deposit_tc_c2", sustained=True),
        "e2e": {"value": n_all / (t_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": h2d_bytes * world, "d2h_bytes_per_step": d2h_bytes * world,
                "ms_per_step": t_e2e, "pipelined": "copies of steps k +- 1 overlap step k",
                "serial_ms_per_step": t_e2e_serial,
                "serial_value": n_all / (t_e2e_serial * 1e-3)},
        "gpu_launches": launches, "clocks": clocks,
        "inputs": {"generate_s": round(gen_s, 2), "pin_s": round(pin_s, 2),
                   "particles_this_rank": n, "halos_pasted_this_rank": hhi - hlo},
    }
    ctx.close()
    ctx_hp.close()
    del d_in, h_in, h_parts, rec, buf, pp, hp, flush
    torch.cuda.empty_cache()
    return res, cat


# ------------------------------------------------------------------ side sections (one GPU)
def lightcone_4m_section(api, dev, args, peaks):
    """The 4e6-particle 2x2 deg^2 cone (3000 halos, 1024^2 maps): the same step, on one GPU."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

    lc = I.lightcone()
    n, cat = lc.parts["x"].size, lc.halos
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    parts = {k: t(v) for k, v in lc.parts.items()}
    M, c, z, pos, thx, thy, vl = (t(a) for a in (cat.M, cat.c, cat.z, cat.pos, cat.thx, cat.thy,
                                                 cat.vlos))
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    ctx = api.Context()
    comp = torch.cuda.current_stream()
    hp_stream = torch.cuda.Stream()
    ctx_hp = api.Context(stream=hp_stream)
    pool = concurrent.futures.ThreadPoolExecutor(1)
    rec = torch.empty((n, api.ASSIGNED_STRIDE), dtype=torch.float32, device=dev)
    pp, hp = api.Maps.zeros(g, dev), api.Maps.zeros(g, dev)

    def step():
        pp.zero_()
        hp.zero_()
        model, status = ctx.solve_halos(M, c, z)
        solved = torch.cuda.Event()
        solved.record(comp)

        def halo_paste():
            with torch.cuda.stream(hp_stream):
                hp_stream.wait_event(solved)
                ctx_hp.paste_halos(thx, thy, vl, model, status, g, hp)
                ctx_hp.finalize(g, hp)
                done = torch.cuda.Event()
                done.record(hp_stream)
                return done

        fut = pool.submit(halo_paste)
        ctx.assign_particles(parts, lc.Mp, pos, model, status, g, out=rec)
        ctx.paste_particles(rec, g, pp)
        ctx.finalize(g, pp)
        comp.wait_event(fut.result())

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    work = deposit_work(rec, g.nx, g.ny, sspan=small_span_auto(g.nx, g.ny))
    ctx.set_timing(True)
    ctx.phase_times()
    ms, phases = [], []
    for k in range(args.c1_steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        phases.append(ctx.phase_times())
        ms.append(e0.elapsed_time(e1))
    ctx.set_timing(False)
    mean_ph = {k: round(sum(p[k] for p in phases) / len(phases), 4) for k in phases[0]}
    t_step = sum(ms) / len(ms)
    out = {"workload": "PP plain, FP32 deposit: 4e6 particles, 2x2 deg^2 light-cone z 0.05-1.5, "
                       "3000 halos (60% halo / 40% field particles), 1024^2 y and kSZ maps; "
                       "plus HP of the 3000 halos (second stream)",
           "ms_per_step": t_step, "particles_per_s": n / (t_step * 1e-3), "phase_ms": mean_ph,
           "phase_hbm": phase_bandwidth(mean_ph, n, work["pairs"], g.nx, g.ny,
                                        float(peaks.get("hbm_gbs", 6780.4))),
           "roofline": deposit_roofline("k_deposit_tc", mean_ph, work, peaks,
                                        "k_deposit_tc_c1")}
    ctx.close()
    ctx_hp.close()
    return out, lc


def hp_catalogue_section(api, dev, args):
    """HP of the 1000-halo catalogue (1x1 deg^2, 256^2, aperture min(r_f, 3 r500)): solve +
    halo records, tables and paste, inputs resident, maps zeroed outside the timed region."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

    cat, gi = I.halo_catalog(n=1000, npix=256)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M, c, z, thx, thy, vl = (t(a) for a in (cat.M, cat.c, cat.z, cat.thx, cat.thy, cat.vlos))
    g = api.geom(gi.nx, gi.ny, gi.theta0_x, gi.theta0_y, gi.dtheta)
    ctx = api.Context()
    maps = api.Maps.zeros(g, dev)

    def once():
        model, status = ctx.solve_halos(M, c, z)
        ctx.paste_halos(thx, thy, vl, model, status, g, maps, ap_r500=3.0)
        ctx.finalize(g, maps)

    for _ in range(5):
        maps.zero_()
        once()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.phase_times()
    ms, phases = [], []
    for _ in range(args.c0_steps):
        maps.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        once()
        e1.record()
        phases.append(ctx.phase_times())
        ms.append(e0.elapsed_time(e1))
    ctx.set_timing(False)
    ctx.close()
    t_ms = statistics.median(ms)
    ph = {k: round(statistics.median(p[k] for p in phases), 4) for k in phases[0]
          if any(p[k] > 0 for p in phases)}
    return {"workload": "HP plain: 1000 halos (M log-uniform 1e13-1e15 h^-1 Msun, c = 5 "
                        "(M/1e14)^-0.1 x 0.1 dex, z 0.05-1), 1x1 deg^2, 256^2 maps, aperture "
                        "min(r_f, 3 r500); FP64 solve, FP32 projected profiles",
            "ms_per_map": t_ms, "halos_per_s": 1000 / (t_ms * 1e-3), "phase_ms": ph,
            "note": "median of the timed repetitions; one map per repetition"}


def surrogate_section(api, dev, args, c2_cat, npix):
    """Surrogate vs plain solve: train on solver outputs, time both solves on the same
    inference halos, and compare the pasted y of the full-scale cone's 2e5 halos on its
    4096^2 maps with each solve."""
    import torch

    from paper_2201_02632_gb300 import inputs as I
    from paper_2201_02632_gb300.surrogate import Surrogate

    ctx = api.Context()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M, c, z, prm = I.surrogate_halos(args.sur_train, seed=I.SEED_BASE + 4)
    sur = Surrogate.init(dev, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = sur.fit(ctx, t(M), t(c), t(z), t(prm), epochs=args.sur_epochs, batch=4096)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    Mi, ci, zi, pi = I.surrogate_halos(args.sur_infer, seed=I.SEED_BASE + 5)
    a = [t(Mi), t(ci), t(zi), t(pi)]
    w = [x[:50000] for x in a[:3]] + [a[3][:, :50000].contiguous()]
    ctx.solve_halos_ex(*w, raise_on_noconv=False)
    sur.solve(ctx, *w, raise_on_noconv=False)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    sur.solve(ctx, *w, polish_iter=0, raise_on_noconv=False)
    (mp, sp), t_plain = timed(lambda: ctx.solve_halos_ex(*a, raise_on_noconv=False))
    (_, _), t_pol = timed(lambda: sur.solve(ctx, *a, polish_iter=4, raise_on_noconv=False))
    (ms, ss), t_sur = timed(lambda: sur.solve(ctx, *a, polish_iter=0, raise_on_noconv=False))
    fallbacks = ctx.last_fallback_count()
    ok = (sp == 0) & (ss == 0)
    rel = {}
    for name in ("r_f", "T", "rho0"):
        k = api.MF[name]
        r = (ms[k][ok] / mp[k][ok] - 1).abs()
        rel[name] = {"max": float(r.max()), "median": float(r.median())}
    # pasted y of the full-scale cone's halos (Table-1 parameters) with each solve
    nh = c2_cat.M.size
    tab1 = np.stack([np.full(nh, 3.97e-6), np.full(nh, 0.026), np.zeros(nh)])
    hc = [t(c2_cat.M), t(c2_cat.c), t(c2_cat.z)]
    m1, s1 = ctx.solve_halos_ex(*hc, params=t(tab1), raise_on_noconv=False)
    m2, s2 = sur.solve(ctx, *hc, t(tab1), polish_iter=0, raise_on_noconv=False)
    half = 0.5 * 5.0 * math.pi / 180.0
    g = api.geom(npix, npix, -half, -half, 2 * half / npix)
    maps = []
    for m_, s_ in ((m1, s1), (m2, s2)):
        mm = api.Maps.zeros(g, dev)
        ctx.paste_halos(t(c2_cat.thx), t(c2_cat.thy), t(c2_cat.vlos), m_, s_, g, mm)
        ctx.finalize(g, mm)
        maps.append(mm.y[0].double())
    y_err = float(torch.linalg.norm(maps[1] - maps[0]) / torch.linalg.norm(maps[0]))
    ctx.close()
    return {"workload": f"train on {args.sur_train} solver outputs, solve {args.sur_infer} halos "
                        "(log M 12-15.3, z 0.01-3, eps_* 0-1e-5, f_* 0.01-0.04, eps_DM 0-0.1); "
                        f"pasted y of the full-scale cone's {nh} halos on {npix}^2 maps",
            "train_s": round(train_s, 2), "train_loss": loss,
            "plain_solve_ms": t_plain, "plain_solve": "FP32 pre-solve + FP64 Newton to 1e-10",
            "surrogate_solve_ms": t_sur,
            "speedup": t_plain / t_sur, "halos_per_s_plain": args.sur_infer / (t_plain * 1e-3),
            "halos_per_s_surrogate": args.sur_infer / (t_sur * 1e-3),
            "fallbacks": int(fallbacks), "rel_diff_vs_plain": rel,
            "pasted_y_rel_l2_vs_plain": y_err,
            "surrogate_solve": "BF16 MLP on the tensor cores seeds the FP32 pre-solve, whose "
                               "solution is accepted where both FP32 residuals are <= 1e-4 "
                               "(rho0, P0 from the pressure condition in FP64); the rest get "
                               "the full FP64 solve",
            "gate": 1e-4,
            "seeded_with_fp64_polish_ms": t_pol,
            "seeded_with_fp64_polish": "the same seed, then FP64 Newton to 1e-10 (at most 4 "
                                       "steps, gate 1e-4)"}


def hsml_section(api, dev, lc):
    """SPH smoothing lengths (N_ngb = 64) of the 4e6-particle cone's particles: from the grid
    density alone and from the rule-of-thumb h of the generator as starting guesses."""
    import torch

    ctx = api.Context()
    x, y, z = (torch.from_numpy(lc.parts[k]).to(dev) for k in "xyz")
    guess = torch.from_numpy(lc.parts["hsml"]).to(dev)
    n = x.numel()
    out = {"workload": f"{n} light-cone particles (positions of the 4e6-particle cone), N_ngb 64"}
    for name, g in (("no_guess", None), ("rule_of_thumb_guess", guess)):
        for _ in range(2):
            h = ctx.smoothing_lengths(x, y, z, 64.0, guess=g)
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            ctx.smoothing_lengths(x, y, z, 64.0, guess=g, out=h)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = float(np.median(ts))
        out[name] = {"ms": t, "particles_per_s": n / (t * 1e-3)}
    ctx.close()
    return out


def spectrum_section(api, dev, dtheta):
    """Flat-sky C_l (30 logarithmic bins, 1e2-1e5) of a 1024^2 and a 4096^2 map; FP64 FFT
    (5 n log2 n flops per map)."""
    import torch

    ctx = api.Context()
    out = {}
    for name, m, d in (("map_1024", torch.randn((1024, 1024), device=dev), dtheta),
                       ("map_4096", torch.randn((4096, 4096), device=dev), dtheta / 4)):
        for _ in range(3):
            ctx.power_spectrum(m, d)
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.power_spectrum(m, d)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = float(np.median(ts))
        npx = m.numel()
        flops = 5.0 * npx * math.log2(npx)
        out[name] = {"shape": list(m.shape), "ms": t, "fp64_tflops": flops / (t * 1e-3) / 1e12}
    ctx.close()
    return out


def hp_pair_estimate(api, model, thx, thy, g, ap_r500=0.0):
    """Estimated pixel-halo pairs of a flat HP paste: the pixel centres inside each aperture,
    pi r_ap^2 in pixels clipped by the share of the aperture's bounding box on the map."""
    import torch

    MF = api.MF
    rf, da = model[MF["r_f"]], model[MF["D_A"]]
    rap = rf if ap_r500 <= 0 else torch.minimum(rf, ap_r500 * model[MF["r500"]])
    r = rap / da / g.dtheta
    cx = (thx - g.theta0_x) / g.dtheta
    cy = (thy - g.theta0_y) / g.dtheta
    fx = ((cx + r).clamp(0, g.nx) - (cx - r).clamp(0, g.nx)) / (2 * r)
    fy = ((cy + r).clamp(0, g.ny) - (cy - r).clamp(0, g.ny)) / (2 * r)
    est = math.pi * r * r * fx * fy
    return float(torch.nan_to_num(est, nan=0.0).sum())


def batched_section(api, dev, args, peaks):
    """Batched HP: many independent maps of uneven halo extents pasted by one prepared
    plan (one persistent launch), autotuned, captured in a CUDA graph and replayed."""
    import torch

    from paper_2201_02632_gb300 import autotune
    from paper_2201_02632_gb300 import inputs as I

    ctx = api.Context()
    cat, gi = I.batched_catalog(n_maps=args.batch_maps, mean_halos=args.batch_halos,
                                npix=args.batch_npix)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M, c, z = t(cat.M), t(cat.c), t(cat.z)
    thx, thy, vl, mid = t(cat.thx), t(cat.thy), t(cat.vlos), t(cat.map_id)
    n = cat.M.size
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    model, status = ctx.solve_halos(M, c, z, raise_on_noconv=False)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    g = api.geom(gi.nx, gi.ny, gi.theta0_x, gi.theta0_y, gi.dtheta, gi.n_maps)
    maps = api.Maps.zeros(g, dev)
    t0 = time.perf_counter()
    cache = os.path.join(tempfile.gettempdir(), "bp_autotune_hp.json")
    best = autotune.tune_hp(ctx, thx, thy, vl, model, status, g, maps, map_id=mid,
                            units=(0, 1024), ctas=(0, 2), reps=2, cache_path=cache,
                            use_cache=False)
    tune_s = time.perf_counter() - t0
    plan = ctx.hp_plan(thx, thy, model, status, g, 0.0, mid, best["tile"], best["unit"],
                       best["ctas_per_sm"])
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ctx.set_stream(torch.cuda.current_stream())
        maps.zero_()
        plan.execute(thx, thy, vl, model, status, maps, mid)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        ctx.set_stream(torch.cuda.current_stream())
        maps.zero_()
        plan.execute(thx, thy, vl, model, status, maps, mid)
    ctx.set_stream(torch.cuda.current_stream())
    for _ in range(3):
        graph.replay()
    ms = []
    for _ in range(args.batch_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    step = sum(ms) / len(ms)
    pairs = plan.pairs
    pix_pairs = hp_pair_estimate(api, model, thx, thy, g)
    plan.close()
    ctx.close()
    del maps
    torch.cuda.empty_cache()
    flops = pix_pairs * 20.0
    ach = flops / (step * 1e-3) / 1e12
    return {"workload": f"{gi.n_maps} maps of {gi.nx}^2 (5x5 deg^2), {n} halos "
                        f"(Poisson({args.batch_halos:g}) per map), M 1e12-1e15 dN/dlnM ~ M^-0.9, "
                        "z 0.01-3, r_ap = r_f",
            "halos": int(n), "tile_pairs": int(pairs), "ms_per_step": step,
            "halos_per_s": n / (step * 1e-3), "maps_per_s": gi.n_maps / (step * 1e-3),
            "autotuned": {k: best[k] for k in ("tile", "unit", "ctas_per_sm", "ms")},
            "tune_s": round(tune_s, 2), "solve_s_plain_fp64": round(solve_s, 3),
            "graph_replay": True,
            "roofline": {"bound": "alu", "pixel_halo_pairs_estimated": pix_pairs,
                         "flops_per_pair": 20, "achieved": ach, "peak": fp32_peak(peaks),
                         "unit": "TFLOP/s", "frac": ach / fp32_peak(peaks),
                         "note": "pairs estimated as pi r_ap^2 per halo clipped to the map; 20 "
                                 "FP32 flops per pair (distance, table interpolation, two "
                                 "compensated sums); whole replay (tables, per-pixel values, "
                                 "paste, reduction) over the FP32 FMA peak"}}


def allsky_section(api, dev, args, peaks):
    """All-sky HP maps on HEALPix (nside 8192, RING) from an all-sky catalogue of 4.1e7
    halos: the solve of every halo and the paste of its projected profiles, inputs resident
    on the device, maps zeroed before each repetition (outside the timed region)."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

    ctx = api.Context()
    n, nside = args.allsky_halos, args.allsky_nside
    cat = I.allsky_catalog(n)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M, c, z, th, ph, v = (t(cat[k]) for k in ("M", "c", "z", "theta", "phi", "vlos"))
    del cat
    maps = api.healpix_maps(nside, dev)
    reps = []
    for rep in range(3):
        maps.zero_()
        torch.cuda.synchronize()
        ctx.set_timing(True)
        ctx.phase_times()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        model, status = ctx.solve_halos(M, c, z, raise_on_noconv=False)
        e[1].record()
        ctx.paste_halos_healpix(th, ph, v, model, status, nside, maps)
        e[2].record()
        torch.cuda.synchronize()
        ph_t = {k: round(x, 2) for k, x in ctx.phase_times().items() if x > 0}
        reps.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), ph_t))
    ctx.set_timing(False)
    solve_ms, paste_ms, phases = min(reps[1:], key=lambda r: r[0] + r[1])
    total = solve_ms + paste_ms
    # the same map with the FP32-gated solve: the FP32 pre-solve's (r_f, T) where both of its
    # residuals are <= 1e-4, the full FP64 solve for the rest
    gate = 1e-4
    maps2 = api.healpix_maps(nside, dev)
    greps = []
    for rep in range(3):
        maps2.zero_()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        model2, status2 = ctx.solve_halos_ex(M, c, z, gate=gate, gated=True,
                                             raise_on_noconv=False)
        nfb = ctx.last_fallback_count()
        e[1].record()
        ctx.paste_halos_healpix(th, ph, v, model2, status2, nside, maps2)
        e[2].record()
        torch.cuda.synchronize()
        greps.append((e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), nfb))
    gs, gp, nfb = min(greps[1:], key=lambda r: r[0] + r[1])
    ya = (maps.y.double() + maps.ylo.double()).flatten()
    yg = (maps2.y.double() + maps2.ylo.double()).flatten()
    bright = ya > 1e-3 * float(ya.max())
    gated = {"gate": gate, "solve_ms": gs, "paste_ms": gp, "map_ms": gs + gp,
             "halos_per_s": n / ((gs + gp) * 1e-3), "fallback_halos": nfb,
             "solve_speedup": solve_ms / gs,
             "y_rel_l2_vs_fp64_solve": float(torch.linalg.norm(yg - ya) / torch.linalg.norm(ya)),
             "y_max_rel_bright_vs_fp64_solve": float(((yg - ya).abs()[bright] /
                                                      ya[bright]).max()),
             "note": "bp_solve_halos_ex in BP_SOLVE_FP32_GATED mode; errors of the pasted y "
                     "map against the map of the FP64 solve (pixels above 1e-3 of the peak "
                     "for the bright-pixel figure)"}
    del maps2, model2, status2, ya, yg, bright
    y = maps.y
    # pixel-halo pairs: the pixels inside each aperture cap, area pi (r_f / D_A)^2 over the
    # pixel area 4 pi / (12 nside^2)
    MF = api.MF
    ang = model[MF["r_f"]] / model[MF["D_A"]]
    pix_pairs = float(torch.nan_to_num(math.pi * ang * ang / (4 * math.pi / (12.0 * nside * nside)),
                                       nan=0.0).sum())
    flops = pix_pairs * 60.0
    ach = flops / (paste_ms * 1e-3) / 1e12
    out = {"workload": f"{n} halos (dN/dlnM ~ M^-0.9 on 1e12-1e15 h^-1 Msun, uniform in comoving "
                       f"volume to z 3, isotropic), HEALPix nside {nside} RING "
                       f"({12 * nside * nside} pixels), y and b with compensation planes",
           "solve_ms": solve_ms, "paste_ms": paste_ms, "map_ms": total, "phases_ms": phases,
           "halos_per_s": n / (total * 1e-3), "fp32_gated_solve": gated,
           "paper": "170 min on 320 CPU cores for one all-sky map of 4.1e7 halos (Section 5.4)",
           "covered_pixel_frac": float((y > 0).float().mean()),
           "roofline_paste": {"bound": "alu", "pixel_halo_pairs_estimated": pix_pairs,
                              "flops_per_pair": 60, "achieved": ach, "peak": fp32_peak(peaks),
                              "unit": "TFLOP/s", "frac": ach / fp32_peak(peaks),
                              "note": "pairs estimated as the aperture cap area over the pixel "
                                      "area; 60 FP32 flops per pair (haversine, asin, two "
                                      "interpolations); the paste phase (pairs, per-pixel "
                                      "values, segment paste) over the FP32 FMA peak"}}
    ctx.close()
    del maps, model, status
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2201_02632_gb300 import api
    from paper_2201_02632_gb300 import build as B

    B.build()
    dev = torch.device("cuda", local)
    peaks = measured_peaks()
    head, c2_cat = headline(api, args, dev, rank, world, peaks)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    res = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config(args, world),
        "roofline": head["roofline"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"], "phase_ms": head["phase_ms"], "phase_note": head["phase_note"],
        "phase_hbm": head["phase_hbm"], "inputs": head["inputs"],
    }
    if world == 1:
        c1, lc1 = lightcone_4m_section(api, dev, args, peaks) if not args.no_c1 else (None, None)
        if c1:
            res["pp_lightcone_4m"] = c1
        if not args.no_c0:
            res["hp_catalogue_1000"] = hp_catalogue_section(api, dev, args)
        if not args.no_surrogate:
            res["surrogate"] = surrogate_section(api, dev, args, c2_cat, args.npix)
        if lc1 is not None and not args.no_hsml:
            res["smoothing_lengths"] = hsml_section(api, dev, lc1)
        if not args.no_spectrum:
            res["power_spectrum"] = spectrum_section(api, dev, 2.0 * math.pi / 180.0 / 1024)
        if not args.no_batched:
            res["batched_hp"] = batched_section(api, dev, args, peaks)
        if not args.no_allsky:
            res["allsky_hp"] = allsky_section(api, dev, args, peaks)
        if not args.no_cpu_baseline:
            threads = os.cpu_count() or 1
            slc = sample_cone(args)
            t_s, n_s, det = oracle_sample_step(slc, threads)
            res["cpu_baseline"] = {"value": n_s / t_s, "unit": UNIT, "cores": threads,
                                   "kind": "oracle", "sample": sample_text(slc), "detail": det}
            if lc1 is not None and "smoothing_lengths" in res:
                import oracle as O

                n1 = lc1.parts["x"].size
                idx = np.arange(0, n1, n1 // 8)[:8]
                t0 = time.perf_counter()
                O.smoothing_lengths_at(lc1.parts["x"], lc1.parts["y"], lc1.parts["z"], idx, 64.0,
                                       nthreads=threads)
                dt = time.perf_counter() - t0
                res["smoothing_lengths"]["cpu_oracle"] = {
                    "particles_per_s": idx.size / dt, "sample": f"{idx.size} particles of {n1}",
                    "cores": threads, "kind": "oracle"}
    print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def deposit_only(api, dev, args, peaks):
    """Profiling mode (not the benchmark line): the particle deposit alone, on the 4e6-particle
    cone (`4m`) or on a seeded sample of the full-scale cone (`full`, a fraction --sample of its
    halos with all their particles and the same fraction of the field particles).  Solves,
    assigns and sorts once, then times --warmup + --steps deposits (pair list rebuilt each
    time) and prints one JSON line with the phase times and the deposit's algorithmic work."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    if args.deposit_only == "4m":
        lc = I.lightcone()
        parts = {k: t(v) for k, v in lc.parts.items()}
    else:
        smp = None if args.sample >= 1.0 else (args.sample, args.sample)
        lc = I.lightcone_device(n_part=args.particles, n_halo=args.halos, npix=args.npix,
                                device=dev, sample=smp)
        parts = lc.parts
    cat = lc.halos
    ctx = api.Context()
    model, status = ctx.solve_halos(t(cat.M), t(cat.c), t(cat.z), raise_on_noconv=False)
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    rec = ctx.assign_particles(parts, lc.Mp, t(cat.pos), model, status, g)
    del parts, lc.parts
    torch.cuda.empty_cache()
    maps = api.Maps.zeros(g, dev)
    work = deposit_work(rec, g.nx, g.ny, sspan=small_span_auto(g.nx, g.ny))
    ctx.set_timing(True)
    ph = []
    for k in range(args.warmup + args.steps):
        maps.zero_()
        ctx.pp_prepare(rec, g)
        ctx.phase_times()
        ctx.pp_deposit(rec, g, maps)
        if k >= args.warmup:
            ph.append(ctx.phase_times())
    ctx.set_timing(False)
    mean = {k: sum(p[k] for p in ph) / len(ph) for k in ("deposit", "reduce", "deposit_small")}
    print(json.dumps({"deposit_only": args.deposit_only, "sample": args.sample,
                      "particles": int(rec.shape[0]), "maps": f"{g.nx}x{g.ny}",
                      "phase_ms": mean, "work": work,
                      "roofline": deposit_roofline("k_deposit_tc", mean, work, peaks, None)}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=500_000_000)
    ap.add_argument("--halos", type=int, default=200_000)
    ap.add_argument("--npix", type=int, default=4096)
    ap.add_argument("--c1-steps", type=int, default=10)
    ap.add_argument("--c0-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c1", action="store_true")
    ap.add_argument("--no-c0", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-hsml", action="store_true")
    ap.add_argument("--no-allsky", action="store_true")
    ap.add_argument("--no-spectrum", action="store_true")
    ap.add_argument("--allsky-halos", type=int, default=41_000_000)
    ap.add_argument("--allsky-nside", type=int, default=8192)
    ap.add_argument("--batch-maps", type=int, default=108)
    ap.add_argument("--batch-halos", type=float, default=5e4)
    ap.add_argument("--batch-npix", type=int, default=2048)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--sur-train", type=int, default=2_000_000)
    ap.add_argument("--sur-infer", type=int, default=10_000_000)
    ap.add_argument("--sur-epochs", type=int, default=6)
    ap.add_argument("--deposit-only", choices=["4m", "full"], default=None,
                    help="profiling mode: time the particle deposit alone on this workload")
    ap.add_argument("--sample", type=float, default=1.0,
                    help="with --deposit-only full: the fraction of the cone's halos (with "
                         "their particles) and field particles")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.deposit_only:
        import torch

        from paper_2201_02632_gb300 import api
        from paper_2201_02632_gb300 import build as B

        B.build()
        torch.cuda.set_device(0)
        return deposit_only(api, torch.device("cuda", 0), args, measured_peaks())
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
