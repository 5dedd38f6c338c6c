#!/usr/bin/env python
"""Benchmark of the baryon pasting hot path on the light-cone workload.

Workload (one step): 4e6 particles in a 2x2 deg^2 cone (z 0.05-1.5; 60% from 3000
truncated-NFW halos, 40% field), 1024^2 maps.  A step solves the ICM model of the
3000 halos, assigns the particle signals, pastes them (pair list, radix sort,
tiled deposit, partial-tile reduction), pastes the 3000 halos' projected profiles
onto their own 1024^2 maps, and finalises both map pairs.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
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
WORKLOAD = ("PP plain, FP32 deposit: 4M particles, 2x2 deg^2 light-cone z 0.05-1.5, 3000 "
            "halos (60% halo / 40% field particles), 1024^2 y and kSZ maps; plus HP of the "
            "3000 halos on 1024^2 maps")
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_seed(rank, base):
    """Seed of the light-cone a rank pastes: each replica draws its own sky."""
    return base + 1 + rank


def max_over_ranks(value, world, device):
    """The largest of the ranks' values (the step time a weak-scaling job reports)."""
    if world <= 1:
        return float(value)
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


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
        # one 8-bit pass: key read for the histogram, key + value read and written,
        # key read for the tile ranges
        "sort": n_pairs * (4 + 16 + 4),
        # map and lo planes of y and b read and written, for the PP maps (the HP maps are
        # finalised on the second stream)
        "finalize": 4 * maps,
    }
    out = {}
    for k, b in bytes_.items():
        ms = ph.get(k, 0.0)
        if ms > 0:
            gbs = b / (ms * 1e-3) / 1e9
            out[k] = {"bytes": b, "GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)}
    return out


def deposit_flops(rec_np, nx, ny):
    """Algorithmic FP32 flops of one deposit launch: 2 per pixel update (one FMA per map)
    over every particle's clipped 2h x 2h footprint; field particles update one map."""
    ints = rec_np.view(np.int32)
    px = ints[:, 6].astype(np.float64) + rec_np[:, 0]
    py = ints[:, 7].astype(np.float64) + rec_np[:, 1]
    hp, Y, kind = rec_np[:, 2].astype(np.float64), rec_np[:, 3], ints[:, 5]
    with np.errstate(invalid="ignore"):
        i0 = np.floor(px - hp)
        i1 = np.floor(px + hp)
        j0 = np.floor(py - hp)
        j1 = np.floor(py + hp)
    ok = (kind != 2) & (i1 >= 0) & (i0 <= nx - 1) & (j1 >= 0) & (j0 <= ny - 1)
    w = np.clip(i1, 0, nx - 1) - np.clip(i0, 0, nx - 1) + 1
    h = np.clip(j1, 0, ny - 1) - np.clip(j0, 0, ny - 1) + 1
    upd = (w * h)[ok].astype(np.float64)
    maps = np.where(Y[ok] != 0, 2.0, 1.0)
    return float(2.0 * np.sum(upd * maps)), float(np.sum(upd))


def deposit_flops_device(rec, nx, ny):
    """deposit_flops computed with torch on the device (for records too large to copy)."""
    import torch

    ints = rec.view(torch.int32)
    out_f, out_u = 0.0, 0.0
    for a in range(0, rec.shape[0], 50_000_000):
        r = rec[a:a + 50_000_000]
        iv = ints[a:a + 50_000_000]
        px = iv[:, 6].double() + r[:, 0].double()
        py = iv[:, 7].double() + r[:, 1].double()
        hp = r[:, 2].double()
        i0, i1 = torch.floor(px - hp), torch.floor(px + hp)
        j0, j1 = torch.floor(py - hp), torch.floor(py + hp)
        ok = (iv[:, 5] != 2) & (i1 >= 0) & (i0 <= nx - 1) & (j1 >= 0) & (j0 <= ny - 1)
        w = i1.clamp(0, nx - 1) - i0.clamp(0, nx - 1) + 1
        h = j1.clamp(0, ny - 1) - j0.clamp(0, ny - 1) + 1
        upd = (w * h)[ok]
        maps = torch.where(r[:, 3][ok] != 0, 2.0, 1.0).double()
        out_f += float(2.0 * (upd * maps).sum())
        out_u += float(upd.sum())
    return out_f, out_u


def ncu_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it was
    captured on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_counters.json")
    try:
        d = json.load(open(path))[kernel_key]
    except Exception:
        return None
    files = d["sources"] if "sources" in d else [d["source"]]
    src = b"".join(open(os.path.join(ROOT, "paper_2201_02632_gb300", "csrc", f), "rb").read()
                   for f in files)
    if hashlib.sha256(src).hexdigest()[:16] != d.get("source_sha256_16"):
        return None
    return d.get("dram_bytes_per_launch_scaled")


# ------------------------------------------------------------------ CPU oracle legs
def oracle_sample(lc, n_part_sample, n_halo_sample, threads):
    """Times the FP64 oracle on a bounded sample of the workload; returns
    (seconds extrapolated to the full step, detail dict)."""
    import oracle as O

    O.build()
    g = O.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    cat = lc.halos
    t0 = time.perf_counter()
    mo = O.solve_halos(cat.M, cat.c, cat.z, nthreads=threads)
    t_solve = time.perf_counter() - t0
    sub = {k: v[:n_part_sample] for k, v in lc.parts.items()}
    t0 = time.perf_counter()
    a = O.pp_assign(sub, lc.Mp, cat.pos, mo, g, nthreads=threads)
    O.pp_deposit(a, g, nthreads=threads)
    t_pp = time.perf_counter() - t0
    hs = slice(0, n_halo_sample)
    t0 = time.perf_counter()
    O.hp_map(cat.thx[hs], cat.thy[hs], cat.vlos[hs], mo[hs], g, rtol=1e-8, nthreads=threads)
    t_hp = time.perf_counter() - t0
    n = lc.parts["x"].size
    nh = cat.M.size
    t_full = t_solve + t_pp * n / n_part_sample + t_hp * nh / n_halo_sample
    det = {"t_solve_all_halos_s": round(t_solve, 3), "t_pp_sample_s": round(t_pp, 3),
           "t_hp_sample_s": round(t_hp, 3), "n_part_sample": n_part_sample,
           "n_halo_sample": n_halo_sample}
    return t_full, det


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    from paper_2201_02632_gb300 import inputs as I

    lc = I.lightcone()
    threads = os.cpu_count() or 1
    times = []
    for k in range(args.warmup + args.steps):
        t, det = oracle_sample(lc, args.ref_particles, args.ref_halos, threads)
        if k >= args.warmup:
            times.append(t)
    t_step = statistics.mean(times)
    n = lc.parts["x"].size
    v = n / t_step
    sample = (f"per step: FP64 oracle solve of all {lc.halos.M.size} halos, assign+deposit of "
              f"{args.ref_particles} particles and HP of {args.ref_halos} halos, extrapolated "
              f"linearly to the full step")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "none (CPU)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ GPU leg
def surrogate_section(api, ctx, dev, lc, args):
    """Surrogate vs plain solve: train on solver outputs, then time both solves on
    the same inference halos, and compare the pasted y of the light-cone halos."""
    import torch

    from paper_2201_02632_gb300 import inputs as I
    from paper_2201_02632_gb300.surrogate import Surrogate

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

    (mp, sp), t_plain = timed(lambda: ctx.solve_halos_ex(*a, raise_on_noconv=False))
    (ms, ss), t_sur = timed(lambda: sur.solve(ctx, *a, raise_on_noconv=False))
    fallbacks = ctx.last_fallback_count()
    ok = (sp == 0) & (ss == 0)
    rel = {}
    for name in ("r_f", "T", "rho0"):
        k = api.MF[name]
        r = (ms[k][ok] / mp[k][ok] - 1).abs()
        rel[name] = {"max": float(r.max()), "median": float(r.median())}
    # pasted y of the light-cone halos (Table-1 parameters) with each solve
    cat = lc.halos
    nh = cat.M.size
    tab1 = np.stack([np.full(nh, 3.97e-6), np.full(nh, 0.026), np.zeros(nh)])
    hc = [t(cat.M), t(cat.c), t(cat.z)]
    m1, s1 = ctx.solve_halos_ex(*hc, params=t(tab1))
    m2, s2 = sur.solve(ctx, *hc, t(tab1))
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    maps = []
    for m_, s_ in ((m1, s1), (m2, s2)):
        mm = api.Maps.zeros(g, dev)
        ctx.paste_halos(t(cat.thx), t(cat.thy), t(cat.vlos), m_, s_, g, mm)
        ctx.finalize(g, mm)
        maps.append(mm.y[0].double())
    y_err = float(torch.linalg.norm(maps[1] - maps[0]) / torch.linalg.norm(maps[0]))
    return {"workload": f"train on {args.sur_train} solver outputs, solve {args.sur_infer} halos "
                        "(log M 12-15.3, z 0.01-3, eps_* 0-1e-5, f_* 0.01-0.04, eps_DM 0-0.1)",
            "train_s": round(train_s, 2), "train_loss": loss,
            "plain_solve_ms": t_plain, "plain_solve": "FP32 pre-solve + FP64 Newton to 1e-10",
            "surrogate_solve_ms": t_sur,
            "speedup": t_plain / t_sur, "halos_per_s_plain": args.sur_infer / (t_plain * 1e-3),
            "halos_per_s_surrogate": args.sur_infer / (t_sur * 1e-3),
            "fallbacks": int(fallbacks), "rel_diff_vs_plain": rel,
            "pasted_y_rel_l2_vs_plain": y_err,
            "surrogate_solve": "BF16 MLP on the tensor cores seeds the FP32 pre-solve, then "
                               "FP64 Newton to 1e-10 (at most 4 steps, gate 1e-4)",
            "gate": 1e-4, "polish_newton_iters": 4}


def hsml_section(api, ctx, dev, lc, args):
    """SPH smoothing lengths (N_ngb = 64) of the step's light-cone particles: from the grid
    density alone and from the rule-of-thumb h of the generator as starting guesses."""
    import torch

    x, y, z = (torch.from_numpy(lc.parts[k]).to(dev) for k in "xyz")
    guess = torch.from_numpy(lc.parts["hsml"]).to(dev)
    n = x.numel()
    out = {"workload": f"{n} light-cone particles (positions of the pasting step), N_ngb 64"}
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
    return out


def allsky_section(api, ctx, dev, args):
    """All-sky HP maps on HEALPix (nside 8192, RING) from an all-sky catalogue of 4.1e7
    halos: the solve of every halo and the paste of its projected profiles, inputs resident
    on the device, maps zeroed before each repetition (outside the timed region)."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

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
    y = maps.y
    out = {"workload": f"{n} halos (dN/dlnM ~ M^-0.9 on 1e12-1e15 h^-1 Msun, uniform in comoving "
                       f"volume to z 3, isotropic), HEALPix nside {nside} RING "
                       f"({12 * nside * nside} pixels), y and b with compensation planes",
           "solve_ms": solve_ms, "paste_ms": paste_ms, "map_ms": total, "phases_ms": phases,
           "halos_per_s": n / (total * 1e-3),
           "paper": "170 min on 320 CPU cores for one all-sky map of 4.1e7 halos (Section 5.4)",
           "covered_pixel_frac": float((y > 0).float().mean())}
    del maps, model, status
    torch.cuda.empty_cache()
    return out


def spectrum_section(api, ctx, dev, maps_y, dtheta):
    """Flat-sky C_l (30 logarithmic bins, 1e2-1e5) of the step's y map and of a 4096^2 map;
    FP64 FFT (5 n log2 n flops per map)."""
    import torch

    out = {}
    for name, m, d in (("step_y_map", maps_y, dtheta),
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
    return out


def batched_section(api, ctx, dev, args):
    """Batched HP: many independent maps of uneven halo extents pasted by one prepared
    plan (one persistent launch), autotuned, captured in a CUDA graph and replayed."""
    import torch

    from paper_2201_02632_gb300 import autotune
    from paper_2201_02632_gb300 import inputs as I

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
    best = autotune.tune_hp(ctx, thx, thy, vl, model, status, g, maps, map_id=mid,
                            units=(0, 1024), ctas=(0, 2), reps=2,
                            cache_path=os.path.join(ROOT, "gpurun_out", "autotune_hp.json"),
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
    plan.close()
    del maps
    torch.cuda.empty_cache()
    return {"workload": f"{gi.n_maps} maps of {gi.nx}^2 (5x5 deg^2), {n} halos "
                        f"(Poisson({args.batch_halos:g}) per map), M 1e12-1e15 dN/dlnM ~ M^-0.9, "
                        "z 0.01-3, r_ap = r_f",
            "halos": int(n), "tile_pairs": int(pairs), "ms_per_step": step,
            "halos_per_s": n / (step * 1e-3), "maps_per_s": gi.n_maps / (step * 1e-3),
            "autotuned": {k: best[k] for k in ("tile", "unit", "ctas_per_sm", "ms")},
            "tune_s": round(tune_s, 2), "solve_s_plain_fp64": round(solve_s, 3),
            "graph_replay": True}


def full_scale_section(api, ctx, dev, args, fp32_peak):
    """The full-scale cone: 5e8 particles, 2e5 halos, 5x5 deg^2 to z = 3, 4096^2 maps."""
    import torch

    from paper_2201_02632_gb300 import inputs as I

    t0 = time.perf_counter()
    lc = I.lightcone_device(n_part=args.full_particles, n_halo=args.full_halos, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    cat = lc.halos
    tt = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    M, c, z, pos = tt(cat.M), tt(cat.c), tt(cat.z), tt(cat.pos)
    n = args.full_particles
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)
    rec = torch.empty((n, api.ASSIGNED_STRIDE), dtype=torch.float32, device=dev)
    pp = api.Maps.zeros(g, dev)

    def step():
        pp.zero_()
        model, status = ctx.solve_halos(M, c, z, raise_on_noconv=False)
        ctx.assign_particles(lc.parts, lc.Mp, pos, model, status, g, out=rec)
        ctx.paste_particles(rec, g, pp)
        ctx.finalize(g, pp)

    step()
    torch.cuda.synchronize()
    flops, updates = deposit_flops_device(rec, g.nx, g.ny)
    ctx.set_timing(True)
    ctx.phase_times()
    ms, phases = [], []
    for _ in range(args.full_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        phases.append(ctx.phase_times())
        ms.append(e0.elapsed_time(e1))
    ctx.set_timing(False)
    step_ms = sum(ms) / len(ms)
    ph = {k: round(sum(p[k] for p in phases) / len(phases), 3) for k in phases[0]}
    # algorithmic bytes of the streaming phases: assign reads 32 B and writes 32 B per
    # particle; the pair count reads 32 B per particle
    assign_gbs = n * 64 / (ph["assign"] * 1e-3) / 1e9 if ph["assign"] > 0 else None
    dep_tf = flops / (ph["deposit"] * 1e-3) / 1e12 if ph["deposit"] > 0 else None
    res = {"workload": f"{n} particles, {cat.M.size} halos (dN/dlnM ~ M^-0.9, 1e12-1e15), "
                       "5x5 deg^2 z 0.05-3, 4096^2 maps", "generate_s": round(gen_s, 2),
           "ms_per_step": step_ms, "particles_per_s": n / (step_ms * 1e-3), "phase_ms": ph,
           "deposit_tflops": dep_tf, "deposit_frac_fp32_peak": dep_tf / fp32_peak if dep_tf else None,
           "pixel_updates": updates, "assign_gbs": assign_gbs}
    del rec, pp, lc
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2201_02632_gb300 import api
    from paper_2201_02632_gb300 import build as B
    from paper_2201_02632_gb300 import inputs as I

    B.build()
    # each rank pastes its own light-cone realisation (independent maps, no collective)
    lc = I.lightcone(n_part=args.particles, seed=replica_seed(rank, I.SEED_BASE))
    n = lc.parts["x"].size
    cat = lc.halos
    nh = cat.M.size
    dev = torch.device("cuda", local)
    ctx = api.Context()
    ctx.set_deposit_kernel(args.deposit_kernel)
    # the halo paste needs only the solve: a second context on its own stream (fed by a
    # host thread, since the list build synchronises its stream) runs it beside the particle
    # chain (assign, pairs, sort, deposit)
    comp = torch.cuda.current_stream()
    hp_stream = torch.cuda.Stream()
    ctx_hp = api.Context(stream=hp_stream)
    hp_pool = concurrent.futures.ThreadPoolExecutor(1)
    uses_tc = args.deposit_kernel in ("auto", "tensor")
    g = api.geom(lc.geom.nx, lc.geom.ny, lc.geom.theta0_x, lc.geom.theta0_y, lc.geom.dtheta)

    host = {k: torch.from_numpy(v).pin_memory() for k, v in lc.parts.items()}
    hM = torch.from_numpy(cat.M).pin_memory()
    hc = torch.from_numpy(cat.c).pin_memory()
    hz = torch.from_numpy(cat.z).pin_memory()
    hpos = torch.from_numpy(cat.pos).pin_memory()
    hthx = torch.from_numpy(cat.thx).pin_memory()
    hthy = torch.from_numpy(cat.thy).pin_memory()
    hv = torch.from_numpy(cat.vlos).pin_memory()
    h_in = list(host.values()) + [hM, hc, hz, hpos, hthx, hthy, hv]
    d_in = [t.to(dev) for t in h_in]
    parts_d = dict(zip(host.keys(), d_in[:len(host)]))
    M, c, z, pos, thx, thy, vl = d_in[len(host):]
    rec = torch.empty((n, api.ASSIGNED_STRIDE), dtype=torch.float32, device=dev)
    pp = api.Maps.zeros(g, dev)
    hp = api.Maps.zeros(g, dev)
    out_host = [torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory() for _ in range(4)]
    h2d_bytes = sum(t.numel() * t.element_size() for t in h_in)
    d2h_bytes = sum(t.numel() * t.element_size() for t in out_host)

    def step(ins=None, maps=None):
        """One pass of the hot path; ins: the device inputs (default the resident set),
        maps: the (PP, HP) maps to fill (default pp, hp)."""
        ins = d_in if ins is None else ins
        mpp, mhp = (pp, hp) if maps is None else maps
        parts = dict(zip(host.keys(), ins[:len(host)]))
        hM_, hc_, hz_, hpos_, hthx_, hthy_, hv_ = ins[len(host):]
        mpp.zero_()
        mhp.zero_()
        model, status = ctx.solve_halos(hM_, hc_, hz_)
        solved = torch.cuda.Event()
        solved.record(comp)

        def halo_paste():
            with torch.cuda.stream(hp_stream):
                hp_stream.wait_event(solved)
                ctx_hp.paste_halos(hthx_, hthy_, hv_, model, status, g, mhp)
                ctx_hp.finalize(g, mhp)
                done = torch.cuda.Event()
                done.record(hp_stream)
                return done

        fut = hp_pool.submit(halo_paste)
        ctx.assign_particles(parts, lc.Mp, hpos_, model, status, g, out=rec)
        ctx.paste_particles(rec, g, mpp)
        ctx.finalize(g, mpp)
        comp.wait_event(fut.result())  # the maps and the model are released after both

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flops, updates = deposit_flops(rec.cpu().numpy(), g.nx, g.ny)
    tile_pairs = int(ctx.pp_pairs(rec, g, 64)[0].numel())
    ctx.set_timing(True)
    ctx_hp.set_timing(True)
    ctx.phase_times()
    ctx_hp.phase_times()

    sampler = ClockSampler(local)
    barrier()
    if rank == 0:
        sampler.start()
    launches0 = ctx.kernel_launches() + ctx_hp.kernel_launches()
    step_ms, dep_ms, phases = [], [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        ph = ctx.phase_times()  # synchronises the stream
        ph_hp = ctx_hp.phase_times()  # elapsed on the second stream (overlapped, with waits)
        ph["hp_stream_total"] = sum(ph_hp.values())
        step_ms.append(e0.elapsed_time(e1))
        dep_ms.append(ph["deposit"])
        phases.append(ph)
    barrier()
    launches = ctx.kernel_launches() + ctx_hp.kernel_launches() - launches0
    clocks = sampler.stop() if rank == 0 else None
    ctx_hp.set_timing(False)
    # the HP phases timed alone (solve, then the halo paste on one stream) for their own
    # breakdown and the halos/s figure; in the step they overlap the particle chain
    hp_alone_ms, hp_phases = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        model_a, status_a = ctx.solve_halos(M, c, z)
        ctx.paste_halos(thx, thy, vl, model_a, status_a, g, hp)
        e1.record()
        hp_phases.append(ctx.phase_times())
        hp_alone_ms.append(e0.elapsed_time(e1))
    ctx.set_timing(False)
    t_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)

    # end to end through the public API: inputs from pinned host memory, maps back
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

    # the same, pipelined as a production loop runs it: an upload stream copies step k + 1's
    # inputs and a download stream reads step k - 1's maps back while step k computes (inputs
    # and result maps double-buffered); every step's uploads, L2 flush, compute and downloads
    # lie inside the timed region, which runs from the first upload to the last download
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ins2 = [d_in, [torch.empty_like(t) for t in d_in]]
    maps2 = [(pp, hp), (api.Maps.zeros(g, dev), api.Maps.zeros(g, dev))]
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

    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(up)
    upload(0)
    for k in range(args.steps):
        b = k % 2
        if k + 1 < args.steps:
            upload(k + 1)  # queued before step k's host-synchronising calls
        comp.wait_event(in_ready[k])
        if k >= 2:
            comp.wait_event(drained[k - 2])  # those maps have been read back
        flush.fill_(float(k))
        step(ins2[b], maps2[b])
        done[k].record(comp)
        with torch.cuda.stream(down):
            down.wait_event(done[k])
            m_pp, m_hp = maps2[b]
            for hdst, dsrc in zip(outs2[b], (m_pp.y[0], m_pp.b[0], m_hp.y[0], m_hp.b[0])):
                hdst.copy_(dsrc, non_blocking=True)
            drained[k].record(down)
    down.wait_event(drained[args.steps - 1])
    t1.record(down)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(t0.elapsed_time(t1) / args.steps, world, dev)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    mean_ph = {k: round(sum(p[k] for p in phases) / len(phases), 4) for k in phases[0]}
    for key in ("hp_table", "hp_pairs", "hp_paste"):
        mean_ph[key] = round(sum(p[key] for p in hp_phases) / len(hp_phases), 4)
    dep = sum(dep_ms) / len(dep_ms)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    achieved = flops / (dep * 1e-3) / 1e12
    if uses_tc:
        # TF32 dense peak: the measured cuBLAS bf16 burst x the nominal TF32 / BF16 ratio
        tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * (1.1 / 2.25)
        # MMA work the kernel issues: per (tile, particle) pair a 128 x 64 rank-1 update
        # in three split-TF32 products
        mma_flops = tile_pairs * 128 * 64 * 2 * 3
        roofline = {"kernel": "k_deposit_tc", "bound": "tensor", "achieved": achieved,
                    "peak": tf32_peak, "unit": "TFLOP/s", "frac": achieved / tf32_peak,
                    "traffic": ncu_traffic("k_deposit_tc_c1"), "deposit_ms": dep,
                    "algorithmic_flops_per_launch": flops, "pixel_updates": updates,
                    "tile_pairs": tile_pairs, "mma_flops_issued_per_launch": mma_flops,
                    "mma_tflops_issued": mma_flops / (dep * 1e-3) / 1e12,
                    "frac_fp32_alu_peak": achieved / fp32_peak,
                    "peak_note": "of measured: bf16 burst 1901.5 TFLOP/s x 1.1/2.25 (nominal "
                                 "TF32/BF16 dense ratio)"}
    else:
        roofline = {"kernel": "k_deposit<64>", "bound": "alu", "achieved": achieved,
                    "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                    "traffic": ncu_traffic("k_deposit_c1"), "deposit_ms": dep,
                    "algorithmic_flops_per_launch": flops, "pixel_updates": updates,
                    "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"}
    hp_ms = sum(hp_alone_ms) / len(hp_alone_ms)
    res = {
        "metric": METRIC, "value": job_rate(n, world, t_step), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": n, "halos": nh,
                   "maps": f"{g.nx}x{g.ny}", "pp_tile": 64,
                   "deposit_kernel": "tcgen05 split-TF32" if uses_tc else "SIMT FP32",
                   "l2": "flushed: 256 MB write "
                   "between timed steps", "parallelism": f"replicas x{world} (weak)"},
        "hp_halos_per_s": nh / (hp_ms * 1e-3) if hp_ms > 0 else None,
        "phase_hbm": phase_bandwidth(mean_ph, n, tile_pairs, g.nx, g.ny,
                                     float(peaks.get("hbm_gbs", 6785.9))),
        "phase_ms": mean_ph,
        "phase_note": "solve .. finalize: the particle chain on the main stream; hp_*: the "
                      "halo paste timed alone (in the step it runs on a second stream beside "
                      "the particle chain, hp_stream_total = its elapsed time there)",
        "roofline": roofline,
        "e2e": {"value": job_rate(n, world, t_e2e), "unit": UNIT,
                "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
                "ms_per_step": t_e2e, "pipelined": "copies of steps k +- 1 overlap step k",
                "serial_ms_per_step": t_e2e_serial,
                "serial_value": job_rate(n, world, t_e2e_serial)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_surrogate:
        res["surrogate"] = surrogate_section(api, ctx, dev, lc, args)
    if not args.no_hsml:
        res["smoothing_lengths"] = hsml_section(api, ctx, dev, lc, args)
    if not args.no_spectrum:
        res["power_spectrum"] = spectrum_section(api, ctx, dev, pp.y[0], g.dtheta)
    if not args.no_batched:
        res["batched_hp"] = batched_section(api, ctx, dev, args)
    if not args.no_allsky:
        res["allsky_hp"] = allsky_section(api, ctx, dev, args)
    if not args.no_full_scale:
        res["pp_full_scale"] = full_scale_section(api, ctx, dev, args, fp32_peak)
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        t_full, det = oracle_sample(lc, args.ref_particles, args.ref_halos, threads)
        res["cpu_baseline"] = {
            "value": n / t_full, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"FP64 oracle: solve of all {nh} halos, assign+deposit of "
                       f"{det['n_part_sample']} particles, HP of {det['n_halo_sample']} "
                       f"halos, extrapolated linearly to the full step"), "detail": det}
        if "smoothing_lengths" in res:  # the oracle's smoothing lengths at 8 particles
            import oracle as O

            idx = np.arange(0, n, n // 8)[:8]
            t0 = time.perf_counter()
            O.smoothing_lengths_at(lc.parts["x"], lc.parts["y"], lc.parts["z"], idx, 64.0,
                                   nthreads=threads)
            dt = time.perf_counter() - t0
            res["smoothing_lengths"]["cpu_oracle"] = {
                "particles_per_s": idx.size / dt, "sample": f"{idx.size} particles of the {n}",
                "cores": threads, "kind": "oracle"}
    print(json.dumps(res))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=4_000_000)
    ap.add_argument("--ref-particles", type=int, default=1_000_000)
    ap.add_argument("--ref-halos", type=int, default=600)
    ap.add_argument("--deposit-kernel", default="auto", choices=["auto", "simt", "tensor"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-hsml", action="store_true")
    ap.add_argument("--no-allsky", action="store_true")
    ap.add_argument("--no-spectrum", action="store_true")
    ap.add_argument("--allsky-halos", type=int, default=41_000_000)
    ap.add_argument("--allsky-nside", type=int, default=8192)
    ap.add_argument("--no-full-scale", action="store_true")
    ap.add_argument("--full-particles", type=int, default=500_000_000)
    ap.add_argument("--full-halos", type=int, default=200_000)
    ap.add_argument("--full-steps", type=int, default=3)
    ap.add_argument("--batch-maps", type=int, default=108)
    ap.add_argument("--batch-halos", type=float, default=5e4)
    ap.add_argument("--batch-npix", type=int, default=2048)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--sur-train", type=int, default=2_000_000)
    ap.add_argument("--sur-infer", type=int, default=10_000_000)
    ap.add_argument("--sur-epochs", type=int, default=6)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
