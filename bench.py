"""Benchmark: voxel Monte Carlo photon migration on the 256^3 spinodal mask.

One step = one pass of the whole hot path over one batch: reset the tallies,
transport 1e8 photons through the resident bit-packed mask (full Q32.32 voxel
fluence tally), FP64 normalisation and estimators on the GPU, results to the
host.  Workload: 256^3 Cahn-Hilliard spinodal mask (4000 steps, mask seed 0),
porosity 0.90, solid mu_s h = 0.5, mu_a h = 0.005, HG g = 0.7, FP32 transport.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VOX = 256
POROSITY = 0.90
CH_STEPS = 4000
MUS, MUA, G = 0.5, 0.005, 0.7
SEED = 20260809
PHOTONS = 100_000_000
METRIC = "photons/s & voxel-steps/s at 256³ φ=0.9"
WORKLOAD = ("256^3 Cahn-Hilliard spinodal mask (dt 0.1, 4000 steps, seed 0), porosity 0.90; "
            "solid mu_s h 0.5, mu_a h 0.005, HG g 0.7; pores void; periodic x/y; "
            "1e8 photons per step; FP32 transport; Q32.32 voxel fluence field")
# Algorithmic lane-operations per unit of work: the method's own operations
# (Sec. 2.5 transport step, interaction and photon life cycle), not the
# compiled code's, term by term:
#   any voxel step   26 = next face 4 (two compares, two selects), segment 1,
#                    path cap 2, deposit 6 (multiply, quantise 2, address 2,
#                    RED 1), path 1, crossing 9 (face parameter 1, index 2,
#                    wrap 2, brick and bit address 4), phase bit 2, pore path 1
#   solid step      +11 = optical depth 3 (multiply, compare, subtract) and
#                    Beer-Lambert 8 (mu_a l, 1 - e^-x as a quartic 4, dA,
#                    A += dA, w -= dA)  -> 37 in total
#   interaction    130 = Philox4x32-10 40 (10 rounds x 2 wide multiplies and
#                    2 three-way XORs), 4 uniforms 12, roulette 2, HG 7,
#                    azimuth 3, sin theta 3, rotation 25, renormalise 8,
#                    new optical depth 2, ray set-up 15, position in voxel 12
#   photon         100 = launch (Philox 40, uniforms 12, position 6, optical
#                    depth 2, state 15, brick 6, claim 3) and exit tallies 16
OPS_STEP, OPS_SOLID_EXTRA, OPS_INTERACT, OPS_PHOTON = 26, 11, 130, 100
# special-function (SFU / XU pipe) operations per unit: interaction 10 (HG
# reciprocal, sine and cosine, square root, two reciprocal square roots,
# logarithm, three reciprocals), photon 1 (logarithm); none per step (the
# Beer-Lambert factor is a polynomial)
SFU_INTERACT, SFU_PHOTON = 10, 1
ISSUE_PER_SM_CLK = 4          # warp instructions per SM per clock (4 schedulers)
SFU_PER_SM_CLK = 16           # XU lane-operations per SM per clock
# DRAM bytes (read + write) per photon of the transport kernel from one ncu capture
# (a 2e6-photon launch of this workload: 3.593e9 B read + 2.897e10 B written),
# valid only for the kernel source it was taken on.
TRAFFIC_CAPTURE = {"kernel_sha256_prefix": "3e0680a07320195d", "dram_bytes_per_photon": 16283.4,
                   "source": "profiles/transport_kernel_256cubed_phi090.md"}
# Hardware fractions of peak of the transport kernel from the same ncu capture
# (smsp__issue_active, sm__inst_executed_pipe_xu, lts__d_atomic_input_cycles_active),
# reported only while the kernel source matches the capture.
NCU_FRACTIONS = {"kernel_sha256_prefix": "3e0680a07320195d", "issue_slots": 0.5831,
                 "sfu_xu_pipe": 0.0164, "l2_atomic_unit": 0.1924, "warps_active": 0.3668,
                 "l2_red_hit_rate": 0.6543, "registers_per_thread": 72,
                 "source": "profiles/transport_kernel_256cubed_phi090.md"}


def _kernel_sha_prefix():
    """Hash of the transport kernel sources (generic template and FP32 kernel)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("spmc_transport.cuh", "spmc_transport_f32.cuh"):
        with open(os.path.join(ROOT, "paper_2604_13929_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons in the background."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=5)
            self.thread.join(timeout=2)

    def summary(self):
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            if len(r) >= 8:
                for n, v in zip(names, r[4:8]):
                    if v.lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_masks(device):
    """The 256^3 Cahn-Hilliard field (4000 steps, seed 0) thresholded at the
    headline porosity 0.90 and at 0.70 (the same field, as the paper's pair)."""
    from paper_2604_13929_gb300 import inputs
    c = inputs.cahn_hilliard((N_VOX,) * 3, CH_STEPS, seed=0, device=device)
    m90 = inputs.rank_threshold(c, POROSITY)
    m70 = inputs.rank_threshold(c, 0.70)
    del c
    return m90, m70


def make_mask(device):
    return make_masks(device)[0]


def profile_mode(spmc, torch, stream, mask, photons):
    """The headline workload in the depth-profile tally mode (per-phase depth
    bins staged in shared memory instead of the 134 MB voxel field): every
    estimator of the bench line except the voxel field itself."""
    sim = spmc.Simulation(mask, MUS, MUA, G, tally_field=0)
    sim.run(photons // 10, SEED + 1, stream)
    sim.reset(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.run(photons, SEED, stream)
    e1.record(stream)
    t = sim.tallies(stream)
    sim.close()
    sec = e0.elapsed_time(e1) / 1e3
    return {"photons": photons, "photons_per_s": photons / sec, "voxel_steps_per_s": t["steps"] / sec,
            **{k: t[k] for k in ("R", "T", "A", "phi_3d", "r", "ratio")}}


def other_workloads(spmc, torch, stream, m70, photons):
    """256^3 phi = 0.70 (same Cahn-Hilliard field) and homogeneous 256^3 slabs
    at the optics matched to phi = 0.90 and 0.70 (mu h (1 - phi), Eq.
    EMA_scaling): photons/s, voxel-steps/s and the estimators, one warm-up and
    one timed launch each, full Q32.32 field as in the headline."""
    from paper_2604_13929_gb300 import inputs
    slab = inputs.all_solid(N_VOX, N_VOX, N_VOX)
    cases = [("spinodal_phi0.70", m70, MUS, MUA),
             ("slab_matched_phi0.90", slab, MUS * (1 - POROSITY), MUA * (1 - POROSITY)),
             ("slab_matched_phi0.70", slab, MUS * 0.30, MUA * 0.30)]
    out = {}
    for name, mask, mus, mua in cases:
        sim = spmc.Simulation(mask, mus, mua, G)
        sim.run(photons // 10, SEED + 1, stream)
        sim.reset(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(photons, SEED, stream)
        e1.record(stream)
        t = sim.tallies(stream)
        sim.close()
        sec = e0.elapsed_time(e1) / 1e3
        out[name] = {"mu_s_h": mus, "mu_a_h": mua, "photons": photons,
                     "photons_per_s": photons / sec, "voxel_steps_per_s": t["steps"] / sec,
                     "steps_per_photon": t["steps"] / photons,
                     **{k: t[k] for k in ("R", "T", "A", "R_se", "T_se", "A_se", "closure", "phi_3d",
                                          "phi_1d", "r", "ratio", "pore_path_mean", "porosity")}}
    return out


def cpu_baseline(mask, target_s=15.0):
    """The FP64 oracle, as it stands, on all host cores over a bounded sample."""
    from oracle import oracle as orc
    cores = os.cpu_count() or 1
    n = 2000
    while True:                      # calibrate on samples of at least ~1 s
        t0 = time.perf_counter()
        orc.run(mask, MUS, MUA, G, n, SEED, n_threads=cores, field=True)
        dt = time.perf_counter() - t0
        if dt > 1.0 or n >= 5_000_000:
            break
        n *= 4
    n = int(min(max(n * target_s / max(dt, 1e-3), 2000), 20_000_000))
    t0 = time.perf_counter()
    r = orc.run(mask, MUS, MUA, G, n, SEED, n_threads=cores, field=True)
    dt = time.perf_counter() - t0
    steps = r["counts"]["steps"]
    return {"value": n / dt, "unit": "photons/s", "cores": cores, "kind": "oracle",
            "sample": f"photon ids [0, {n}) of the same 256^3 phi=0.90 workload with the full "
                      f"voxel field, {dt:.1f} s wall on {cores} threads",
            "voxel_steps_per_s": steps / dt, "photons": n, "seconds": dt}


def reference_arm(args, rank):
    if rank != 0:
        return
    from paper_2604_13929_gb300 import inputs
    mask = make_mask(inputs.default_device())
    per_step = []
    base = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(mask, target_s=args.cpu_seconds)
        if i >= args.warmup:
            per_step.append(cb)
        base = cb
    value = statistics.median(c["value"] for c in per_step)
    ms = statistics.median(c["seconds"] * 1e3 for c in per_step)
    line = {"metric": METRIC, "value": value, "unit": "photons/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD.replace("1e8 photons per step",
                                                    f"{base['photons']} photons per step")
                       .replace("FP32 transport", "FP64 CPU oracle")},
            "voxel_steps_per_s": statistics.median(c["voxel_steps_per_s"] for c in per_step),
            "cpu_baseline": {"value": value, "unit": "photons/s", "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": value, "unit": "photons/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_bench(args, torch, dist, spmc, world, rank, local_rank, barrier):
    """64 masks of uneven size and optics, 1e7 photons each, one persistent
    launch per step (CUDA-graph replay), launch shape picked by the autotuner."""
    from paper_2604_13929_gb300 import inputs
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    problems = inputs.batch_workload(64, device="cuda")
    gen_s = time.perf_counter() - t0
    if args.profile_launch:
        # profiling case: the one-launch mode at its default shape, no graph, no
        # autotuning; one warm-up launch of N/10 photons per problem, then one of N
        n = args.profile_launch
        with spmc.Batch(problems, graph=0, batch_mode=0) as pb:
            pb.run([max(n // 10, 1)] * len(problems), SEED + 1, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pb.run([n] * len(problems), SEED, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            steps = sum(pb.tallies(i, stream)["steps"] for i in range(len(problems)))
        print(json.dumps({"profile_launch_photons_per_problem": n, "problems": len(problems),
                          "ms": e0.elapsed_time(e1), "steps": steps}), flush=True)
        return
    n_each = 10_000_000
    b = spmc.Batch(problems)
    # the autotuner times each candidate on a tenth of a step: large enough that
    # per-launch overheads weigh as they do in the timed steps
    tuned = b.autotune([n_each // 10] * len(problems), SEED + 7, stream)
    tuned_mode = int(b.get_option("batch_mode"))

    def timed(mode):
        b.set_option("batch_mode", mode)
        for _ in range(args.warmup):
            b.run([n_each] * len(problems), SEED + rank, stream)
        torch.cuda.synchronize()
        b.reset(stream)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local_rank) as clk_:
            e0.record(stream)
            for _ in range(args.steps):
                b.run([n_each] * len(problems), SEED + rank, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
        st = sum(b.tallies(i, stream)["steps"] for i in range(len(problems)))
        b.reset(stream)
        return e0.elapsed_time(e1), st, clk_

    # both strategies at the autotuned launch shape; the headline is the
    # tuned one, the one-launch number is reported beside it
    other = 1 - tuned_mode
    ms_o, _, _ = timed(other)
    ms, steps, clk = timed(tuned_mode)
    b.set_option("batch_mode", tuned_mode)
    photons = n_each * len(problems) * args.steps * world
    by_mode = {tuned_mode: photons / world / (ms / 1e3), other: photons / world / (ms_o / 1e3)}
    # the same problems one launch at a time (sp_mc_run per mask), for comparison
    sims = [spmc.Simulation(m, mus, mua, g) for (m, mus, mua, g) in problems]
    for sim in sims:
        sim.run(n_each // 10, SEED, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for sim in sims:
        sim.run(n_each, SEED + rank, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_rate = n_each * len(problems) / (e0.elapsed_time(e1) / 1e3)
    for sim in sims:
        sim.close()
    line = {"metric": "photons/s, batched (64 masks 64^3-256^3)", "value": photons / (ms / 1e3),
            "unit": "photons/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 Cahn-Hilliard masks (1000 FP32 steps) of sizes "
                                   "64^3..256^3, porosity U[0.5,0.95], mu_s h logU[0.1,2], "
                                   "mu_a h U[0.001,0.05], g U[0,0.9]; 1e7 photons each per step; "
                                   "one persistent launch per step, CUDA graph replay",
                       "launch": {k: b.get_option(k) for k in ("threads", "blocks", "compact", "batch_mode",
                                                               "kernel", "steps_per_pass")},
                       "autotune_photons_per_s": tuned, "mask_generation_s": gen_s},
            "voxel_steps_per_s": steps * world / (ms / 1e3),
            "one_launch_photons_per_s": by_mode[0], "per_problem_launches_photons_per_s": by_mode[1],
            "sequential_photons_per_s": seq_rate,
            "gpu_launches": 2 * args.steps, "clocks": clk.summary()}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def paper_comparison(torch, spmc):
    """MC at the paper's shell optics (Table tab:optics: g = 0, mu_s' = 20118,
    mu_a = 5159 m^-1, a_vox = 1.45 um), mirror lateral faces, n = 1, against
    the collimated diffusion approximation with EMA optics: fluence-weighted
    RMS_w (Eq. RMSw) for a homogeneous solid slab, the matched EMA slabs and
    256^3 spinodal masks at porosity 0.70 and 0.90 (Sec. 4.3, Table S1)."""
    from paper_2604_13929_gb300 import diffusion, inputs
    h, mus, mua, nz = 1.45e-6, 20118.0, 5159.0, 256
    L = nz * h
    out = {"optics": "g=0, mu_s'=20118/m, mu_a=5159/m, a_vox=1.45um, mirror x/y, n=1",
           "photons": 20_000_000, "cases": {}}

    def run(mask, mus_, mua_):
        sim = spmc.Simulation(mask, mus_, mua_, 0.0, voxel_h=h, lateral_bc=1)
        sim.run(out["photons"], SEED)
        t = sim.tallies()
        sim.close()
        return t

    def depth_profile(t, mask):
        # per-layer mean fluence from the exact per-bin sums (64 bins of 4 layers)
        return t["depth"][2]

    edges = np.arange(0, 65) * (nz // 64) * h
    slab = np.zeros((nz, 8, 8), np.uint8)
    cases = [("homogeneous solid", slab, mus, mua, 0.0)]
    for phi in (0.70, 0.90):
        cases.append((f"EMA slab phi={phi}", slab, diffusion.ema(mus, phi), diffusion.ema(mua, phi), phi))
        cases.append((f"spinodal 256^3 phi={phi}",
                      inputs.spinodal_mask(256, phi, 4000, seed=0, device="cuda"), mus, mua, phi))
    for name, mask, ms, ma, phi in cases:
        t = run(mask, ms, ma)
        da = diffusion.CollimatedDA(diffusion.ema(mua, phi), diffusion.ema(mus, phi), L, 1.0)
        prof_da = da.layer_means(edges)
        prof_mc = depth_profile(t, mask)
        out["cases"][name] = {
            "R": t["R"], "T": t["T"], "A": t["A"], "closure": t["closure"],
            "RMS_w": diffusion.rms_weighted(prof_mc, prof_da),
            "RMS_unweighted": diffusion.rms_unweighted(prof_mc, prof_da),
            "RMS_log": diffusion.rms_log(prof_mc, prof_da),
            "phi_3d": t["phi_3d"], "phi_1d": t["phi_1d"], "ratio": t["ratio"], "r": t["r"],
            "L_opt_MC1D_um": t["phi_1d"] * L * 1e6, "L_opt_DA_um": da.optical_length * 1e6}
    print(json.dumps(out), flush=True)


def precision_study(torch, spmc, args):
    """512^3 porosity-0.90 mask (Cahn-Hilliard, 4000 FP32 steps, seed 0): FP32
    transport at 1e9 photons; FP32 and FP64 transport on the same 1e6- and
    1e7-photon subsets; the FP64 CPU oracle on the 1e6 subset.  Per-result
    errors on identical photon streams, beside the 1e9-photon standard errors."""
    from oracle import oracle as orc
    from paper_2604_13929_gb300 import inputs
    t0 = time.perf_counter()
    c = inputs.cahn_hilliard((512,) * 3, 4000, seed=0, device="cuda", dtype=torch.float32)
    mask = inputs.rank_threshold(c, 0.90)
    del c
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    keys = ("R", "T", "A", "phi_3d", "phi_1d", "phi_pore", "r", "ratio", "pore_path_mean",
            "escape_weight")

    def gpu(n, precision):
        sim = spmc.Simulation(mask, MUS, MUA, G, precision=precision)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.run(n, SEED)
        e1.record()
        torch.cuda.synchronize()
        t = sim.tallies()
        t["_ms"] = e0.elapsed_time(e1)
        sim.close()
        return t

    n_sub, n_mid, n_big = 1_000_000, 10_000_000, args.precision_photons
    f32_sub, f64_sub = gpu(n_sub, 32), gpu(n_sub, 64)
    f32_mid, f64_mid = gpu(n_mid, 32), gpu(n_mid, 64)
    f32_big = gpu(n_big, 32)
    t0 = time.perf_counter()
    o = orc.normalise(orc.run(mask, MUS, MUA, G, n_sub, SEED, n_threads=os.cpu_count() or 1,
                              field=False))
    oracle_s = time.perf_counter() - t0

    def rel(a, b):
        return float(abs(a - b) / abs(b)) if b else float(abs(a - b))

    def prof_dev(a, b):
        da, db = np.asarray(a["depth"][:2]), np.asarray(b["depth"][:2])
        ok = np.isfinite(da) & np.isfinite(db) & (db > 0)
        return float(np.max(np.abs(da[ok] / db[ok] - 1)))

    table = {}
    for k in keys:
        table[k] = {"oracle_1e6": o[k],
                    "fp32_vs_oracle_1e6": rel(f32_sub[k], o[k]),
                    "fp64_vs_oracle_1e6": rel(f64_sub[k], o[k]),
                    "fp32_vs_fp64_1e7": rel(f32_mid[k], f64_mid[k]),
                    "fp32_1e9": f32_big[k]}
        if k in ("R", "T", "A"):
            table[k]["se_1e9"] = f32_big[k + "_se"]
            table[k]["se_1e6"] = o[k + "_se"]
    odepth = {"depth": o["depth"]}
    out = {"workload": "512^3 CH mask phi=0.90 (16 MiB bricks, 1 GiB Q32.32 field), mu_s h 0.5, "
                       "mu_a h 0.005, g 0.7", "mask_generation_s": gen_s,
           "photons": {"subset": n_sub, "mid": n_mid, "fp32_full": n_big},
           "ms": {"fp32_1e6": f32_sub["_ms"], "fp64_1e6": f64_sub["_ms"], "fp32_1e7": f32_mid["_ms"],
                  "fp64_1e7": f64_mid["_ms"], "fp32_full": f32_big["_ms"],
                  "oracle_1e6_s": oracle_s, "oracle_cores": os.cpu_count()},
           "fp32_photons_per_s": n_big / (f32_big["_ms"] / 1e3),
           "fp64_photons_per_s": n_mid / (f64_mid["_ms"] / 1e3),
           "steps_per_photon": f32_big["steps"] / n_big,
           "events_fp32_vs_oracle_1e6": {k: [f32_sub[k], o["counts"][kk]] for k, kk in
                                        (("interactions", "interactions"), ("exit_R", "exit_R"),
                                         ("exit_T", "exit_T"), ("rr_kill", "rr_kill"))},
           "events_fp64_vs_oracle_1e6": {k: [f64_sub[k], o["counts"][kk]] for k, kk in
                                        (("interactions", "interactions"), ("exit_R", "exit_R"),
                                         ("exit_T", "exit_T"), ("rr_kill", "rr_kill"))},
           "depth_profile_max_rel_dev": {"fp32_vs_oracle_1e6": prof_dev(f32_sub, odepth),
                                         "fp64_vs_oracle_1e6": prof_dev(f64_sub, odepth),
                                         "fp32_vs_fp64_1e7": prof_dev(f32_mid, f64_mid)},
           "closure_fp32_1e9": f32_big["closure"], "identity_residual_fp32_1e9":
               f32_big["identity_residual"], "status_fp32_1e9": f32_big["status"],
           "results": table}
    print(json.dumps(out), flush=True)


def surrogate_bench(torch, args):
    """The learned surrogate on 64^3 masks: Monte Carlo training fields from
    the transport engine, training, held-out profile error (Eq. RMSw) and
    fields per second against the Monte Carlo producing the same field."""
    from paper_2604_13929_gb300 import spnn, surrogate as sg
    c0, n, batch = 32, 64, args.surrogate_batch
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    t0 = time.perf_counter()
    train_set = sg.make_fields(args.surrogate_train, seed=1, photons=args.surrogate_photons, n=n)
    # held-out masks are judged against a Monte Carlo reference of many more
    # photons than a training field, so its own noise is negligible
    test_set = sg.make_fields(args.surrogate_test, seed=2, photons=args.surrogate_ref_photons, n=n)
    data_s = time.perf_counter() - t0
    net = spnn.UNet(c0, n, batch)
    net.set_params(spnn.init_params(c0, 7))
    log = []
    spnn.spnn_set_option("loss_fluence_weight", 1 if args.surrogate_loss == "fluence" else 0)
    try:
        losses, train_s = sg.train(net, train_set, args.surrogate_steps, batch,
                                   on_log=lambda st, l: log.append((st, l)))
    finally:
        spnn.spnn_set_option("loss_fluence_weight", 0)
    ev = sg.evaluate(net, test_set, batch)
    with Clocks(0) as clk:
        rate = sg.inference_rate(net, test_set, batch, reps=10)
    # algorithmic FLOPs of one field's forward: 2 x input voxels x ci x co x taps
    # per input voxel (27 for conv3, 1 for the stride-2 down, 8 for the up)
    fl = 0
    lv = {"e0": 0, "d1": 0, "e1": 1, "d2": 1, "e2": 2, "d3": 2, "b1": 3, "b2": 3, "u2": 3, "c2": 2,
          "u1": 2, "c1": 1, "u0": 1, "c0": 0}
    for name, kind, ci, co in spnn.layer_table(c0):
        v = (n >> lv[name[:2]]) ** 3
        fl += 2 * v * ci * co * {"conv3": 27, "down": 1, "up": 8}[kind]
    # Monte Carlo fields/s: the engine producing one 64^3 field at the
    # training photon count (1e7), from the training set's measured rate
    mc_photons_per_s = train_set.info["mc_photons_per_s"]
    mc_rate = mc_photons_per_s / args.surrogate_photons
    # Monte Carlo given the surrogate's time per field: its profile error on the held-out masks
    eq_photons = max(1000, int(mc_photons_per_s / rate["fields_per_s"]))
    eq_target, _ = sg.simulate(test_set.mask, test_set.optics, eq_photons, seed=sg.MC_SEED + 99)
    eq_rms = sg.profile_rms(sg.profiles(eq_target, test_set.mask), sg.profiles(test_set.target, test_set.mask))
    eq_d = (eq_target - test_set.target).double()
    achieved = fl * batch / (rate["ms_per_batch"] / 1e3) / 1e12
    line = {"metric": "surrogate fields/s (64^3 ln-fluence + per-phase depth profiles)",
            "value": rate["fields_per_s"], "unit": "fields/s", "n_gpus": 1, "steps": args.surrogate_steps,
            "warmup": 1, "ms_per_step": rate["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"3D U-Net c0={c0} (4 levels, 32-256 channels) on {n}^3 Cahn-Hilliard masks, "
                                   f"porosity U[0.5,0.95], mu_s h logU[0.1,2], mu_a h U[0.001,0.05], "
                                   f"g U[0,0.9]; {args.surrogate_train} training fields of "
                                   f"{args.surrogate_photons:.0e} photons, {args.surrogate_test} held-out masks "
                                   f"judged against {args.surrogate_ref_photons:.0e}-photon Monte Carlo; "
                                   f"batch {batch}",
                       "params": net.param_count, "loss": args.surrogate_loss},
            "mc_fields_per_s": mc_rate, "speedup_vs_mc": rate["fields_per_s"] / mc_rate,
            "heldout": ev,
            "equal_time_mc": {"photons": eq_photons, "rms_w_mean": float(np.nanmean(eq_rms)),
                              "rms_w_median": float(np.nanmedian(eq_rms)),
                              "voxel_ln_rmse": float(torch.sqrt((eq_d * eq_d).mean()).item()),
                              "voxel_rel_rmse": float(torch.sqrt(((torch.exp(eq_d) - 1) ** 2).mean()).item()),
                              "frac_voxels_without_track": float((eq_target <= np.log(2e-6)).double().mean().item())},
            "training": {"steps": args.surrogate_steps, "seconds": train_s,
                         "ms_per_step": 1e3 * train_s / args.surrogate_steps,
                         "tflops": 3 * fl * batch * args.surrogate_steps / train_s / 1e12,
                         "loss_first": float(losses[0]), "loss_last": float(np.mean(losses[-10:])),
                         "log": log[::max(1, len(log) // 12)]},
            "data_seconds": data_s, "mc_photons_per_s": mc_photons_per_s,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_tflops_sustained"],
                         "unit": "TFLOP/s", "frac": achieved / peaks["bf16_tflops_sustained"], "traffic": None,
                         "kernel": "spnn rows_kernel, all 20 forward layers", "flop_per_field": fl,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"},
            "gpu_launches": 22 * 10, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    net.close()


def surrogate_profile(torch, args):
    """Profiling case: the c0 = 32 U-Net at 64^3, one warm-up forward+backward
    (skipped with --surrogate-profile-cold), then one forward+backward at
    batch B on random masks and optics; prints the milliseconds."""
    from paper_2604_13929_gb300 import spnn
    c0, n, B = 32, 64, args.surrogate_profile
    net = spnn.UNet(c0, n, B)
    net.set_params(spnn.init_params(c0, 7))
    rng = np.random.default_rng(5)
    mask = torch.from_numpy((rng.random((B, n, n, n)) < 0.8).astype(np.uint8)).cuda()
    optics = torch.tensor(np.tile([[0.5, 0.005, 0.7]], (B, 1)), dtype=torch.float32).cuda()
    x = spnn.planes_empty(B, n, n, n, 16)
    spnn.spnn_pack_input(mask, optics, x)
    pred = torch.empty((B, n, n, n), dtype=torch.float32, device="cuda")
    target = torch.zeros_like(pred)

    def step():
        net.forward(x, pred)
        net.backward(target)

    if not args.surrogate_profile_cold:
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step()
    e1.record()
    torch.cuda.synchronize()
    spnn.spnn_status()
    print(json.dumps({"surrogate_profile_batch": B, "ms": e0.elapsed_time(e1)}), flush=True)
    net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--photons", type=int, default=PHOTONS)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the phi=0.70 and matched-slab throughput keys")
    ap.add_argument("--workload", default="c2", choices=["c2", "batch", "paper", "precision", "surrogate"],
                    help="c2: the 256^3 phi=0.90 headline; batch: 64 masks of uneven size "
                         "(64^3..256^3) and optics, 1e7 photons each, one launch per step")
    ap.add_argument("--precision-photons", type=int, default=1_000_000_000)
    ap.add_argument("--surrogate-train", type=int, default=8192)
    ap.add_argument("--surrogate-test", type=int, default=128)
    ap.add_argument("--surrogate-steps", type=int, default=3000)
    ap.add_argument("--surrogate-loss", default="mse", choices=["mse", "fluence"],
                    help="training loss: squared log-fluence error, or the same weighted by fluence")
    ap.add_argument("--surrogate-batch", type=int, default=256)
    ap.add_argument("--surrogate-photons", type=int, default=10_000_000)
    ap.add_argument("--surrogate-ref-photons", type=int, default=100_000_000,
                    help="photons per held-out reference field")
    ap.add_argument("--surrogate-profile", type=int, default=0, metavar="B",
                    help="profiling case: one surrogate forward+backward at batch B (64^3, c0 32)")
    ap.add_argument("--surrogate-profile-cold", action="store_true",
                    help="with --surrogate-profile: no warm-up step")
    ap.add_argument("--profile-launch", type=int, default=0, metavar="N",
                    help="profiling case: one warm-up launch of N/10 photons, then one timed "
                         "launch of N photons on the workload (per problem with --workload "
                         "batch); prints its time and exits")
    args = ap.parse_args()

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_2604_13929_gb300 import build as spbuild
    spbuild.build()
    from paper_2604_13929_gb300 import shard, spmc

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.workload == "batch":
        batch_bench(args, torch, dist, spmc, world, rank, local_rank, barrier)
        return
    if args.workload == "paper":
        if rank == 0:
            paper_comparison(torch, spmc)
        return
    if args.workload == "precision":
        if rank == 0:
            precision_study(torch, spmc, args)
        return
    if args.workload == "surrogate":
        if rank == 0:
            if args.surrogate_profile:
                surrogate_profile(torch, args)
            else:
                surrogate_bench(torch, args)
        return
    mask, mask70 = make_masks("cuda")
    stream = torch.cuda.current_stream()
    if args.profile_launch:
        prof = spmc.Simulation(mask, MUS, MUA, G)
        prof.run(max(args.profile_launch // 10, 1), SEED + 1, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prof.run(args.profile_launch, SEED, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = prof.tallies(stream)
        print(json.dumps({"profile_launch_photons": args.profile_launch,
                          "ms": e0.elapsed_time(e1), "steps": t["steps"],
                          "interactions": t["interactions"]}), flush=True)
        prof.close()
        return
    # ranks run disjoint photon-id ranges of one stream (same key), so their
    # integer tallies would sum to one larger run; no collective on the path
    seed = SEED
    first_pid, _ = shard.photon_range(rank, world, args.photons * world)
    sim = spmc.Simulation(mask, MUS, MUA, G, pid_offset=first_pid)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)

    def step(ev=None):
        sim.reset(stream)
        if ev is not None:
            ev[0].record(stream)
        sim.run(args.photons, seed, stream)
        if ev is not None:
            ev[1].record(stream)
        return sim.tallies(stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    barrier()

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        barrier()
        start.record(stream)
        for i in range(args.steps):
            flush.fill_(1)
            torch.cuda.nvtx.range_push("spmc_step")
            results.append(step(kev[i]))
            torch.cuda.nvtx.range_pop()
        stop.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms_total = start.elapsed_time(stop)
    kernel_ms = [a.elapsed_time(b) for a, b in kev]
    if world > 1:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    last = results[-1]
    steps_per_photon = last["steps"] / last["photons"]
    photons_total = args.photons * args.steps * world
    value = photons_total / (ms_total / 1e3)
    clocks = clk.summary()

    # roofline of the transport kernel: algorithmic lane-operations / issue peak
    launch_ms = statistics.mean(kernel_ms)
    ops = (OPS_STEP * last["steps"] + OPS_SOLID_EXTRA * last["solid_steps"]
           + OPS_INTERACT * last["interactions"] + OPS_PHOTON * last["launched"]) / 32.0
    sfu = SFU_INTERACT * last["interactions"] + SFU_PHOTON * last["launched"]
    props = torch.cuda.get_device_properties(local_rank)
    max_mhz = clocks["sm_max_mhz"] or 2070.0
    peak = props.multi_processor_count * ISSUE_PER_SM_CLK * max_mhz * 1e6
    sfu_peak = props.multi_processor_count * SFU_PER_SM_CLK * max_mhz * 1e6
    achieved = ops / (launch_ms / 1e3)
    sha = _kernel_sha_prefix()
    traffic = None
    if sha == TRAFFIC_CAPTURE["kernel_sha256_prefix"]:
        traffic = TRAFFIC_CAPTURE["dram_bytes_per_photon"] * args.photons
    variant = int(sim.get_option("kernel"))
    roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                "unit": "Gwarp-inst/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_note": "DRAM read+write bytes per launch, ncu capture scaled by the "
                                "photon count (null if the kernel source changed since)",
                "kernel": ("spmc::transport_f32_kernel<true,false>" if variant == 1
                           else "spmc::transport_kernel<float,true,false,false>"),
                "kernel_sha256_prefix": sha,
                "ops_per_unit": {"voxel_step": OPS_STEP, "solid_step_extra": OPS_SOLID_EXTRA,
                                 "interaction": OPS_INTERACT, "photon": OPS_PHOTON},
                "units_per_launch": {"voxel_steps": last["steps"], "solid_steps": last["solid_steps"],
                                     "interactions": last["interactions"], "photons": last["launched"]},
                "peak_source": f"{props.multi_processor_count} SMs x {ISSUE_PER_SM_CLK} "
                               f"warp-inst/clk x {max_mhz:.0f} MHz (max SM clock)",
                "launch_ms": launch_ms,
                "frac_at_measured_clock": (achieved / (peak * clocks["sm_mhz"] / max_mhz)
                                           if clocks["sm_mhz"] else None),
                "sfu": {"achieved_gops": sfu / (launch_ms / 1e3) / 1e9, "peak_gops": sfu_peak / 1e9,
                        "frac": sfu / (launch_ms / 1e3) / sfu_peak,
                        "peak_source": f"{props.multi_processor_count} SMs x {SFU_PER_SM_CLK} "
                                       f"XU lane-ops/clk x {max_mhz:.0f} MHz"},
                "ncu_fractions": (NCU_FRACTIONS if NCU_FRACTIONS
                                  and NCU_FRACTIONS.get("kernel_sha256_prefix") == sha else None)}

    # measured ceiling of the step pattern: straight rays through an all-pore
    # 256^3 volume, with and without one Q32.32 RED per step into a 256^3 field
    ceil_red = spmc.sp_mc_probe_step_ceiling(N_VOX, True)["steps_per_s"]
    ceil_nored = spmc.sp_mc_probe_step_ceiling(N_VOX, False)["steps_per_s"]
    ceil_fit = spmc.sp_mc_probe_step_ceiling(240, True)["steps_per_s"]
    roofline["step_ceiling"] = {
        "with_field_red_steps_per_s": ceil_red, "without_red_steps_per_s": ceil_nored,
        "with_field_red_240cubed_steps_per_s": ceil_fit,
        "frac_of_red_ceiling": value * steps_per_photon / ceil_red,
        "note": "sp_mc_probe_step_ceiling: the kernel's traversal and tally memory pattern "
                "with no physics; the 256^3 Q32.32 field (134 MB) is past the L2 knee, a 240^3 "
                "field (111 MB) is not"}

    # end to end through the C ABI with host buffers: upload + pack the host
    # mask, transport, normalise, copy the results back
    host_mask = np.ascontiguousarray(mask)
    e2e_times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = spmc.Simulation(host_mask, MUS, MUA, G, pid_offset=first_pid)
        s2.run(args.photons, seed, stream)
        s2.tallies(stream)
        s2.close()
        torch.cuda.synchronize()
        if i:                                   # first pass is a warm-up
            e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times) if e2e_times else float("nan")
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    line = {
        "metric": METRIC, "value": value, "unit": "photons/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "mask": "256x256x256", "porosity": POROSITY,
                   "photons_per_step": args.photons,
                   "parallelism": f"photon-id shards x{world} (no collective)",
                   "l2": "flushed between steps (256 MiB write)"},
        "voxel_steps_per_s": value * steps_per_photon,
        "steps_per_photon": steps_per_photon,
        "interactions_per_photon": last["interactions"] / last["photons"],
        "results": {k: last[k] for k in ("R", "T", "A", "closure", "phi_3d", "phi_1d",
                                         "phi_pore", "r", "ratio", "identity_residual",
                                         "pore_path_mean", "p_pore_gt_L")},
        "roofline": roofline,
        "e2e": {"value": args.photons * world / e2e_s, "unit": "photons/s",
                "h2d_bytes_per_step": int(host_mask.nbytes),
                "d2h_bytes_per_step": int(spmc.load().sp_mc_result_size())},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_other_workloads:
        line["other_workloads"] = other_workloads(spmc, torch, stream, mask70, args.photons)
        line["profile_mode"] = profile_mode(spmc, torch, stream, mask, args.photons)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mask.copy(), target_s=args.cpu_seconds)
        line["cpu_baseline"].pop("photons", None)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
