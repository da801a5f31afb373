#!/usr/bin/env python
"""Throughput of the 1D radiative PIC time step (push + QED + deposit +
Ampere, with the amortised store compaction) in macroparticle-steps/s.

Workload (one GPU): Nx = 2^20 periodic cells, 200 e- + 200 e+ per cell
(4.19e8 macroparticles), 1D Maxwell-Juttner theta = 0.1, 1e-3 Langmuir seed,
QED off: the roofline microbenchmark of the method.  The headline is the FP32
particle state with the FP64 field; the FP64 plain state is reported beside
it.  Inputs are resident in HBM and larger than L2 (no flush needed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own independent replica (weak scaling,
no collective on the data path); the timed region is bracketed by barriers
and the maximum over ranks is reported.  `--impl reference` times the FP64
CPU oracle of the same method on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "macroparticle-steps/s (push+QED+deposit)"
UNIT = "macroparticle-steps/s"
NX, PPC = 1 << 20, 200
WORKLOAD = dict(nx=NX, ppc=PPC, dx=0.1, dt=0.045, theta=0.1, seed_amp=1e-3, density=1.0,
                init=2, boundary=1, qed=0)
N_PARTICLES = 2 * NX * PPC


def set_size(nx):
    """Smaller copies of the workload (same density and temperature) serve
    profiling captures; the bench line is always the full size."""
    global NX, N_PARTICLES
    NX = nx
    WORKLOAD["nx"] = nx
    N_PARTICLES = 2 * NX * PPC
WORKLOAD_NAME = ("cfg2 push+deposit roofline: Nx=2^20 periodic, 4.19e8 e+- (200+200 per cell, "
                 "0.5 n_co each), Maxwell-Juttner theta=0.1, 1e-3 Langmuir seed, QED off")
SETUP = {"filter_passes": 0, "inject_theta": 0.0, "qed_quantum": 0, "em": 0, "beta_y": 0.0}  # off for the headline
BETA_ROT = 3e-6  # the co-rotating frame's velocity in Sect. 6.1
PML_CELLS = 16   # absorbing layer below the top of the batch's surface gaps


def set_setup(filter_passes, inject_theta, qed_quantum=0, em=0):
    """Sect. 6.1's binomial current filter and hot atmosphere, the quantum
    photon spectrum, and the transverse fields of the co-rotating frame
    (App. A), applied to the workloads (the atmosphere and the spectrum only
    matter for the QED surface gaps of the batch; the absorbing layer only
    for surface gaps)."""
    global WORKLOAD_NAME, BATCH_NAME
    SETUP.update(filter_passes=filter_passes, inject_theta=inject_theta, qed_quantum=qed_quantum,
                 em=1 if em else 0, beta_y=BETA_ROT if em else 0.0)
    if em:
        WORKLOAD.update(em=1, beta_y=BETA_ROT)
        WORKLOAD_NAME += f", transverse fields of the co-rotating frame (beta={BETA_ROT:g})"
        BATCH_NAME += f", transverse fields (beta={BETA_ROT:g}, {PML_CELLS}-cell absorbing layer)"
    if qed_quantum:
        BATCH_NAME += ", quantum photon spectrum"
    if filter_passes:
        WORKLOAD["filter_passes"] = filter_passes
        WORKLOAD_NAME += f", {filter_passes}-pass binomial current filter"
        BATCH_NAME += f", {filter_passes}-pass binomial current filter"
    if inject_theta:
        BATCH_NAME += f", atmosphere T={inject_theta:g} m_e c^2"


# algorithmic bytes of the push kernel per particle-step (no QED, uniform
# weights): read cell int32 + offset + momentum, write them back
BYTES_PER_PARTICLE = {"fp32": 24, "fp64": 40}


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# the source text of each recorded kernel: from the template line above its
# signature to the next separator line
TRAFFIC_KERNELS = {"k_push": "k_push_lean(View v)", "k_push_qed": "k_push(View v)"}


def kernel_sha(kernel):
    src = open(os.path.join(ROOT, "paper_2608_21920_b300", "csrc", "step.cu")).read()
    i = src.index(TRAFFIC_KERNELS[kernel])
    i = src.rfind("template", 0, i)
    j = src.index("// -----------", i)
    return hashlib.sha256(src[i:j].encode()).hexdigest()[:16]


def traffic_record(kernel, precision, units=None):
    """DRAM traffic per launch of a push kernel from a committed ncu summary,
    valid only while the kernel's source text is unchanged; with `units`
    (leptons per launch), the recorded bytes per lepton times the units."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[f"{kernel}:{precision}"]
    except Exception:
        return None
    if rec.get("step_cu_sha") != kernel_sha(kernel):
        return None
    if units is not None:
        return rec.get("bytes_per_lepton") * units
    return rec.get("bytes_per_launch")


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's time (every rank gets it); x alone without a
    process group."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(units_per_rank, steps, ms_max, world):
    """Whole-job rate of independent replicas (weak scaling): the units
    all ranks processed over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2608_21920_b300 import Gap
    from paper_2608_21920_b300 import _abi as A

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def rank_max(x):
        return max_over_ranks(x, dist if world > 1 else None, "cuda")

    peaks, peak_kind = measured_peaks()
    cfg = dict(WORKLOAD, seed=rank, gap_index=rank)
    results = {}
    tuned = None
    if args.autotune:
        from paper_2608_21920_b300 import autotune
        (args.tile, args.threads, args.variant), times = autotune.tune(cfg, "fp32", verbose=(rank == 0))
        tuned = {f"{t}x{th}v{vv}": round(ms, 4) for (t, th, vv), ms in times.items()}
    for precision in (["fp32", "fp64"] if not args.fp32_only else ["fp32"]):
        K = args.steps if precision == "fp32" else max(3, min(args.steps, args.fp64_steps))
        g = Gap(cfg, precision=precision, tile=args.tile, threads=args.threads,
                variant=args.variant if precision == "fp32" else 0, rebin_every=args.rebin_every)
        g.step(args.warmup)
        barrier()
        clocks = ClockSampler(local)
        if precision == "fp32":
            clocks.start()
        g.profile(True)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(s)
        g.step(K)
        e1.record(s)
        barrier()
        ms = e0.elapsed_time(e1)
        push_ms, push_n, lps = g.profile(False)
        clk = clocks.stop() if precision == "fp32" else None
        ms = rank_max(ms)
        d = g.diag(spectrum=False)
        r = dict(ms=ms, K=K, push_ms=push_ms / max(push_n, 1), push_n=push_n, launches=lps * K,
                 gauss=d["gauss_residual"], E_abs_max=d["E_abs_max"],
                 n=d["n_electrons"] + d["n_positrons"], clocks=clk)
        if precision == "fp32" and args.steady_steps > 0:
            # after the timed window: enough steps that compactions and the
            # drifted store order are inside (the store is compacted every
            # rebin_every steps)
            g.profile(True)
            barrier()
            e0.record(s)
            g.step(args.steady_steps)
            e1.record(s)
            barrier()
            sms = rank_max(e0.elapsed_time(e1))
            sp_ms, sp_n, _ = g.profile(False)
            r["steady"] = dict(steps=args.steady_steps, ms_per_step=sms / args.steady_steps,
                               push_ms_per_launch=sp_ms / max(sp_n, 1),
                               value=job_throughput(N_PARTICLES, args.steady_steps, sms, world))
        if precision == "fp32" and world == 1 and not args.no_cpu and not (SETUP["filter_passes"] or SETUP["em"]):
            r["error_vs_oracle"] = oracle_window_error(g, args.tile or 256)
        results[precision] = r
        if precision == "fp32" and not args.no_e2e:
            # end to end through the public API: init from host parameters,
            # then every step the result (E) read back to pinned host memory,
            # the transfer on a second stream overlapping the next step
            del g
            torch.cuda.empty_cache()
            Ehost = torch.empty(NX, dtype=torch.float64, pin_memory=True)
            copy = torch.cuda.Stream()
            Ke = args.e2e_steps or args.steps  # the timed steps of the headline, end to end
            barrier()
            t0 = time.perf_counter()
            g = Gap(cfg, precision=precision, tile=args.tile, threads=args.threads, variant=args.variant,
                    rebin_every=args.rebin_every)
            torch.cuda.synchronize()
            t_init = time.perf_counter() - t0
            for _ in range(Ke):
                g.step(1)
                g.field_async(Ehost, copy)
            copy.synchronize()
            torch.cuda.synchronize()
            barrier()
            t_e2e = rank_max(time.perf_counter() - t0)
            # host->device bytes of gap_init: gap and tile tables, tile-edge
            # counts, segment layout, spectrum tables (the plasma is loaded on
            # the device from the parameters); device->host per step: E and
            # the control block that locates it
            tile = args.tile or 256
            nt = (NX + tile - 1) // tile
            h2d_init = 256 + 16 * nt + NX + 2 * 12 * nt + 1024 * 8 + 2 * 577 * 8
            r["e2e"] = dict(value=world * N_PARTICLES * Ke / t_e2e, steps=Ke, init_s=rank_max(t_init),
                            h2d_bytes_per_step=int(math.ceil(h2d_init / Ke)),
                            d2h_bytes_per_step=int(NX * 8))
        del g
        torch.cuda.empty_cache()
    qr = None
    if not args.no_qed:  # the QED leg: the batch of surface gaps in discharge, every rank its own replica
        qa = argparse.Namespace(**vars(args))
        qa.steps, qa.tile, qa.variant = 50, 128, 0
        qr = batch_measure(qa, world, local)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    r32 = results["fp32"]
    value = job_throughput(N_PARTICLES, r32["K"], r32["ms"], world)
    bpp = BYTES_PER_PARTICLE["fp32"]
    achieved = bpp * N_PARTICLES / (r32["push_ms"] / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    deferred = bool(SETUP["filter_passes"] or SETUP["em"])  # the push hands Ampere to k_filter_apply
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": r32["K"],
        "warmup": args.warmup, "ms_per_step": r32["ms"] / r32["K"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": "FP32 particle state, FP64 field",
                   "macroparticles_per_gpu": N_PARTICLES, "tile": args.tile or 256,
                   "l2": "inputs larger than L2 (11.7 GB particle state per GPU), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                     "kernel": ("k_push_lean (FP32, no QED, uniform weights)" if not deferred else
                                "k_push_lean (FP32, Ampere deferred) + k_flux_take + k_filter_apply"
                                + (" + k_em_cells + k_em_nodes" if SETUP["em"] else "")),
                     "bytes_per_particle": bpp, "push_ms_per_launch": r32["push_ms"],
                     "traffic": traffic_record("k_push", "fp32") if not deferred else None},
        "gpu_launches": int(r32["launches"]),
        "clocks": r32["clocks"],
        "gauss_residual": r32["gauss"], "E_abs_max": r32["E_abs_max"],
        "particles_alive": r32["n"],
    }
    if "steady" in r32:
        st = r32["steady"]
        a_st = bpp * N_PARTICLES / (st["push_ms_per_launch"] / 1e3) / 1e9
        line["steady_state"] = {"steps": st["steps"], "value": st["value"], "unit": UNIT,
                                "ms_per_step": st["ms_per_step"], "push_ms_per_launch": st["push_ms_per_launch"],
                                "achieved": a_st, "frac": a_st / peak,
                                "window": f"the {st['steps']} steps after the timed ones, compactions included"}
    if "error_vs_oracle" in r32:
        line["error_vs_oracle"] = r32["error_vs_oracle"]
    if tuned:
        line["config"]["autotune_ms_per_push"] = tuned
        line["config"]["threads"] = args.threads
        line["config"]["variant"] = args.variant
    line["config"]["rebin_every"] = args.rebin_every or 64
    if "e2e" in r32:
        e = r32["e2e"]
        line["e2e"] = {"value": e["value"], "unit": UNIT, "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e["d2h_bytes_per_step"], "steps": e["steps"], "init_s": e["init_s"],
                       "includes": "gap_init from host parameters + per-step E readback to pinned host "
                                   "(gap_get_field_async: the transfer overlaps the next step)"}
    if "fp64" in results:
        r64 = results["fp64"]
        v64 = job_throughput(N_PARTICLES, r64["K"], r64["ms"], world)
        a64 = BYTES_PER_PARTICLE["fp64"] * N_PARTICLES / (r64["push_ms"] / 1e3) / 1e9
        line["fp64_plain"] = {"value": v64, "unit": UNIT, "steps": r64["K"], "ms_per_step": r64["ms"] / r64["K"],
                              "achieved_gbs": a64, "frac": a64 / peak, "gauss_residual": r64["gauss"],
                              "bound": "fp64 alu (the FP64 pipe ~85 % busy in the push; profiles/k_push_fp64_cfg2.md)",
                              "fp32_over_fp64": value / v64}
    if qr is not None:
        line["qed"] = {"metric": METRIC, "value": qr["value"], "unit": UNIT, "steps": qr["steps"],
                       "ms_per_step": qr["ms_per_step"], "roofline": qr["roofline"], "clocks": qr["clocks"],
                       "gpu_launches": qr["gpu_launches"], "config": qr["config"],
                       "phases_ms_per_step": qr["phases_ms_per_step"], "phases_window": qr["phases_window"],
                       "counts": {k: qr[k] for k in ("pairs", "merged", "photons_merged", "emit_events")}}
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def oracle_window_error(g, tile, t_lo=1000, n_tiles=4):
    """Error of one FP32 step against the FP64 oracle at full size (outside
    the timed region; part of the baseline leg, the one place that runs the
    oracle): the leptons of n_tiles tiles and one tile of halo on each side
    are exported, pushed one step by the oracle from the GPU's state and E^n,
    and the oracle's E^{n+1} on the window's nodes and the leptons' new
    positions and momenta are compared with the GPU's step."""
    import numpy as np
    import oracle as O
    t_hi = t_lo + n_tiles
    E0 = g.field()
    lep = [g.tile_particles(kind, t_lo - 1, t_hi + 1) for kind in (0, 1)]
    g.step(1)
    E1 = g.field()
    after = [g.tile_particles(kind, t_lo - 2, t_hi + 2) for kind in (0, 1)]
    o = O.Sim(nx=NX, boundary=O.BC_PERIODIC, dx=WORKLOAD["dx"], dt=WORKLOAD["dt"], init=O.INIT_EMPTY,
              filter_passes=SETUP["filter_passes"], em=SETUP["em"], beta_y=SETUP["beta_y"])
    o.set_E(E0)
    for kind, q in ((0, -1), (1, 1)):
        L = lep[kind]
        for i in range(L["id"].size):
            o.add_lepton(int(L["id"][i]), q, float(L["X"][i]), float(L["u"][i]), float(L["w"][i]))
    o.step(1)
    Eo = o.E()
    nodes = np.arange(t_lo * tile, t_hi * tile + 1)
    dE = np.abs(Eo[nodes] - E0[nodes])
    err = np.abs(E1[nodes] - Eo[nodes])
    Lo = o.leptons()
    got = {k: np.concatenate([a[k] for a in after]) for k in ("id", "X", "u")}
    common, ia, ib = np.intersect1d(got["id"], Lo["id"], return_indices=True)
    dX = got["X"][ia] - Lo["X"][ib]
    dX -= NX * np.round(dX / NX)
    du = np.abs(got["u"][ia] - Lo["u"][ib]) / np.maximum(np.abs(Lo["u"][ib]), 1.0)
    return {"E_max_abs": float(err.max()), "E_max_rel_to_step_change": float(err.max() / np.median(dE)),
            "E_max_rel": float(err.max() / np.abs(Eo[nodes]).max()), "nodes": int(nodes.size),
            "X_max_abs_cells": float(np.abs(dX).max()), "u_max_rel": float(du.max()), "leptons": int(common.size),
            "method": f"one FP32 step from the GPU state against the FP64 oracle on tiles {t_lo}-{t_hi - 1} "
                      f"(+1 tile halo) of the full-size workload, after the timed steps"}


def _oracle_sample(nx, steps, warmup):
    import oracle as O
    s = O.Sim(nx=nx, ppc=PPC, dx=0.1, dt=0.045, theta=0.1, seed_amp=1e-3, density=1.0,
              init=O.INIT_PAIR_THERMAL, boundary=O.BC_PERIODIC, seed=0,
              filter_passes=SETUP["filter_passes"], em=SETUP["em"], beta_y=SETUP["beta_y"])
    if warmup:
        s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return 2 * nx * PPC * steps / dt, dt


def host_cpu():
    """CPU model and logical core count of the host (for the baseline record)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"cpu_model": model, "host_cores": os.cpu_count()}


def _oracle_replica(a):
    nx, steps = a
    rate, dt = _oracle_sample(nx, steps, 1)
    return 2 * nx * PPC * steps, dt


def cpu_baseline_parallel(nx, steps, procs):
    """The same oracle on `procs` host cores at once: independent replicas of
    the sample in separate processes (the oracle itself is single-threaded;
    the workload's gaps and samples are independent), aggregate
    macroparticle-steps over the slowest replica's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")  # this process already holds a CUDA context
    with ctx.Pool(procs) as pool:
        out = pool.map(_oracle_replica, [(nx, steps)] * procs)
    work = sum(o[0] for o in out)
    t = max(o[1] for o in out)
    return work / t, t


def cpu_baseline(seconds):
    """The FP64 oracle as it stands, single-threaded on the host, on a bounded
    sample of the workload (same density, temperature and seed; fewer cells)."""
    nx = 1 << 14
    rate, dt = _oracle_sample(nx, 2, 0)
    steps = max(2, int(seconds * rate / (2 * nx * PPC)))
    rate, dt = _oracle_sample(nx, steps, 1)
    rec = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"Nx=2^14 periodic, {2 * nx * PPC:.3g} e+- (200+200/cell), {steps} steps, {dt:.1f} s",
           **host_cpu()}
    procs = min(os.cpu_count() or 1, 16)
    if procs > 1:
        psteps = max(2, steps // 2)
        prate, pt = cpu_baseline_parallel(nx, psteps, procs)
        rec["parallel"] = {"value": prate, "unit": UNIT, "cores": procs, "kind": "oracle replicas",
                           "sample": f"{procs} processes, each the sample above for {psteps} steps, "
                                     f"slowest {pt:.1f} s"}
    return rec


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return
    total = (args.steps + args.warmup)
    nx = 1 << max(8, int(math.log2(max(256, 1.5e9 / (2 * PPC * max(total, 1))))))
    import oracle as O
    s = O.Sim(nx=nx, ppc=PPC, dx=0.1, dt=0.045, theta=0.1, seed_amp=1e-3, density=1.0,
              init=O.INIT_PAIR_THERMAL, boundary=O.BC_PERIODIC, seed=0,
              filter_passes=SETUP["filter_passes"], em=SETUP["em"], beta_y=SETUP["beta_y"])
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    value = 2 * nx * PPC * args.steps / dt
    sample = f"Nx={nx} periodic, {2 * nx * PPC:.3g} e+- (200+200/cell), theta=0.1, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "precision": "FP64 oracle (plain C, 1 thread)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH_NAME = ("cfg4 batch: {n} independent gaps, Nx~U[1024,8192], alpha~U[-1,3], b~logU[0.03,0.3], "
              "rho_c~logU[1e6,1e8] cm, 8-64 cold e-/cell, QED on, per-gap seeds 0..{last}, cap 16x initial")


def _total_leptons(g):
    n = 0
    for i in range(g.n_gaps):
        d = g.diag(i, spectrum=False)
        n += d["n_electrons"] + d["n_positrons"]
    return n


def batch_params(n_gaps, cap_per_cell=0):
    """The batch workload's gap parameters with the options of SETUP (the
    absorbing layer only on surface gaps); cap_per_cell > 0 sets each gap's
    cap to that many macro-particles per initial one (16 in the workload), for
    profiling the merge on a small slice."""
    from paper_2608_21920_b300 import workloads
    params = [dict(p, **SETUP) for p in workloads.batch(n_gaps)]
    if cap_per_cell > 0:
        for p in params:
            p["cap"] = int(cap_per_cell * p["nx"] * p["ppc"])
    if SETUP["em"]:
        for p in params:
            if p.get("boundary", 0) == 0:  # surface gap
                p["pml_cells"] = PML_CELLS
    return params


def batch_measure(args, world=1, local=0):
    """The batched parameter sweep: all gaps advance together, one launch per
    kernel per step, replayed from CUDA graphs of `--graph-chunk` steps; the
    QED push (FP32 state, emission, stored weights) timed on its own."""
    import torch
    from paper_2608_21920_b300 import Gap, autotune
    rank = rank_info()[0]
    params = batch_params(args.gaps, args.cap_per_cell)
    peaks, peak_kind = measured_peaks()
    tuned = None
    tile, threads, rebin = args.tile if args.tile != 256 else 128, args.threads, args.rebin_every or 64
    if args.autotune:
        (tile, threads, rebin), times = autotune.tune_step(params, "fp32", verbose=(rank == 0))
        tuned = {f"{t}x{th}r{rb}": round(ms, 4) for (t, th, rb), ms in times.items()}
    cap_kw = {}
    if args.capacity_factor > 0:  # smaller stores for profiling captures (a few GB)
        init = sum(p["nx"] * p["ppc"] for p in params)
        cap_kw = dict(lepton_capacity=int(args.capacity_factor * init),
                      photon_capacity=int(4 * args.capacity_factor * init // 3))
    g = Gap(params, precision="fp32", tile=tile, threads=threads, rebin_every=rebin, variant=args.variant,
            **cap_kw)
    s = torch.cuda.Stream()
    chunk = args.graph_chunk
    with torch.cuda.stream(s):
        g.step(args.batch_advance, graph_chunk=chunk)  # into the discharge (pairs present)
        g.step(args.warmup * chunk, graph_chunk=chunk)
    s.synchronize()
    n0 = _total_leptons(g)
    K = max(chunk, (args.steps // chunk) * chunk)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        e0.record(s)
        # NVTX ranges mark the timed steps and the eager ones below for launch lists
        torch.cuda.nvtx.range_push("batch_timed")
        g.step(K, graph_chunk=chunk)
        torch.cuda.nvtx.range_pop()
        e1.record(s)
    e1.synchronize()
    import torch.distributed as dist
    ms = max_over_ranks(e0.elapsed_time(e1), dist if world > 1 else None, "cuda")
    clk = clocks.stop()
    n1 = _total_leptons(g)
    # the push kernel alone and the step's phases, over as many eagerly
    # launched steps as were timed (the merge and the compactions are bursty)
    g.profile(True)
    Kp = K
    torch.cuda.nvtx.range_push("batch_eager")  # launch lists: ncu --nvtx --nvtx-include batch_eager/
    g.step(Kp)
    torch.cuda.nvtx.range_pop()
    phases, nph = g.profile_phases()
    push_ms, push_n, lps = g.profile(False)
    n2 = _total_leptons(g)
    push_ms /= max(push_n, 1)
    nmean = 0.5 * (n0 + n1)
    bpp = 36  # FP32 state with QED and stored weights: read k, phi, u, w, tau; write k, phi, u, tau
    achieved = bpp * 0.5 * (n1 + n2) / (push_ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6400.0))
    c = [g.diag(i, spectrum=False)["counters"] for i in range(g.n_gaps)]
    g.close()
    del g
    torch.cuda.empty_cache()
    res = {
        "value": world * nmean * K / (ms / 1e3), "steps": K, "warmup": args.warmup * chunk, "ms_per_step": ms / K,
        "config": {"workload": BATCH_NAME.format(n=args.gaps, last=args.gaps - 1).replace(
                       "cap 16x initial", f"cap {args.cap_per_cell:g}x initial" if args.cap_per_cell else "cap 16x initial"),
                   "gaps": args.gaps,
                   "capacity_factor": args.capacity_factor or None, "graph_chunk": chunk, "tile": tile,
                   "threads": threads, "rebin_every": rebin, "advanced_before_timing": args.batch_advance,
                   "leptons_mean": nmean, "l2": "inputs larger than L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": f"hbm_gbs of {peak_kind}", "kernel": "k_push (FP32, QED, stored weights)",
                     "bytes_per_particle": bpp, "push_ms_per_launch": push_ms,
                     "traffic": traffic_record("k_push_qed", "fp32", units=0.5 * (n1 + n2))},
        "gpu_launches": int(lps * K),
        "clocks": clk,
        "pairs": int(sum(x["pairs"] for x in c)), "merged": int(sum(x["merged"] for x in c)),
        "photons_merged": int(sum(x["photons_merged"] for x in c)),
        "emit_events": int(sum(x["emit_events"] for x in c)),
        "phases_ms_per_step": {k: v / max(nph, 1) for k, v in phases.items()},
        "phases_window": f"the {Kp} steps after the timed ones, eagerly launched between CUDA events",
    }
    if tuned:
        res["config"]["autotune_ms_per_step"] = tuned
    return res


def run_batch(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    r = batch_measure(args, world, local)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": r["steps"],
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    line.update({k: v for k, v in r.items() if k not in line})
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile", type=int, default=256)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--rebin-every", type=int, default=0, help="steps between sorted compactions (0: library default)")
    ap.add_argument("--fp64-steps", type=int, default=30)
    ap.add_argument("--steady-steps", type=int, default=192,
                    help="steps timed after the headline window, compactions included (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="steps of the end-to-end run (0: --steps)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--fp32-only", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-qed", action="store_true", help="leave out the QED batch sub-record")
    ap.add_argument("--autotune", action="store_true", help="pick tile and threads by timing the push kernel")
    ap.add_argument("--nx", type=int, default=0, help="smaller workload for profiling captures only")
    ap.add_argument("--workload", choices=["roofline", "batch"], default="roofline",
                    help="roofline: the Nx=2^20 push+deposit microbenchmark (the headline); "
                         "batch: the 256-gap QED sweep")
    ap.add_argument("--gaps", type=int, default=256)
    ap.add_argument("--cap-per-cell", type=float, default=0.0,
                    help="batch: each gap's cap in macro-particles per initial one (0: the workload's 16)")
    ap.add_argument("--graph-chunk", type=int, default=50)
    ap.add_argument("--batch-advance", type=int, default=1500)
    ap.add_argument("--capacity-factor", type=float, default=0.0,
                    help="batch: lepton store = factor x initial count (profiling captures only; 0: caps)")
    ap.add_argument("--filter-passes", type=int, default=0,
                    help="binomial current-filter passes per step (Sect. 6.1 uses 8; 0: off)")
    ap.add_argument("--inject-theta", type=float, default=0.0,
                    help="batch: temperature of the surface atmosphere (Sect. 6.1 uses 0.3; 0: cold)")
    ap.add_argument("--em", action="store_true",
                    help="transverse fields of the co-rotating frame (App. A) at beta 3e-6; surface gaps "
                         "get a 16-cell absorbing layer (default: off)")
    ap.add_argument("--qed-quantum", action="store_true",
                    help="batch: photon energies from the quantum spectrum (default: classical shape)")
    args = ap.parse_args()
    if args.nx:
        set_size(args.nx)
    set_setup(args.filter_passes, args.inject_theta, 1 if args.qed_quantum else 0, 1 if args.em else 0)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
