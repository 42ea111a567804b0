"""Benchmark: FCIQMC iterations at 1e7 walkers on one GB300 (spawn attempts/s).

Workload: the synthetic 28-orbital molecule (56 spin orbitals, 64-bit keys,
8 up + 7 down electrons, seeded integrals from paper_1811_11679_gb300.inputs),
heat-bath excitation generator, initiator rule (n_a = 3), real weights
(spawn_cutoff 0.1), tau = 0.01, target population 1e7, semi-stochastic core of
1e4 determinants chosen at iteration 2000 ("high" space).  The run grows on the
device from 500 walkers on the reference determinant; the timed steps start
after iteration 2000 + warm-up.  One step = one full FCIQMC iteration (every
phase on the GPU).  The walker and spawn arrays exceed the 129 MB L2, so no
flush is needed between steps.

Arms
  default           the CUDA engine through its C ABI (CUDA-graph launches)
  --impl reference  the CPU oracle (oracle/, its hash-partitioned OpenMP form
                    on all host cores), timed on a 1/5-scale seeded synthetic
                    list of the same workload (2e6 walkers, core 2e3)

Output: one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FCIQMC spawn attempts/s at 1e7 walkers"
UNIT = "attempts/s"
WORKLOAD = "molecule28"
N_WALKERS = 1e7
CORE = 10_000
CORE_START = 2000


def _workload_desc():
    return ("synthetic molecule, 28 spatial orbitals (56 spin orbitals, 64-bit keys), 8a+7b electrons, "
            "heat-bath generator, initiator n_a=3, real weights, tau=0.01, target 1e7 walkers, "
            "semi-stochastic core 1e4 chosen at iteration 2000; grown on the device from 500 walkers")


def _system_and_qmc(scale: float = 1.0):
    from paper_1811_11679_gb300 import inputs
    core = int(CORE * scale) if scale < 1 else CORE
    sysd, q = inputs.workload(WORKLOAD, target_population=N_WALKERS * scale, semi_stoch_size=core,
                              semi_stoch_start=CORE_START, state_capacity=int(16_000_000 * max(scale, 0.1)),
                              spawn_capacity=int(32_000_000 * max(scale, 0.1)))
    return sysd, q


def _grow(step, iterations, until):
    """Advance in blocks until `until` iterations are done."""
    while iterations() < until:
        step(min(250, until - iterations()))


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _phase_bytes(rec, W):
    """Algorithmic bytes per launch of the HBM-bound phases: K = 8W key bytes, a
    main-list entry is K + 17 bytes (key, int64 population, f64 diagonal, flag
    byte), a bucketed spawn K + 9 (key, int64 amount, initiator byte), a staged
    spawn K + 16 (key, amount, bucket/rank word)."""
    K = 8 * W
    ns, nd_pre, nd_post = float(rec["nspawn"]), float(rec["ndet_pre"]), float(rec["ndet"])
    return {
        # bucketed spawns read once, main list read once, new list written once
        "merge": ns * (K + 9) + nd_pre * (K + 17) + nd_post * (K + 17),
        # staged spawns read (key, amount, bucket/rank word), bucketed spawns written
        "scatter": ns * (K + 16) + ns * (K + 9),
        # main list read, populations/flags/attempt counts written
        "det_pass": nd_pre * (K + 17) + nd_pre * (8 + 1 + 8),
        # annihilation as a whole: spawns sorted (read + write) and merged (read),
        # main list read, new list written
        "annihilation": 3 * ns * (K + 9) + nd_pre * (K + 17) + nd_post * (K + 17),
        # whole iteration: the spawn and death phase (main list read, populations
        # and flags written, spawns written) plus the annihilation
        "iteration": nd_pre * (K + 17) + nd_pre * 9 + ns * (K + 9)
                     + 3 * ns * (K + 9) + nd_pre * (K + 17) + nd_post * (K + 17),
    }


# Spawning kernel (k_attempt) issue-slot roofline.  Warp instructions issued
# per spawn attempt and DRAM bytes per attempt, from one ncu capture of the
# kernel on the profile case (profiles/kernels_molecule28_profile_case.md);
# the peak is 4 warp instructions per cycle per SM (one per sub-partition) on
# 152 SMs at the maximum SM clock.
ATTEMPT_INST_PER_ATTEMPT = 235755617 / 7571203
ATTEMPT_DRAM_BYTES_PER_ATTEMPT = (89.771008e6 + 7.630336e6) / 7571203
N_SM = 152
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of each phase's
# kernels in the profile case's 4th iteration, and that iteration's counts
# (profiles/traffic_molecule28_profile_case.md).  A phase's `traffic` in the
# bench line is its ratio of these bytes to its algorithmic bytes times the
# bench's own algorithmic bytes: both grow with the list and the spawns.
PROFILE_CASE_REC = {"nspawn": 892485, "ndet_pre": 4040607, "ndet": 4031282}
PROFILE_CASE_DRAM = {"det_pass": 101613056 + 22525952,
                     "scatter": 23025408 + 1524736,
                     "merge": (118296320 + 54569472) + (1056000 + 330240) + (109726464 + 49445888),
                     "annihilation": 92928 + (23025408 + 1524736) + (118296320 + 54569472)
                                     + (1056000 + 330240) + (109726464 + 49445888)}


def _issue_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return 4 * N_SM * mhz * 1e6 / 1e9, mhz


def aggregate_ranks(ms: float, attempts: float, device: str):
    """Whole-job figures over the ranks of the process group: the slowest
    rank's timed region (max) and the attempts of all ranks (sum)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    a = torch.tensor([attempts], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(a, op=torch.distributed.ReduceOp.SUM)
    return float(t[0]), float(a[0])


def run_ours(args, rank, world):
    import torch

    from paper_1811_11679_gb300 import hande

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = torch.cuda.current_device()
    sysd, q = _system_and_qmc()
    q["replica"] = rank
    W = sysd["key_words"]
    eng = hande.Hande(sysd, q)
    t_grow = time.perf_counter()
    _grow(eng.iterate, lambda: eng.iterations, CORE_START + 50)
    eng.iterate(args.warmup)
    eng.synchronize()
    t_grow = time.perf_counter() - t_grow
    eng.estimators()
    stream = torch.cuda.current_stream(dev)
    assert stream.cuda_stream == eng.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        e0.record(stream)
        eng.iterate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        torch.distributed.barrier()
    rec = eng.estimators()
    attempts = float(rec["natt"].sum())
    t_max = ms
    if world > 1:
        t_max, attempts = aggregate_ranks(ms, attempts, "cuda")
    value = attempts / (t_max / 1e3)

    # per-phase device time (kernel-by-kernel launches with events), same stream
    ph = eng.iterate_timed(args.steps)
    rec2 = eng.estimators()
    nd_prev = np.concatenate([[rec["ndet"][-1]], rec2["ndet"][:-1]])
    per = {"nspawn": rec2["nspawn"].mean(), "ndet_pre": nd_prev.mean(), "ndet": rec2["ndet"].mean()}
    total = sum(ph.values())
    share = {k: v / total for k, v in ph.items()}
    dominant = max(ph, key=ph.get)
    peak, peak_kind = _peaks()
    byt = _phase_bytes(per, W)
    roof = {}
    t_phase = {k: ph[k] / args.steps for k in ph}
    t_phase["annihilation"] = t_phase["bucket_scan"] + t_phase["scatter"] + t_phase["merge"]
    t_phase["iteration"] = t_max / args.steps
    byt_pc = _phase_bytes(PROFILE_CASE_REC, W)
    for k in ("annihilation", "merge", "scatter", "det_pass", "iteration"):
        t_s = t_phase[k] / 1e3
        ach = byt[k] / t_s / 1e9
        ratio = PROFILE_CASE_DRAM[k] / byt_pc[k] if k in PROFILE_CASE_DRAM else None
        roof[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                   "frac": round(ach / peak, 4), "traffic": int(ratio * byt[k]) if ratio else None,
                   "traffic_over_algorithmic": round(ratio, 3) if ratio else None,
                   "bytes_per_launch": int(byt[k]), "ms_per_launch": round(t_phase[k], 4), "peak_source": peak_kind}
    ipeak, imhz = _issue_peak()
    att_launch = attempts / args.steps / world
    t_att = ph["attempt"] / args.steps / 1e3
    ach_i = ATTEMPT_INST_PER_ATTEMPT * att_launch / t_att / 1e9
    spawns_launch = float(rec["nspawn"].sum()) / args.steps / world
    roof_attempt = {"bound": "alu", "achieved": round(ach_i, 1), "peak": round(ipeak, 1),
                    "unit": "G warp-instructions/s", "frac": round(ach_i / ipeak, 4),
                    "traffic": int(ATTEMPT_DRAM_BYTES_PER_ATTEMPT * att_launch),
                    "ms_per_launch": round(ph["attempt"] / args.steps, 4),
                    "attempts_per_s": att_launch / t_att, "spawns_per_attempt": spawns_launch / att_launch,
                    "warp_instructions_per_spawn": ATTEMPT_INST_PER_ATTEMPT * att_launch / spawns_launch,
                    "kernel": "k_attempt (spawning: Philox draw, excitation, spawn amount, bucket)",
                    "per_unit": f"{ATTEMPT_INST_PER_ATTEMPT:.1f} warp instructions per attempt (ncu)",
                    "peak_source": f"4 warp instructions/cycle/SM x {N_SM} SMs x {imhz:.0f} MHz"}

    # end to end through the C ABI with host buffers: upload, iterate, download
    e2e_steps = min(args.steps, 10)
    nd_now = int(eng.diagnostics()["ndet"])
    bufs = eng.host_buffers(int(nd_now * 1.5) + 1024)   # page-locked, reused every step
    k_h, p_h, h_h, _ = eng.walkers(out=bufs)
    eng.set_walkers(k_h, p_h, h_h)                       # one untimed step of the same form
    eng.iterate(1)
    k_h, p_h, h_h, _ = eng.walkers(out=bufs)
    eng.estimators()
    h2d = d2h = 0
    att_e2e = 0.0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        eng.set_walkers(k_h, p_h, h_h)
        h2d += k_h.nbytes + p_h.nbytes + h_h.nbytes
        eng.iterate(1)
        k_h, p_h, h_h, f_h = eng.walkers(out=bufs)
        r = eng.estimators()
        d2h += k_h.nbytes + p_h.nbytes + h_h.nbytes + f_h.nbytes + 88 * len(r["iter"])
        att_e2e += float(r["natt"].sum())
    t_e2e = time.perf_counter() - t0
    e2e = {"value": att_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d / e2e_steps),
           "d2h_bytes_per_step": int(d2h / e2e_steps),
           "step": "set_walkers(host list; the deterministic space is kept, not rebuilt) + iterate(1) + "
                   "get_walkers + estimators"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
        "config": {"workload": _workload_desc(), "walkers_target": N_WALKERS,
                   "mean_walkers": float(rec["nw_post"].mean()) / 2 ** 32,
                   "mean_determinants": float(rec["ndet"].mean()),
                   "mean_attempts_per_step": attempts / args.steps / world,
                   "mean_spawns_per_step": float(rec["nspawn"].mean()),
                   "first_timed_iteration": int(rec["iter"][0]), "grow_seconds": round(t_grow, 2),
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"independent replicas x{world}"},
        "roofline": roof_attempt,
        "roofline_phases": roof,
        "annihilated_keys_per_s": float(rec2["nspawn"].sum()) / (t_phase["annihilation"] * args.steps / 1e3),
        "phase_ms_per_step": {k: round(v / args.steps, 4) for k, v in ph.items()},
        "phase_share": {k: round(v, 4) for k, v in share.items()},
        "dominant_phase": dominant,
        "e2e": e2e,
        "gpu_launches": int(args.steps * eng.launches_per_iteration()),
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        k_h, p_h, _, _ = eng.walkers()
        out["cpu_baseline"] = cpu_baseline(sysd, q, k_h, p_h)
    eng.close()
    if rank == 0 and not args.no_configs:
        small = lambda d: batched_leg(d, replicas=256, lo=2e3, hi=2e4)   # noqa: E731
        for key, leg in (("configs", config_lines), ("learned_proposal", learned_leg),
                         ("learned_proposal_full_basis", learned_full_basis_leg),
                         ("batched_replicas", batched_leg), ("batched_small_replicas", small),
                         ("tensor_core_gemm", tensor_core_leg)):
            try:
                out[key] = leg(dev)
            except Exception as exc:   # one failing extra leg must not lose the headline line
                out[key] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def config_lines(dev):
    """Throughput of the two smaller configurations on the same engine (extra
    keys of the default line; each timed with CUDA events on the engine's
    stream, graph launches, no host synchronisation inside the timed region):
      hubbard8  1D Hubbard ring, 8 sites, 4+4 electrons, U/t = 4, integer
                walkers, tau 0.01, target 1e4: the whole 2000-iteration run
                (the population grows from 500 walkers inside it);
      ueg14     UEG 14 electrons in 38 plane waves (128-bit keys), r_s = 1,
                initiator n_a = 3, real weights, tau 0.002, target 1e6 walkers:
                grown from 1e4 walkers until the shift varies (the population
                reached 1e6), 200 more iterations, then 400 timed iterations."""
    import torch

    from paper_1811_11679_gb300 import hande, inputs
    stream = torch.cuda.current_stream(dev)
    out = {}

    def timed(eng, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        eng.iterate(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sysd, q = inputs.workload("hubbard8")
    eng = hande.Hande(sysd, q)
    ms = timed(eng, 2000)
    r = eng.estimators()
    eng.close()
    out["hubbard8"] = {"iterations": 2000, "us_per_iteration": ms * 1e3 / 2000,
                       "attempts_per_s": float(r["natt"].sum()) / (ms / 1e3),
                       "final_walkers": float(r["nw_post"][-1]) / 2 ** 32,
                       "final_determinants": int(r["ndet"][-1]),
                       "workload": "1D Hubbard ring L=8, 4+4 electrons, t=1, U=4, integer walkers, tau=0.01, "
                                   "target 1e4, 500 walkers on the Neel determinant at the start; all 2000 "
                                   "iterations timed"}

    sysd, q = inputs.workload("ueg14", target_population=1e6, init_pop=1e4, state_capacity=2_500_000,
                              spawn_capacity=4_000_000)
    eng = hande.Hande(sysd, q)
    grown = 0
    while grown < 20000:
        eng.iterate(250)
        grown += 250
        if eng.estimators()["shift"][-1] != 0.0:
            break
    eng.iterate(200)
    eng.synchronize()
    eng.estimators()
    ms = timed(eng, 400)
    r = eng.estimators()
    eng.close()
    try:
        sysd, q = inputs.workload("hubbard18_2d")
        eng = hande.Hande(sysd, q)
        grown = 0
        while grown < 5000:
            eng.iterate(100)
            grown += 100
            if eng.estimators()["shift"][-1] != 0.0 and eng.iterations > q["semi_stoch_start"]:
                break
        eng.iterate(200)
        eng.synchronize()
        eng.estimators()
        ms2 = timed(eng, 400)
        r2 = eng.estimators()
        ncore = int(eng.diagnostics()["ncore"])
        eng.close()
        out["hubbard18_2d"] = {"iterations": 400, "first_timed_iteration": int(r2["iter"][0]),
                               "ms_per_iteration": ms2 / 400, "attempts_per_s": float(r2["natt"].sum()) / (ms2 / 1e3),
                               "mean_walkers": float(r2["nw_post"].mean()) / 2 ** 32,
                               "mean_determinants": float(r2["ndet"].mean()), "deterministic_space": ncore,
                               "workload": "2D Hubbard model, tilted 18-site square cluster (lattice vectors (3,3), "
                                           "(3,-3)), 9+9 electrons, U/t=1.3, initiator, real weights, tau=0.002, target "
                                           "1e6 walkers, deterministic space 1e4 chosen at iteration 500"}
    except Exception as exc:   # an extra line must not lose the others
        out["hubbard18_2d"] = {"error": f"{type(exc).__name__}: {exc}"}
    out["ueg14"] = {"iterations": 400, "first_timed_iteration": int(r["iter"][0]),
                    "ms_per_iteration": ms / 400, "attempts_per_s": float(r["natt"].sum()) / (ms / 1e3),
                    "annihilated_spawns_per_s": float(r["nspawn"].sum()) / (ms / 1e3),
                    "mean_walkers": float(r["nw_post"].mean()) / 2 ** 32,
                    "mean_determinants": float(r["ndet"].mean()),
                    "workload": "UEG 14 electrons in 38 spatial plane waves (76 spin orbitals, 128-bit keys), "
                                "r_s=1, initiator n_a=3, real weights, spawn_cutoff 0.1, tau=0.002, target 1e6 "
                                "walkers; grown from 1e4 walkers until the shift varies, +200 iterations"}
    return out


def learned_leg(dev, iterations=4000, nel=14, norb=38, tau=0.002, target=2e5, equil=500, grow_blocks=80):
    """The learned excitation proposal against the uniform generator on the
    same UEG run (14 electrons in 38 plane waves, r_s=1, initiator, real
    weights, tau=0.002, target 2e5 walkers): each grown until the shift varies,
    equilibrated 500 iterations, then `iterations` timed iterations (CUDA
    events; the learned run keeps training every 10 iterations inside the timed
    region).  Error-bar-normalised cost = (reblocked error of E_proj)^2 x time."""
    import torch

    from paper_1811_11679_gb300 import analysis, hande, inputs
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name in ("uniform", "learned"):
        sysd = inputs.ueg_system(nel, norb, 1.0)
        q = inputs.qmc_params(tau=tau, target_population=target, init_pop=target / 10, initiator=1,
                              real_amplitudes=1, spawn_cutoff=0.1, seed=7,
                              state_capacity=int(12 * target) + (1 << 16),
                              spawn_capacity=int(24 * target) + (1 << 17),
                              excit_gen=1 if name == "learned" else 0)
        eng = hande.Hande(sysd, q)
        if name == "learned":
            eng.learn_proposal(width=256, batch=4096, period=10, learning_rate=2e-3, seed=1)
        for _ in range(grow_blocks):
            eng.iterate(250)
            if eng.estimators()["shift"][-1] != 0.0:
                break
        eng.iterate(equil)
        eng.synchronize()
        eng.estimators()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        eng.iterate(iterations)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = eng.estimators()
        e_ref, _ = eng.reference()
        E, err = analysis.projected_energy(r, e_ref)
        eng.close()
        out[name] = {"E_proj": E, "error": err, "ms_per_iteration": ms / iterations,
                     "attempts_per_s": float(r["natt"].sum()) / (ms / 1e3),
                     "spawns_per_attempt": float(r["nspawn"].sum()) / max(float(r["natt"].sum()), 1.0),
                     "mean_walkers": float(r["nw_post"].mean()) / 2 ** 32,
                     "cost_error2_x_seconds": err * err * ms / 1e3}
    u, l = out["uniform"], out["learned"]
    out["efficiency_gain"] = u["cost_error2_x_seconds"] / l["cost_error2_x_seconds"]
    out["agreement_sigma"] = abs(u["E_proj"] - l["E_proj"]) / float(np.hypot(u["error"], l["error"]))
    out["workload"] = (f"UEG {nel}e in {norb} plane waves, r_s=1, initiator n_a=3, real weights, tau={tau}, "
                       f"target {target:.0e}; {iterations} timed iterations each; learned = MLP 3 layers width 256 "
                       "(BF16 tensor cores), Adam every 10 iterations on 4096 recorded attempts")
    return out


def learned_full_basis_leg(dev, target=1e5, pretrain=2000, taus=(5e-5, 1e-3), iterations=(40000, 8000)):
    """The learned proposal at the full basis of its configuration (UEG 54
    electrons in 246 plane waves, 512-bit keys, r_s = 1, initiator, real
    weights; 1e5 target walkers instead of 1e8) against the uniform generator,
    each at its own stable time step: the uniform generator at the time-step
    search's value for it (5e-5; at 1e-3 its spawns of up to ~18 walkers per
    attempt make the population explode), the learned one at 1e-3.  The network
    is warm-started from a 2000-iteration run at tau = 2e-4 and keeps training
    every 10 iterations.  Each arm: grown from a tenth of the target until the
    shift varies, 3000 iterations of equilibration, then the timed iterations
    (CUDA events).  Cost = (reblocked error of E_proj)^2 x time."""
    import torch

    from paper_1811_11679_gb300 import analysis, hande, inputs
    stream = torch.cuda.current_stream(dev)
    sysd = inputs.ueg_system(54, 246, 1.0)

    def qmc(gen, tau):
        return inputs.qmc_params(tau=tau, target_population=target, init_pop=target / 10, initiator=1,
                                 real_amplitudes=1, spawn_cutoff=0.1, seed=7,
                                 state_capacity=int(20 * target) + (1 << 20),
                                 spawn_capacity=int(40 * target) + (1 << 21), excit_gen=gen)

    pre = hande.Hande(sysd, qmc(1, 2e-4))
    pre.learn_proposal(width=256, batch=4096, period=10, learning_rate=2e-3, seed=1)
    pre.iterate(pretrain)
    params = pre.learn_params()
    pre.close()
    out = {}
    for name, tau, iters in (("uniform", taus[0], iterations[0]), ("learned", taus[1], iterations[1])):
        eng = hande.Hande(sysd, qmc(1 if name == "learned" else 0, tau))
        if name == "learned":
            eng.learn_proposal(width=256, batch=4096, period=10, learning_rate=2e-3, seed=1)
            eng.learn_params(params)
            eng.learn_refresh()
        for _ in range(200):
            eng.iterate(100)
            if eng.estimators()["shift"][-1] != 0.0:
                break
        eng.iterate(3000)
        eng.synchronize()
        eng.estimators()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        eng.iterate(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        r = eng.estimators()
        e_ref, _ = eng.reference()
        E, err = analysis.projected_energy(r, e_ref)
        eng.close()
        out[name] = {"tau": tau, "iterations": iters, "E_proj": E, "error": err, "ms_per_iteration": ms / iters,
                     "attempts_per_s": float(r["natt"].sum()) / (ms / 1e3),
                     "spawns_per_attempt": float(r["nspawn"].sum()) / max(float(r["natt"].sum()), 1.0),
                     "mean_walkers": float(r["nw_post"].mean()) / 2 ** 32,
                     "cost_error2_x_seconds": err * err * ms / 1e3}
    u, l = out["uniform"], out["learned"]
    out["efficiency_gain"] = u["cost_error2_x_seconds"] / l["cost_error2_x_seconds"]
    out["agreement_sigma"] = abs(u["E_proj"] - l["E_proj"]) / float(np.hypot(u["error"], l["error"]))
    out["workload"] = (f"UEG 54e in 246 plane waves (512-bit keys), r_s=1, initiator n_a=3, real weights, target "
                       f"{target:.0e}; uniform at tau={taus[0]} ({iterations[0]} timed iterations), learned at "
                       f"tau={taus[1]} ({iterations[1]}), network warm-started from {pretrain} iterations at "
                       "tau=2e-4, Adam every 10 iterations on 4096 recorded attempts")
    return out


def batched_leg(dev, replicas=64, grow=300, steps=50, lo=1e4, hi=1e6):
    """Batched replicas (inputs.batched_replicas: UEG 14 electrons in 38 or 66
    orbitals, four r_s, uneven targets log-uniform in [lo, hi]; the default
    line runs 64 replicas of 1e4-1e6 walkers and 256 of 2e3-2e4) advanced by the batched graphs
    (one launch per phase per key-width group, launch shape autotuned) against
    the same replicas advanced back to back on the plain path (each replica's
    own captured iteration graph on its own stream, no host synchronisation),
    both timed with CUDA events on the caller's stream.  Both forms produce the
    same Markov chains bit for bit, so their error bars are equal and the time
    ratio is the error-bar-normalised cost ratio."""
    import torch

    from paper_1811_11679_gb300 import hande, inputs
    stream = torch.cuda.current_stream(dev)
    systems, qmcs = inputs.batched_replicas(replicas, lo=lo, hi=hi)
    b = hande.HandeBatch(systems, qmcs)
    b.iterate(grow)
    scale, tuned_ms = b.autotune(iterations=3)
    for v in b.replicas:
        v.estimators()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ms_b = timed(lambda: b.iterate(steps))
    att_b = float(sum(v.estimators()["natt"].sum() for v in b.replicas))
    groups, cap = b.layout()

    def plain():
        for _ in range(steps):
            for v in b.replicas:
                v.iterate(1)
        for v in b.replicas:
            v.synchronize()
    ms_p = timed(plain)
    att_p = float(sum(v.estimators()["natt"].sum() for v in b.replicas))
    launches = sum(v.launches_per_iteration() for v in b.replicas)
    b.close()
    return {"replicas": replicas, "steps": steps, "grow_iterations": grow,
            "batched": {"attempts_per_s": att_b / (ms_b / 1e3), "ms_per_step": ms_b / steps,
                        "autotuned_scale": scale, "launch_groups": groups, "replicas_per_group_max": cap},
            "plain_back_to_back": {"attempts_per_s": att_p / (ms_p / 1e3), "ms_per_step": ms_p / steps,
                                   "kernel_launches_per_step": launches},
            "speedup": (att_b / ms_b) / (att_p / ms_p),
            "workload": f"{replicas} UEG replicas: 14 electrons in 38 or 66 spatial orbitals (128- or 512-bit "
                        f"keys), r_s 0.5/1/2/5, targets log-uniform in [{lo:.0e}, {hi:.0e}], initiator, real "
                        "weights, tau=0.002"}


def tensor_core_leg(dev, calls=20):
    """The tensor-core GEMM alone (tcgen05 MMAs, TMA tiles, TMEM accumulators)
    at the learned proposal's shapes: the table refresh of a 246-orbital basis
    (2 x 246^2 rows, first layer K = 512 and hidden layer K = 256) and a
    4096-sample training batch; FLOP/s against the measured BF16 burst peak
    and, since these shapes sit below the ridge point, algorithmic bytes/s
    against the measured copy bandwidth."""
    import torch

    from paper_1811_11679_gb300 import hande
    peak = _bf16_peak()
    hbm = _peaks()
    stream = torch.cuda.current_stream(dev)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rows = []
    g = torch.Generator(device="cuda").manual_seed(3)
    for what, m, n, k in (("table refresh, 246 orbitals, layer 1", 121088, 256, 512),
                          ("table refresh, 246 orbitals, layer 2", 121088, 256, 256),
                          ("training batch 4096, layer 2", 4096, 256, 256)):
        a = torch.randn((m, k), generator=g, device="cuda").to(torch.bfloat16)
        b = torch.randn((n, k), generator=g, device="cuda").to(torch.bfloat16)
        d = torch.empty((m, n), dtype=torch.float32, device="cuda")
        for _ in range(3):
            hande.gemm_bf16(a, b, d, status=status)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(calls):
            hande.gemm_bf16(a, b, d, status=status)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / calls
        tf = 2.0 * m * n * k / (ms / 1e3) / 1e12
        # algorithmic bytes: A and B read once (BF16), D written once (FP32)
        byt = 2.0 * (m * k + n * k) + 4.0 * m * n
        gbs = byt / (ms / 1e3) / 1e9
        rows.append({"shape": what, "m": m, "n": n, "k": k, "us_per_launch": ms * 1e3, "tflops": tf,
                     "frac": tf / peak[0], "bytes": int(byt), "hbm_gbs": gbs, "hbm_frac": gbs / hbm[0]})
    assert int(status.item()) == 0, "tensor-core GEMM wait timed out"
    best = max(rows, key=lambda x: x["tflops"])
    return {"bound": "tensor", "achieved": round(best["tflops"], 1), "peak": peak[0], "unit": "TFLOP/s",
            "frac": round(best["frac"], 4), "traffic": None, "peak_source": peak[1], "kernel": "k_gemm_bf16_tn_p (persistent, two TMEM accumulators)",
            "hbm": {"achieved": round(best["hbm_gbs"], 1), "peak": hbm[0], "unit": "GB/s",
                    "frac": round(best["hbm_frac"], 4), "peak_source": hbm[1]},
            "shapes": rows}


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def cpu_baseline(sysd, q, keys, pops):
    """The oracle as it stands on the host's cores: one iteration of its
    hash-partitioned OpenMP form (all cores; the same source as the serial
    oracle and bit-identical to it) on the device's current 1e7-walker list
    (its deterministic space re-chosen from that list), and one iteration of
    the serial oracle on the same list for comparison."""
    import oracle
    cores = os.cpu_count() or 1
    out = {}
    for name, threads in (("all", cores), ("one", None)):
        o = oracle.Oracle(sysd, dict(q, semi_stoch_start=0), threads=threads)
        o.set_walkers(keys, pops)
        t0 = time.perf_counter()
        o.iterate(1)
        dt = time.perf_counter() - t0
        out[name] = (float(o.records()["natt"][-1]) / dt, dt)
    return {"value": out["all"][0], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one oracle iteration (OpenMP, hash-partitioned, all host cores) on the GPU run's "
                      "steady-state list (1e7 walkers)",
            "seconds": round(out["all"][1], 3),
            "single_core": {"value": out["one"][0], "cores": 1, "seconds": round(out["one"][1], 3)}}


def run_reference(args):
    """The oracle arm on the host cores: the workload's system and run
    parameters on a seeded synthetic walker list (the reference holds 10% of
    the walkers, the rest on 1-4-fold excitations with Pareto populations;
    deterministic space chosen from that list), one oracle iteration per step.
    The list holds up to 1e6 walkers (1/10 of the GPU run) and fewer when many
    steps are asked for, so the whole run stays within a few minutes."""
    import oracle
    from paper_1811_11679_gb300 import inputs
    walkers = int(min(2e6, max(4e4, 2.4e8 / (args.steps + args.warmup))))
    ndet = walkers // 4
    sysd, q = _system_and_qmc(scale=walkers / N_WALKERS)
    q = dict(q, semi_stoch_start=0, target_population=float(walkers))
    keys, pops = inputs.synthetic_walkers(sysd, ndet, float(walkers))
    cores = os.cpu_count() or 1
    o = oracle.Oracle(sysd, q, threads=cores)
    o.set_walkers(keys, pops)
    o.iterate(args.warmup)
    n0 = len(o.records()["iter"])
    t0 = time.perf_counter()
    o.iterate(args.steps)
    dt = time.perf_counter() - t0
    r = o.records()
    att = float(r["natt"][n0:].sum())
    v = att / dt
    sample = (f"seeded synthetic list of {ndet} determinants / {walkers} walkers with the workload's system and "
              f"run parameters (core {q['semi_stoch_size']} chosen from the list), one oracle iteration per step, "
              f"hash-partitioned OpenMP form on {cores} threads")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64", "data": "synthetic",
            "config": {"workload": _workload_desc(), "sample": sample,
                       "mean_walkers": float(r["nw_post"][n0:].mean()) / 2 ** 32},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """Small case for ncu captures: a seeded synthetic list of 4e6 determinants
    (8e6 walkers; main list and spawn arrays larger than L2) set on the device,
    then 3 + 3 iterations; few kernel launches precede the captured ones."""
    import torch

    from paper_1811_11679_gb300 import hande, inputs
    torch.cuda.set_device(0)
    sysd, q = inputs.workload(WORKLOAD, target_population=7e6, semi_stoch_size=CORE, semi_stoch_start=0,
                              state_capacity=12_000_000, spawn_capacity=16_000_000)
    keys, pops = inputs.synthetic_walkers(sysd, 4_000_000, 8e6)
    eng = hande.Hande(sysd, q)
    eng.set_walkers(keys, pops)
    eng.iterate(3)
    eng.iterate(3)
    eng.synchronize()
    r = eng.estimators()
    print(json.dumps({"profile_case": True, "ndet": int(r["ndet"][-1]), "natt": int(r["natt"][-1]),
                      "nspawn": int(r["nspawn"][-1]), "ndet_per_iteration": [int(x) for x in r["ndet"]],
                      "nspawn_per_iteration": [int(x) for x in r["nspawn"]]}))
    eng.close()


def run_profile_batched(args):
    """Launch-list case of the batched form: the batched leg's replicas grown
    300 iterations and autotuned, then 3 batched iterations and 3 iterations of
    every replica on the plain path inside one profiler range."""
    import torch

    from paper_1811_11679_gb300 import hande, inputs
    torch.cuda.set_device(0)
    systems, qmcs = inputs.batched_replicas(args.profile_batched)
    b = hande.HandeBatch(systems, qmcs)
    b.iterate(300)
    scale, ms = b.autotune(iterations=3)
    groups, cap = b.layout()
    b.synchronize()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    b.iterate(3)
    torch.cuda.synchronize()
    for _ in range(3):
        for v in b.replicas:
            v.iterate(1)
    for v in b.replicas:
        v.synchronize()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_batched": True, "replicas": len(b), "autotuned_scale": scale,
                      "launch_groups": groups, "replicas_per_group_max": cap, "tuned_ms_per_iteration": ms}))
    b.close()


def run_batched(args):
    """Batched replicas (inputs.batched_replicas: UEG 14e in 38/66 orbitals, four
    r_s, targets log-uniform in [1e4, 1e6]) advanced together through
    hande_batch_iterate, against the same replicas advanced one after another
    (each run alone on the GPU, as separate plain runs would be)."""
    import torch

    from paper_1811_11679_gb300 import hande, inputs
    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    systems, qmcs = inputs.batched_replicas(args.batched)
    b = hande.HandeBatch(systems, qmcs)
    t_grow = time.perf_counter()
    _grow(b.iterate, lambda: b.replicas[0].iterations, args.batched_grow)
    b.iterate(args.warmup)
    b.synchronize()
    t_grow = time.perf_counter() - t_grow
    for v in b.replicas:
        v.estimators()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        w0 = time.perf_counter()
        e0.record(stream)
        b.iterate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    ms = e0.elapsed_time(e1)
    recs = [v.estimators() for v in b.replicas]
    attempts = float(sum(r["natt"].sum() for r in recs))
    walkers = float(sum(r["nw_post"].mean() for r in recs)) / 2 ** 32
    dets = float(sum(r["ndet"].mean() for r in recs))
    # the same replicas one at a time: each replica's steps, then the next one
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    for v in b.replicas:
        v.iterate(args.steps)
        v.synchronize()
    seq_wall = time.perf_counter() - s0
    seq_attempts = float(sum(v.estimators()["natt"].sum() for v in b.replicas))
    launches = sum(v.launches_per_iteration() for v in b.replicas) * args.steps
    b.close()
    return {"metric": "FCIQMC spawn attempts/s, batched replicas", "value": attempts / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64+f64",
            "data": "synthetic",
            "config": {"workload": f"{args.batched} UEG replicas: 14 electrons in 38 or 66 spatial orbitals "
                                   "(128- or 512-bit keys), r_s 0.5/1/2/5, targets log-uniform in [1e4, 1e6], "
                                   "initiator, real weights, tau=0.002",
                       "replicas": args.batched, "grow_iterations": args.batched_grow,
                       "grow_seconds": round(t_grow, 2), "mean_walkers_total": walkers,
                       "mean_determinants_total": dets, "l2": "inputs larger than L2 (no flush)"},
            "wall_value": attempts / wall,
            "sequential": {"value": seq_attempts / seq_wall, "unit": UNIT,
                           "ms_per_step": seq_wall * 1e3 / args.steps,
                           "how": "each replica iterated alone for the same steps, then synchronised, "
                                  "one replica after another (host wall clock)"},
            "gpu_launches": launches, "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the Hubbard and UEG lines")
    ap.add_argument("--profile-case", action="store_true",
                    help="small synthetic-start case for ncu captures (no timing output)")
    ap.add_argument("--profile-gemm", action="store_true",
                    help="the tensor-core GEMM shapes alone, two timed calls each (for ncu captures)")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="this many batched UEG replicas: 3 batched then 3 plain iterations inside a "
                         "profiler range (ncu --profile-from-start off)")
    ap.add_argument("--batched", type=int, default=0,
                    help="time this many batched UEG replicas instead of the molecule workload")
    ap.add_argument("--batched-grow", type=int, default=600,
                    help="iterations before the timed region in --batched mode")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.profile_case:
        run_profile_case(args)
        return
    if args.profile_batched > 0:
        run_profile_batched(args)
        return
    if args.profile_gemm:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"profile_gemm": True, **tensor_core_leg(torch.cuda.current_device(), calls=2)}))
        return
    if args.batched > 0:
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
