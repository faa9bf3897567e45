"""Benchmark: Fock-space H psi terms/s and RK4 steps/s on one GB300.

Workload (default): the batched coherent state -- M=7 ring modes, w_p = p^2/2,
contact coupling C = -0.05/n_tot, alpha = sqrt(n_tot/2) on p = -1 and p = +1 at
n_tot = 16, every Poisson-weighted sector N <= n_tot + 6 sqrt(n_tot) = 40 (281
non-empty sectors, 62,891,499 kets, complex128), advanced together.  A step is one RK4
step of the whole state (four fused H psi stages over every sector).

The state (1 GB) is larger than L2 (129 MB), so no L2 flush is needed between
steps.  Prints ONE JSON line (rank 0).

--impl reference times the CPU oracle (oracle/) as it stands, its rows on every
host core (OpenMP), on a bounded sample of the same workload (RK4 steps of the N=16
sectors).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as wl  # noqa: E402

# FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz; the
# roofline uses the DFMA rate measured on the GPU by the run itself (qb_measure_fp64_fma)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM bytes per ket of one stage launch (the first stage of a step), from an ncu capture
# of the current stage kernel (batched coherent at n_tot=12: 617.2 MB read + 226.8 MB
# written over 15,380,937 kets); scaled by kets
STAGE_DRAM_BYTES_PER_KET = (617.219072e6 + 226.820352e6) / 15380937
# the same capture's issue-slot and L1 data-pipe utilisation (the kernel's real limits:
# the FP64 pipe is idle)
STAGE_NCU_ISSUE_ACTIVE = 0.670
STAGE_NCU_L1_WAVEFRONTS = 0.920


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int = 0):
        self.rows = []
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, value: float, device: str) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank_step: float, ms_per_step: float) -> float:
    """Whole-job units per second: every rank (an independent replica) processes
    units_per_rank_step per step, and a step takes the slowest rank's time."""
    return world * units_per_rank_step / (ms_per_step * 1e-3)


def workload(name: str, n_tot: int = 16):
    if name == "batched_coherent":
        W = wl.batched_coherent(n_tot=n_tot)
        return W, dict(n_min=0, n_max=W.n_max, p_list=None)
    if name == "large_sector":
        W = wl.large_sector()
        return W, dict(n_min=20, n_max=20, p_list=[0])
    if name == "plain_single_sector":
        W = wl.plain_single_sector()
        return W, dict(n_min=6, n_max=6, p_list=[0])
    raise SystemExit(f"unknown config {name}")


def init_state(qs, W, psi):
    if W.kind == "coherent":
        qs.init_coherent(W.z, psi)
    elif W.kind == "number":
        qs.init_number(W.occ, psi)
    else:
        qs.init_field_number(W.z, W.n_tot, psi)


def run_reference(args):
    """The CPU oracle on every host core (its row-parallel RK4), one RK4 step per
    timed step on a bounded sample of the workload."""
    import oracle as orc

    W, sp = workload(args.config, args.n_tot)
    if W.kind == "coherent":
        Ns = [min(16, W.n_max)]
    else:
        Ns = [W.n_min]
    sectors = [(N, P) for N in Ns for P in range(W.M) if orc.sector_dim(W.M, N, P) > 0]
    space = orc.Space(W.M, sectors)
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    psi /= np.linalg.norm(psi)
    terms = orc.count_terms(space, W.L)
    for _ in range(args.warmup):
        psi = orc.rk4_rows(space, W.w, W.L, psi, W.dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = orc.rk4_rows(space, W.w, W.L, psi, W.dt, 1)
    dt_s = (time.perf_counter() - t0) / args.steps
    value = 4 * terms / dt_s
    sample = f"one RK4 step (4 H psi) of the sectors N={Ns} (all P) of {W.name}: {space.total} kets, {terms} terms"
    line = {
        "impl": "reference", "metric": "H_psi_terms_per_s", "value": value, "unit": "terms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W.name, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "terms/s", "cores": orc.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline(W, seconds_cap: float = 15.0):
    """Times the oracle's row-parallel RK4 on every host core (OpenMP) on one N layer
    of the workload (all P): RK4 steps until about seconds_cap of wall time."""
    import oracle as orc

    N = min(16, W.n_max) if W.kind == "coherent" else W.n_min
    sectors = [(N, P) for P in range(W.M) if orc.sector_dim(W.M, N, P) > 0]
    space = orc.Space(W.M, sectors)
    if space.total > 300000:  # bound the sample: the first sector only
        sectors = sectors[:1]
        space = orc.Space(W.M, sectors)
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(space.total) + 1j * rng.standard_normal(space.total)
    terms = orc.count_terms(space, W.L)
    t0 = time.perf_counter()
    n = 0
    while True:
        psi = orc.rk4_rows(space, W.w, W.L, psi, W.dt, 1)
        n += 1
        if time.perf_counter() - t0 > seconds_cap or n >= 50:
            break
    el = (time.perf_counter() - t0) / n
    return {"value": 4 * terms / el, "unit": "terms/s", "cores": orc.threads(), "kind": "oracle",
            "sample": f"{n} RK4 step(s) of sectors N={N} ({space.total} kets, {terms} terms/H psi) of {W.name}, "
                      f"rows of each H psi on {orc.threads()} host threads"}


def adjoint_extra(qb, torch, steps: int = 20, ckpt_every: int = 10):
    """Adjoint workload (M=5, contact C=-0.1, complex-Gaussian alpha scaled to n_tot=40,
    N <= 77: 386 sectors, 27.3M kets): forward RK4 time per step against the time per
    step of qb_adjoint (forward pass with checkpoints + loss + backward costate pass)."""
    W = wl.adjoint_coherent()
    L0 = wl.contact_coupling(W.M, 1.0)
    qs = qb.Space(W.M, W.w, L0, 0, W.n_max)
    psi = qs.empty_state()
    qs.init_coherent(W.z, psi)
    work = qs.workspace(1)
    qs.evolve_batch(psi, [-0.1], W.dt, 2, work)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qs.evolve_batch(psi, [-0.1], W.dt, steps, work)
    torch.cuda.synchronize()
    fwd = (time.perf_counter() - t0) / steps
    del psi, work

    def timed(ck, cg=False):
        nbytes = int(qb.lib().qb_adjoint_workspace_bytes(qs._h, steps, ck))
        aw = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        qs.adjoint(W.z, -0.1, W.dt, 2, ckpt_every=ck if ck == 0 else 2, loss="Q", work=aw, coupling_grad=cg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = qs.adjoint(W.z, -0.1, W.dt, steps, ckpt_every=ck, loss="Q", work=aw, coupling_grad=cg)
        torch.cuda.synchronize()
        del aw
        torch.cuda.empty_cache()
        return (time.perf_counter() - t0) / steps, r, nbytes

    adj, r, nb = timed(ckpt_every)
    out = {"workload": W.name, "kets": qs.total, "sectors": qs.n_sectors, "steps": steps, "ckpt_every": ckpt_every,
           "forward_ms_per_step": fwd * 1e3, "adjoint_ms_per_step": adj * 1e3, "adjoint_over_forward": adj / fwd,
           "loss_Q": r["loss"], "grad_scale": r["grad_scale"], "workspace_GB": nb / 1e9}
    # the tape mode (every step's stage vectors kept) where its workspace fits
    tape_bytes = int(qb.lib().qb_adjoint_workspace_bytes(qs._h, steps, 0))
    free, _ = torch.cuda.mem_get_info()
    if tape_bytes < 0.8 * free:
        adj0, r0, nb0 = timed(0)
        out["tape"] = {"ckpt_every": 0, "adjoint_ms_per_step": adj0 * 1e3, "adjoint_over_forward": adj0 / fwd,
                       "workspace_GB": nb0 / 1e9, "grad_scale": r0["grad_scale"],
                       "grad_scale_rel_diff": abs(r0["grad_scale"] - r["grad_scale"]) / abs(r["grad_scale"])}
        # with the gradient of every coupling entry (qb_adjoint_couplings)
        adjc, rc, _ = timed(0, True)
        L0u = wl.contact_coupling(W.M, 1.0)
        along = float(np.sum((np.conj(rc["grad_L"]) * L0u).real))
        out["tape_couplings"] = {"adjoint_ms_per_step": adjc * 1e3, "adjoint_over_forward": adjc / fwd,
                                 "along_L0_minus_grad_scale_rel": abs(along - rc["grad_scale"]) / abs(rc["grad_scale"])}
    del qs
    torch.cuda.empty_cache()
    return out


def small_extra(qb, torch):
    """The plain single-sector workload (M=5, |0,2,2,2,0>, 42 kets), the full run of
    10^4 RK4 steps: resident (one launch for every step) against one launch per stage."""
    W = wl.plain_single_sector()
    qs = qb.Space(W.M, W.w, W.L, 6, 6, [0])
    psi = qs.empty_state()
    work = qs.workspace(1)
    out = {"workload": W.name, "kets": qs.total, "steps": W.steps}
    for label, kets in (("resident", 1024), ("stage_launches", 0)):
        qs.set_resident_max(kets)
        qs.init_number(W.occ, psi)
        qs.evolve(psi, W.dt, 50, work)
        qs.init_number(W.occ, psi)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        qs.evolve(psi, W.dt, W.steps, work)
        e1.record()
        torch.cuda.synchronize()
        out[label + "_steps_per_s"] = W.steps / (e0.elapsed_time(e1) * 1e-3)
    return out


def exact_extra(qb, torch, steps: int = 3):
    """The batched coherent workload (M=7, n_tot=16, N <= 40) with momentum conserved
    exactly (the contact coupling restricted to p+q = r+s): every exact (N, P) sector
    in one launch per stage, with the ranking tables in global memory."""
    W = wl.batched_coherent()
    L = wl.contact_coupling(W.M, -0.05 / 16, exact=True)
    qs = qb.Space(W.M, W.w, L, 0, W.n_max, exact=True)
    terms, _ = qs.terms()
    psi = qs.empty_state()
    qs.init_coherent(W.z, psi)
    work = qs.workspace(1)
    resident_max = qs.autotune(W.dt, psi, steps=1, work=work)
    qs.evolve(psi, W.dt, 1, work)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qs.evolve(psi, W.dt, steps, work)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": W.name + "_exact_momentum", "kets": qs.total, "sectors": qs.n_sectors,
           "terms_per_hpsi": terms, "ms_per_step": ms, "terms_per_s": 4 * terms / (ms * 1e-3),
           "rk4_steps_per_s": 1e3 / ms, "resident_max_kets": resident_max}
    del psi, work, qs
    torch.cuda.empty_cache()
    return out


def long_range_extra(qb, torch, steps: int = 3):
    """The long-range field-number workload (M=9, L = -(0.1/n_tot) / (M (p-r)^2), n_p from
    Poisson(3) with seed-0 phases: one particle number, every P sector): RK4 steps through
    the specialised M=9 stage kernel, shape and resident threshold autotuned."""
    W = wl.long_range_field_number()
    qs = qb.Space(W.M, W.w, W.L, W.n_min, W.n_max)
    terms, _ = qs.terms()
    psi = qs.empty_state()
    qs.init_field_number(W.z, W.n_tot, psi)
    work = qs.workspace(1)
    resident_max = qs.autotune(W.dt, psi, steps=1, work=work)
    qs.evolve(psi, W.dt, 1, work)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qs.evolve(psi, W.dt, steps, work)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"workload": W.name, "kets": qs.total, "sectors": qs.n_sectors, "terms_per_hpsi": terms,
           "ms_per_step": ms, "terms_per_s": 4 * terms / (ms * 1e-3), "rk4_steps_per_s": 1e3 / ms,
           "tile_shape": qs.tuning.get("tile_shape"), "resident_max_kets": resident_max}
    del psi, work, qs
    torch.cuda.empty_cache()
    return out


def squeezing_extra(qb, torch, n_list=(4, 8, 12)):
    """Sec. IV E's squeezing analysis (the paper's n_tot sweep, scaled down): for each
    n_tot the M=7 long-range system from a Gaussian coherent profile, its strength set
    so that |n_tot chi| = 0.242, runs to t = 1.6
    with observables every 10 steps (qb_evolve_observe); onset t_sqz (V_- <= 0.8)
    and maximal squeezing (V_min, tau_min = |n_tot chi| t_min) from qb_squeezing,
    beside the one-mode estimates, then the fits V_min = c0 n^c1 and
    tau_min = c0 + c1 log n over the runs (qb_fit)."""
    runs = []
    for n in n_list:
        unit = wl.squeezing_coherent(n)  # strength 1: n_tot chi scales with the strength
        G = 0.242 / abs(qb.api.interaction_per_occupation(unit.M, unit.w, unit.L, unit.z))
        W = wl.squeezing_coherent(n, G=G)
        qs = qb.Space(W.M, W.w, W.L, W.n_min, W.n_max)
        psi = qs.empty_state()
        qs.init_coherent(W.z, psi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        series = qs.evolve_observe(psi, W.dt, W.steps, W.obs_every)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        sq = qb.api.squeezing([o["Vminus_p"] for o in series], W.dt * W.obs_every, 0.8)
        chi = abs(qb.api.interaction_per_occupation(W.M, W.w, W.L, W.z))
        runs.append({"n_tot": n, "kets": qs.total, "steps": W.steps, "wall_s": wall, "t_sqz": sq["t_sqz"],
                     "crossed": sq["flag"] == qb.QB_CROSSED, "v_min": sq["v_min"], "t_min": sq["t_min"],
                     "tau_min": chi * sq["t_min"], "t_sqz_one_mode": 0.05 / chi,
                     "v_min_one_mode": n ** (-1.0 / 3.0), "ntot_chi": chi})
        del qs, psi
        torch.cuda.empty_cache()
    ns = [r["n_tot"] for r in runs]
    vfit = qb.api.fit(ns, [r["v_min"] for r in runs], "power")
    tfit = qb.api.fit(ns, [r["tau_min"] for r in runs], "log")
    return {"runs": runs, "v_min_power_law": {"c0": vfit[0], "c1": vfit[1]},
            "tau_min_log_law": {"c0": tfit[0], "c1": tfit[1]}}


def breaktime_sweep(qb, torch, r_list=(1, 2, 3, 4, 6, 8), chunk: int = 1000):
    """Sec. IV C-D's breaktime scaling with n_tot (run with --breaktime-sweep): for each
    average mode occupation r the M=5 long-range coherent system evolves with
    observables every 20 steps until Q >= 0.15 and 1 - lam_p / n_tot >= 0.1 have both
    been crossed (or t = 30); breaktimes from qb_breaktime, then logarithmic and
    power-law fits of t_br against n_tot (qb_fit) with their rms residuals."""
    runs = []
    for r in r_list:
        W = wl.breaktime_coherent(r)
        qs = qb.Space(W.M, W.w, W.L, W.n_min, W.n_max)
        psi = qs.empty_state()
        qs.init_coherent(W.z, psi)
        work = qs.workspace(1)
        Q, PO = [], []
        t0 = time.perf_counter()
        done = 0
        while done < W.steps:
            k = min(chunk, W.steps - done)
            ser = qs.evolve_observe(psi, W.dt, k, W.obs_every, work)
            part = ser if done == 0 else ser[1:]  # the first sample repeats the last of the previous chunk
            Q += [o["Q"] for o in part]
            PO += [o["PO"] for o in part]
            done += k
            if max(Q) >= 0.15 and max(PO) >= 0.1:
                break
        torch.cuda.synchronize()
        dt_obs = W.dt * W.obs_every
        tq, fq = qb.breaktime(Q, dt_obs, 0.15)
        tp, fp = qb.breaktime(PO, dt_obs, 0.1)
        runs.append({"r": r, "n_tot": W.n_tot, "kets": qs.total, "steps": done, "wall_s": time.perf_counter() - t0,
                     "t_br_Q": tq, "Q_crossed": fq == qb.QB_CROSSED, "t_br_PO": tp, "PO_crossed": fp == qb.QB_CROSSED})
        del qs, psi, work
        torch.cuda.empty_cache()
    fits = {}
    for key in ("t_br_Q", "t_br_PO"):
        pts = [(x["n_tot"], x[key]) for x in runs if x[key] == x[key]]
        if len(pts) < 2:
            continue
        n = np.array([p[0] for p in pts], dtype=float)
        t = np.array([p[1] for p in pts], dtype=float)
        out = {}
        for kind in ("log", "power"):
            c0, c1 = qb.api.fit(n, t, kind)
            pred = c0 + c1 * np.log(n) if kind == "log" else c0 * n ** c1
            out[kind] = {"c0": c0, "c1": c1, "rms": float(np.sqrt(np.mean((pred - t) ** 2)))}
        fits[key] = out
    return {"workload": "breaktime_coherent_M5", "runs": runs, "fits": fits}


def large_sector_roofline(qb, torch, peaks, dfma_tflops, steps: int = 20):
    """One H psi of the largest single sector of the workloads: M=11, w=|p|, contact
    C=-0.02, N=20, P=0 (2,731,365 kets), timed as RK4 steps of the single state (four
    stage launches each, the first weighted copy of the call amortised over `steps`),
    against the algorithmic 32 B per ket and H psi (read psi, write the output) and
    the FP64-equivalent 4 flop per term."""
    W = wl.large_sector()
    qs = qb.Space(W.M, W.w, W.L, 20, 20, [0])
    terms = qs.terms()[0]
    psi = qs.empty_state()
    qs.init_number(W.occ, psi)
    work = qs.workspace(1)
    qs.autotune(W.dt, psi, steps=2, work=work)
    qs.evolve(psi, W.dt, 2, work)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qs.evolve(psi, W.dt, steps, work)
    e1.record()
    torch.cuda.synchronize()
    stage_s = e0.elapsed_time(e1) * 1e-3 / steps / 4
    hbm_gbs = 32.0 * qs.total / stage_s / 1e9
    achieved = 4.0 * terms / stage_s / 1e12
    out = {"workload": W.name + "_P0", "kets": qs.total, "terms_per_hpsi": terms, "stage_ms": stage_s * 1e3,
           "terms_per_s": terms / stage_s, "bound": "alu", "achieved_tflops_fp64_equiv": achieved,
           "peak_dfma_tflops": dfma_tflops, "frac": achieved / dfma_tflops,
           "hbm_GBps_algorithmic": hbm_gbs, "hbm_peak_GBps": peaks.get("hbm_gbs"),
           "hbm_frac": hbm_gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
           "bytes_per_ket_algorithmic": 32, "tile_shape": qs.tile_shape, "tuning": qs.tuning}
    del psi, work, qs
    torch.cuda.empty_cache()
    return out


def sweep_extra(qb, torch, steps: int = 3):
    """8-member coupling sweep on the M=11, N=20, P=0 sector (2,731,365 kets, number state
    (...,7,6,7,...), w=|p|, C_k = -0.005 k): one batched launch per stage for all 8
    members against the members one at a time."""
    W = wl.large_sector()
    qs = qb.Space(W.M, W.w, W.L, 20, 20, [0])
    terms = qs.terms()[0]
    B = len(W.sweep)
    psi = torch.empty((B, qs.total), dtype=torch.complex128, device="cuda")
    for b in range(B):
        qs.init_number(W.occ, psi[b])
    work = qs.workspace(B)
    qs.evolve_batch(psi, W.sweep, W.dt, 1, work)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    qs.evolve_batch(psi, W.sweep, W.dt, steps, work)
    e1.record()
    torch.cuda.synchronize()
    batched = e0.elapsed_time(e1) / steps
    one = psi[0].clone()
    w1 = qs.workspace(1)
    e0.record()
    for b in range(B):
        qs.evolve_batch(one, [W.sweep[b]], W.dt, steps, w1)
    e1.record()
    torch.cuda.synchronize()
    separate = e0.elapsed_time(e1) / steps
    out = {"workload": W.name + "_sweep8", "kets": qs.total, "members": B, "terms_per_hpsi": terms,
           "batched_ms_per_step": batched, "separate_ms_per_step": separate,
           "batched_member_terms_per_s": 4 * terms * B / (batched * 1e-3),
           "separate_member_terms_per_s": 4 * terms * B / (separate * 1e-3), "batched_speedup": separate / batched}
    del psi, work, one, w1, qs
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qb", choices=["qb", "reference"])
    ap.add_argument("--config", default="batched_coherent")
    ap.add_argument("--n-tot", type=int, default=16, help="mean occupation of the batched coherent workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint and sweep measurements")
    ap.add_argument("--breaktime-sweep", action="store_true",
                    help="run only the breaktime scaling experiment (Sec. IV C-D) and print its JSON line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    import paper_2111_00050_gb300 as qb

    if args.breaktime_sweep:
        if rank == 0:
            print(json.dumps(breaktime_sweep(qb, torch)))
        return
    W, sp = workload(args.config, args.n_tot)
    t_setup = time.perf_counter()
    qs = qb.Space(W.M, W.w, W.L, sp["n_min"], sp["n_max"], sp["p_list"])
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    terms, tuples = qs.terms()
    psi = qs.empty_state()
    torch.cuda.synchronize()
    ei0, ei1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ei0.record()
    init_state(qs, W, psi)
    ei1.record()
    torch.cuda.synchronize()
    init_ms = ei0.elapsed_time(ei1)
    work = qs.workspace(1)
    resident_max = qs.autotune(W.dt, psi, steps=1, work=work)
    for _ in range(args.warmup):
        qs.evolve(psi, W.dt, 1, work)
    torch.cuda.synchronize()

    # ---- timed region: K RK4 steps of the whole state
    stream = torch.cuda.current_stream()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    qs.evolve(psi, W.dt, args.steps, work)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist is not None:
        ms = max_over_ranks(dist, ms, "cuda")
        dist.barrier()
    clocks = clk.stop()
    ms_step = ms / args.steps
    value = job_throughput(world, 4 * terms, ms_step)
    steps_per_s = 1e3 / ms_step

    # ---- dominant kernel: one fused RK4 stage == one H psi over all sectors; a step is
    # four launches of it, timed above with CUDA events on the launching stream
    stage_time = ms_step * 1e-3 / 4
    flops = 4.0 * terms  # >= 2 FP64 FMA per term (real coefficient x complex amplitude)
    achieved = flops / stage_time / 1e12
    peaks = _peaks()
    # algorithmic bytes per ket and stage, averaged over the four stages of a step: the
    # gathered input (16 B), the diagonal (16 B), the output (16 B), the psi copy of the
    # inner stages (16 B, d = 3, 2) and the FP64 psi read + write of the last (32 B)
    hbm_bytes = (48.0 + 64.0 + 64.0 + 80.0) / 4 * qs.total
    # FP64 H psi (qb_hpsi) for comparison with the double-float stage
    out = qs.empty_state()
    qs.hpsi(psi, out)
    torch.cuda.synchronize()
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record(stream)
    qs.hpsi(psi, out)
    b_ev.record(stream)
    torch.cuda.synchronize()
    fp64_ms = a_ev.elapsed_time(b_ev)
    del out
    dfma_tflops = qb.api.measure_fp64_fma(3)
    roofline = {
        "bound": "alu", "achieved": achieved, "peak": dfma_tflops, "unit": "TFLOP/s",
        "frac": achieved / dfma_tflops, "peak_kind": "measured DFMA rate of this GPU (qb_measure_fp64_fma)",
        "peak_unit_count": FP64_PEAK_TFLOPS, "frac_of_unit_count": achieved / FP64_PEAK_TFLOPS,
        "traffic": STAGE_DRAM_BYTES_PER_KET * qs.total if args.config == "batched_coherent" else None,
        "kernel": f"stage_df_kernel<{W.M},1,0,0,1,{qs.tile_shape}> (one RK4 stage = one H psi over all sectors, weighted basis)",
        "stage_ms": stage_time * 1e3,
        "peak_note": "FP64-equivalent flops (2 FMA/term) vs the FP64 FMA rate measured on this GPU; the "
                     "kernel itself runs double-float on the FP32/ALU pipes (FP64 pipe idle), so frac > 1 "
                     "is its speed-up over native FP64; traffic scaled from an ncu capture at n_tot=12",
        "hbm_GBps": hbm_bytes / stage_time / 1e9, "hbm_peak_GBps": peaks.get("hbm_gbs"),
        "hbm_frac": (hbm_bytes / stage_time / 1e9) / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
        "fp64_hpsi_ms": fp64_ms,
        "ncu_issue_active": STAGE_NCU_ISSUE_ACTIVE if args.config == "batched_coherent" else None,
        "ncu_l1_data_pipe": STAGE_NCU_L1_WAVEFRONTS if args.config == "batched_coherent" else None,
        "ncu_note": "issue-slot and L1/shared data-pipe wavefront utilisation of the stage kernel from the "
                    "ncu capture at n_tot=12 (profiles/stage_df_kernel_batched_coherent_ntot12.md)",
    }

    # ---- plain path: one launch per sector per stage, same workload and arithmetic
    k_plain = max(1, min(args.steps, 3))
    e0p, e1p = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0p.record(stream)
    qs.evolve_plain(psi, W.dt, k_plain, work)
    e1p.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0p.elapsed_time(e1p) / k_plain
    plain = {"ms_per_step": plain_ms, "terms_per_s": 4 * terms / (plain_ms * 1e-3), "steps": k_plain,
             "launches_per_step": 4 * qs.n_sectors, "batched_speedup": plain_ms / ms_step}

    # ---- the second-order Taylor step of Sec. III B (two stage launches per step)
    qs.set_order(2)
    qs.evolve(psi, W.dt, 1, work)
    e0t, e1t = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0t.record(stream)
    qs.evolve(psi, W.dt, k_plain, work)
    e1t.record(stream)
    torch.cuda.synchronize()
    qs.set_order(4)
    t2_ms = e0t.elapsed_time(e1t) / k_plain
    taylor2 = {"ms_per_step": t2_ms, "steps_per_s": 1e3 / t2_ms, "terms_per_s": 2 * terms / (t2_ms * 1e-3),
               "steps": k_plain}

    # ---- end to end through the public API with host buffers: every step copies its
    # input state from pinned host memory (on a copy stream, into the buffer the
    # previous step is not using, so that the copy of step k+1 overlaps step k),
    # runs one RK4 step and reads the observables back to the host
    host_in = torch.empty(qs.total, dtype=torch.complex128).pin_memory()
    host_in.copy_(psi.cpu())
    bufs = [psi, torch.empty_like(psi)]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    # one untimed pass first: the first call of a kernel pays its module load and
    # launch-attribute set-up
    bufs[1].copy_(host_in, non_blocking=True)
    qs.evolve(bufs[1], W.dt, 1, work)
    qs.observables(bufs[1])
    torch.cuda.synchronize()
    k_e2e = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    with torch.cuda.stream(copy_stream):
        bufs[0].copy_(host_in, non_blocking=True)
        ready[0].record(copy_stream)
    for k in range(k_e2e):
        cur = bufs[k % 2]
        if k + 1 < k_e2e:
            with torch.cuda.stream(copy_stream):
                bufs[(k + 1) % 2].copy_(host_in, non_blocking=True)
                ready[(k + 1) % 2].record(copy_stream)
        torch.cuda.current_stream().wait_event(ready[k % 2])
        qs.evolve(cur, W.dt, 1, work)
        ob = qs.observables(cur)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / k_e2e
    psi = bufs[(k_e2e - 1) % 2]
    del bufs
    if dist is not None:  # replicas: the job's step is its slowest rank's
        e2e_s = max_over_ranks(dist, e2e_s, "cuda")
    nmom = 4 + 2 * W.M + 4 * W.M * W.M
    e2e = {"value": job_throughput(world, 4 * terms, e2e_s * 1e3), "unit": "terms/s",
           "h2d_bytes_per_step": 16 * qs.total,
           "d2h_bytes_per_step": 8 * nmom + 8 * 2, "steps_per_s": 1.0 / e2e_s,
           "note": "per step: H2D of psi from pinned memory (copy stream, overlapping the previous step), "
                   "one RK4 step, qb_observables (moments D2H, host sync)"}

    # ---- the other rows of the path, each timed once: sector build + device tables (host
    # wall clock), initial state, one observables call, observation steps + breaktime,
    # the mean-field trajectory of the workload's full length
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qs.observables(psi)
    obs_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    series = qs.evolve_observe(psi, W.dt, 2, 1, work)
    torch.cuda.synchronize()
    evobs_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    bt = qb.breaktime([o["Q"] for o in series], W.dt, 0.1)
    bt_us = (time.perf_counter() - t0) * 1e6
    t0 = time.perf_counter()
    qb.meanfield(W.M, W.w, W.L, W.z if W.z is not None else np.sqrt(W.occ), W.dt, W.steps, W.obs_every)
    mf_ms = (time.perf_counter() - t0) * 1e3
    rows = {"sector_build_and_tables_s": setup_s, "init_state_ms": init_ms,
            "observables_ms": obs_ms, "observables_kets_per_s": qs.total / (obs_ms * 1e-3),
            "evolve_observe_2_steps_3_obs_ms": evobs_ms, "breaktime_us": bt_us, "breaktime_flag": bt[1],
            "meanfield_ms": mf_ms, "meanfield_steps": W.steps}
    # kernel launches of the timed call: four stage launches per step, the weighted copy,
    # and the resident kernel when some sector is small enough
    resident = resident_max > 0 and int(qs.dims[0]) <= resident_max  # leading sectors run resident
    launches = 4 * args.steps + 1 + (1 if resident else 0)

    line = {
        "metric": "H_psi_terms_per_s", "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 (H psi in double-float: fp32 pairs)", "data": "synthetic",
        "config": {"workload": W.name, "kets": qs.total, "sectors": qs.n_sectors, "terms_per_hpsi": terms,
                   "ordered_tuples_per_hpsi": tuples, "dt": W.dt, "rk4_steps_per_s": steps_per_s,
                   "l2": "state (16 B/ket, %.2f GB) larger than L2; no flush" % (16 * qs.total / 1e9),
                   "resident_max_kets": resident_max, "tile_shape": qs.tile_shape, "tuning": qs.tuning,
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "rk4_steps_per_s": steps_per_s,
        "plain_per_sector": plain,
        "taylor2": taylor2,
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roofline,
        "e2e": e2e,
        "path_rows": rows,
    }
    line["large_sector_roofline"] = None
    if not args.no_extras:
        del work, psi
        torch.cuda.empty_cache()
        line["large_sector_roofline"] = large_sector_roofline(qb, torch, peaks, dfma_tflops)
        line["adjoint"] = adjoint_extra(qb, torch)
        line["sweep"] = sweep_extra(qb, torch)
        line["small_sector"] = small_extra(qb, torch)
        line["exact_momentum"] = exact_extra(qb, torch)
        line["long_range"] = long_range_extra(qb, torch)
        line["squeezing"] = squeezing_extra(qb, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
