"""Throughput of the batched ROS4 chemistry integrator on GB300 (one JSON line on stdout).

A step = one pass of the batched hot path over the whole workload.  The default workload is the
batched flame-front configuration: the 111-species / 784-reaction synthetic mechanism on
262,144 cells (90% relaxed products, 10% ignition-front cells), 20 consecutive operator-split
steps of dt = 1e-6 s (h carried from step to step) captured once as a CUDA graph and replayed
per bench step, adaptive ROS4 in FP64 at rtol 1e-6 / atol 1e-10, in the kernel configuration the
library's autotuner picks on a sample of the cells (autotune time reported, not timed).  Inputs
are restored before every step and L2 is flushed (a 512 MiB write); steps are timed with CUDA
events on the launching stream.  value = cell split-steps per second.

Beside the timed line: the plain one-launch-per-attempt GPU driver on the same inputs, the same
workload end to end from pinned host arrays through chem_integrate_host, the 53-species forward
workload (65,536 cells, one split step), the discrete adjoint on the 53-species ignition
workload and on the 111-species workload under a stated HBM budget, FP64 roofline figures
against an in-run FMA-chain peak and the cuBLAS float64 GEMM, and the CPU oracle on the host
cores (a bounded sample).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

--impl reference times the CPU oracle (the plain FP64 C++ reference written from the paper) on
a bounded sample of the same workload on the host cores.
Under torchrun (N > 1) every rank integrates its own copy of the workload (replicas, no
collective on the data path); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MECH_DIR = os.path.join(ROOT, "paper_2205_05681_gb300", "_cache", "mechs")
METRIC = "cells integrated/s (ROS4, FP64, rtol 1e-6) vs plain GPU kernel; adjoint/fwd time"


# stages and evaluations of f per attempt of each Rosenbrock method: (s, f evaluations incl. f(y))
METHOD_SHAPE = {0: (4, 3), 1: (3, 2), 2: (4, 3), 3: (6, 6), 4: (6, 6), 5: (2, 2)}  # (stages, f evaluations)
EXPLICIT = {4}  # RKF45: no Jacobian, no factorisation, no solves
METHODS = ["ROS4", "ROS3", "RODAS3", "RODAS4", "RKF45", "ROS2W"]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one chem_integrate_k launch on the
# full bench workload, from a single-pass ncu capture; valid only for the device source they were
# taken on (sha1 of csrc/ros4_device.cuh), reported as null once that source changes.
MEASURED_TRAFFIC = {"device_src_sha1": "4ff7f10b7da918bc04f1b55c6db25a30a4a18cc9",
                    "ch4_111_batched": 250775808 + 204967680}


def measured_traffic(wl, full_size):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2205_05681_gb300",
                       "csrc", "ros4_device.cuh")
    sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    if not full_size or sha != MEASURED_TRAFFIC["device_src_sha1"]:
        return None
    return MEASURED_TRAFFIC.get(wl)


def algorithmic_flops_per_attempt(spec, tableau=0):
    """FP64 operations of one step attempt by the algorithm's own operation counts, with the
    transcendentals counted separately (returned as a dict of exp and log calls):
      LU 2N^3/3, s triangular solves 2N^2 each, the Jacobian's dense chain-rule pass 6N^2,
      and per evaluation of f: thermo 27 per species, 4 + 2*(orders) + 2*(species entries) per
      reaction (+2 per efficiency entry and +2 for third-body/falloff reactions, +12 for the
      falloff blend, +40 for Troe); the Jacobian adds per reaction 2 p^2 + 10 (+2 per efficiency
      entry x participant) for its p participants.  RKF45: six evaluations of f and the stage
      combinations only.  ROS4 evaluates f at 3 points (stage 4 reuses stage 3's argument).
      Transcendentals per evaluation of f: one exp per species (equilibrium factor) and per
      reaction (forward rate constant), one more per falloff reaction (low-pressure limit), and
      for Troe reactions three exp (the blending terms, two without T**) plus the final exp and
      two log10; one log of T."""
    s, nf = METHOD_SHAPE[tableau]
    N = spec["ns"]
    fl = 0.0 if tableau in EXPLICIT else 2.0 * N ** 3 / 3.0 + s * 2.0 * N ** 2 + 6.0 * N ** 2
    f_eval = 27.0 * N
    jac = 0.0
    n_exp, n_log = N, 1
    for r in spec["reactions"]:
        nre, npr = sum(r["rnu"]), sum(r["pnu"])
        f_eval += 4 + 2 * (nre + npr) + 2 * (len(r["rnu"]) + len(r["pnu"]))
        n_exp += 1
        if r["kind"] != "ELEM":
            f_eval += 2 * r["neff"] + 2
        if r["kind"] in ("LIND", "TROE"):
            f_eval += 12
            n_exp += 1
        if r["kind"] == "TROE":
            f_eval += 40
            n_exp += 3 + (1 if r.get("t2", 0.0) > 0.0 else 0)
            n_log += 2
        p = len(r["rnu"]) + len(r["pnu"])
        jac += 2 * p * p + 10 + (2 * r["neff"] * p if r["kind"] != "ELEM" else 0)
    if tableau in EXPLICIT:
        jac = 0.0
        fl += 2.0 * s * N  # the stage combinations
    total = fl + nf * f_eval + jac
    return total, {"exp": nf * n_exp, "log": nf * n_log}


def read_spec_counts(path):
    ns = 0
    rx = []
    for line in open(path):
        t = line.split()
        if not t:
            continue
        if t[0] == "SPECIES":
            ns = int(t[1])
        elif t[0] == "R":
            p = 2
            nre = int(t[p]); rnu = [int(t[p + 2 + 2 * i]) for i in range(nre)]; p += 1 + 2 * nre
            npr = int(t[p]); pnu = [int(t[p + 2 + 2 * i]) for i in range(npr)]
            rx.append({"kind": t[1], "rnu": rnu, "pnu": pnu, "neff": 0})
        elif t[0] == "EFF":
            rx[-1]["neff"] = int(t[1])
        elif t[0] == "TROE":
            rx[-1]["t2"] = float(t[4])
    return {"ns": ns, "reactions": rx}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def fp64_peak_tflops(torch, dev):
    """Measured FP64 peak of this GPU: float64 GEMM (cuBLAS) 4096^3, best of 5."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * n ** 3 / best / 1e12


_ORACLE_INPUTS = {}


def cpu_oracle_rate(path, wl, budget_s=15.0, max_cells=4096, tableau=0, rtol=1e-6, atol=1e-10):
    """Oracle cells/s (cells x split steps per second) on the host cores, on a bounded, evenly
    strided sample of the workload.  For the flame-front workload the oracle relaxes its own
    product templates first (as the GPU leg does), untimed."""
    from oracle import oracle as O
    from paper_2205_05681_gb300 import synth
    mech_name, n_cells, recipe, seed, dt, splits = synth.WORKLOADS[wl]
    if (path, wl) not in _ORACLE_INPUTS:  # the oracle's mechanism and the states, once per process
        _ORACLE_INPUTS[(path, wl)] = (O.Mechanism(path), synth.make_states(
            synth.mechanism(mech_name), n_cells, recipe, seed))
    om, st = _ORACLE_INPUTS[(path, wl)]
    cores = os.cpu_count() or 1

    def sample_states(idx):
        """The sample's states and pressures; for the flame-front workload its product cells take
        the state and pressure of one of 8 product templates relaxed for 1e-3 s (the first 8
        product cells of the workload, relaxed once per process), as the GPU leg tiles its own."""
        y = om.state_from_TY(st.T[idx], st.Y[idx])
        P = st.P[idx].copy()
        if recipe == "ch4_front":
            prod = np.where(st.T[idx] >= 1500.0)[0]
            if len(prod):
                key = ("templates", path, wl)
                if key not in _ORACLE_INPUTS:
                    tid = np.where(st.T >= 1500.0)[0][:8]
                    yt, _ = om.integrate(om.state_from_TY(st.T[tid], st.Y[tid]), st.P[tid], 1e-3,
                                         threads=cores)
                    _ORACLE_INPUTS[key] = (yt, st.P[tid].copy())
                yt, Pt = _ORACLE_INPUTS[key]
                src = np.arange(len(prod)) % len(yt)
                y[prod] = yt[src]
                P[prod] = Pt[src]
        return y, P

    def run(idx, yP):
        y, P = yP
        hh = np.zeros(len(idx))
        for _ in range(splits):
            y, info = om.integrate(y, P, dt, rtol=rtol, atol=atol, h=hh, threads=cores,
                                   tableau=tableau)
            hh = info["h"]
        return y

    # calibrate on a small sample, then size the timed sample to ~budget_s
    idx = np.arange(0, n_cells, max(1, n_cells // (2 * cores)))[: 2 * cores]
    y = sample_states(idx)
    t0 = time.perf_counter()
    run(idx, y)
    per = (time.perf_counter() - t0) / len(idx)
    ns = int(min(max_cells, n_cells, max(len(idx), budget_s / max(per, 1e-9))))
    idx = np.linspace(0, n_cells - 1, ns).astype(int)
    y = sample_states(idx)
    reps = 0  # a small workload is repeated until ~2 s have passed
    t0 = time.perf_counter()
    while True:
        run(idx, y)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min(2.0, budget_s) or reps >= 1000:
            break
    return {"value": reps * ns * splits / el, "cores": cores, "seconds": el, "cells": ns,
            "repeats": reps,
            "sample": "%d of %d cells (evenly strided) x %d split steps%s, %.1f s on %d host threads" % (
                ns, n_cells, splits, "" if reps == 1 else " x %d repeats" % reps, el, cores)}


def relax_products(m, st, T0, P, Y0, torch, np, n_templates=1024, t_relax=1e-3):
    """Near-equilibrium cells of the flame-front workload: 1,024 template product states are
    relaxed on the GPU for 1e-3 s (input preparation, untimed) and tiled over the product cells
    with a 1e-9 relative perturbation of the mass fractions."""
    front = st.T < 1500.0
    idx = np.where(~front)[0]
    if len(idx) == 0:
        return {}
    k = min(n_templates, len(idx))
    tid = idx[:k]
    Tt, Pt = T0[tid].clone(), P[tid].clone()
    Yt = Y0[:, tid].clone().contiguous()
    t0 = time.perf_counter()
    m.integrate(Tt.contiguous(), Pt.contiguous(), Yt, t_relax)
    torch.cuda.synchronize()
    rel_s = time.perf_counter() - t0
    src = torch.tensor(np.arange(len(idx)) % k, device=T0.device)
    dst = torch.tensor(idx, device=T0.device)
    rng = np.random.default_rng(12)
    noise = torch.tensor(1.0 + 1e-9 * rng.standard_normal((Y0.shape[0], len(idx))), device=T0.device)
    T0[dst] = Tt[src]
    P[dst] = Pt[src]
    Ynew = Yt[:, src] * noise
    Y0[:, dst] = Ynew / Ynew.sum(0, keepdim=True)
    return {"relaxed_templates": k, "relax_time_s": t_relax, "relax_wall_s": rel_s,
            "front_cells": int(front.sum()), "product_cells": int(len(idx))}


def adjoint_leg(chem, synth, torch, np, dev, wl="ch4_53_adjoint", cells=0, cap=4096,
                interval=16, hbm_budget_gib=None):
    """Checkpointed forward + discrete adjoint on an adjoint workload: loss = sum (T - T_target)^2
    with T_target from a seeded ln A perturbation + noise; times the taped forward, the untaped
    forward and the reverse sweep (CUDA events), after an untimed call on a few cells that loads
    the adjoint module.  Reports the tape and adjoint-workspace bytes against hbm_budget_gib."""
    mech_name, n, recipe, seed, dt, _ = synth.WORKLOADS[wl]
    if cells:
        n = min(n, cells)
    st = synth.make_states(synth.mechanism(mech_name), synth.WORKLOADS[wl][1], recipe, seed)
    st = synth.States(st.T[:n], st.P[:n], st.Y[:n])
    m = chem.Mechanism(synth.mechanism_file(mech_name, MECH_DIR))
    T0 = torch.tensor(st.T, device=dev)
    P = torch.tensor(st.P, device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(st.Y.T), device=dev)
    rng = np.random.default_rng(seed)
    lnA = torch.tensor(m.lnA(), device=dev)
    lnA_t = lnA + torch.tensor(rng.normal(0.0, 0.1, m.nr), device=dev)
    Tt, Yt = T0.clone(), Y0.clone()
    m.integrate(Tt, P, Yt, dt, opts=m.opts(lnA=lnA_t))
    T_target = Tt + torch.tensor(rng.normal(0.0, 1.0, n), device=dev)
    # untimed: compile and load the adjoint module on a few cells
    k = min(n, 4)
    tw = m.make_tape(k, cap, interval, device=dev)
    Tw, Yw = T0[:k].clone(), Y0[:, :k].contiguous()
    m.integrate_ckpt(Tw, P[:k].contiguous(), Yw, dt * 1e-3, tw)
    m.adjoint(P[:k].contiguous(), torch.ones_like(Tw), torch.zeros_like(Yw), tw)
    del tw
    tape = m.make_tape(n, cap, interval, device=dev)
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    status = torch.empty(n, dtype=torch.int32, device=dev)
    T, Y = T0.clone(), Y0.clone()
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)
    e0, e1 = ev()
    e0.record()
    m.integrate_ckpt(T, P, Y, dt, tape, status=status, opts=m.opts(lnA=lnA))
    e1.record()
    e1.synchronize()
    t_fwd = e0.elapsed_time(e1)
    gT = 2.0 * (T - T_target)
    gY = torch.zeros_like(Y)
    ws_bytes = int(m._lib.chem_adjoint_workspace(m._h, n, chem.C.byref(m.opts(lnA=lnA)), interval))
    e0, e1 = ev()
    e0.record()
    g_lnA, gT0, gY0 = m.adjoint(P, gT, gY, tape, opts=m.opts(lnA=lnA))
    e1.record()
    e1.synchronize()
    t_adj = e0.elapsed_time(e1)
    peak = torch.cuda.max_memory_allocated(dev) - base
    T2, Y2 = T0.clone(), Y0.clone()
    e0, e1 = ev()
    e0.record()
    m.integrate(T2, P, Y2, dt, opts=m.opts(lnA=lnA))
    e1.record()
    e1.synchronize()
    t_plain = e0.elapsed_time(e1)
    nacc = tape.n_accepted().float()
    res = {"workload": wl, "mechanism": mech_name, "cells": n, "dt_s": dt, "interval": interval,
           "capacity": cap, "fwd_ckpt_ms": t_fwd, "fwd_ms": t_plain, "adjoint_ms": t_adj,
           "adjoint_over_fwd": t_adj / t_plain, "tape_bytes": int(tape.buf.numel()),
           "adjoint_workspace_bytes": ws_bytes,
           "peak_bytes_during_sweep": int(peak),
           "accepted_mean": float(nacc.mean().item()), "accepted_max": int(nacc.max().item()),
           "ok_cells": int((status == 0).sum().item()),
           "loss": float(((T - T_target) ** 2).sum().item()),
           "grad_lnA_norm": float(g_lnA.norm().item()),
           "temperature_rise_K": {"p50": float((T - T0).median().item()),
                                  "max": float((T - T0).max().item())}}
    if hbm_budget_gib is not None:
        need = res["tape_bytes"] + ws_bytes
        res["hbm_budget_bytes"] = int(hbm_budget_gib * 2 ** 30)
        res["within_budget"] = bool(need <= res["hbm_budget_bytes"])
    return res


def reduce_max_seconds(sec, world, device=None):
    """Max of the per-rank step time over all ranks (the slowest replica sets the job time)."""
    if world == 1:
        return sec
    import torch
    import torch.distributed as dist
    t = torch.tensor([sec], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_value(cells_per_rank, splits, world, sec):
    """Whole-job throughput: every rank integrates its own replica of the workload."""
    return cells_per_rank * splits * world / sec


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(wl, args, world):
    """The `config` dict of a workload, identical on the GPU arm and the reference arm."""
    from paper_2205_05681_gb300 import synth
    mech_name, n_cells, recipe, seed, dt, splits = synth.WORKLOADS[wl]
    spec = read_spec_counts(synth.mechanism_file(mech_name, MECH_DIR))
    if args.cells:
        n_cells = min(n_cells, args.cells)
    if getattr(args, "splits", 0):
        splits = args.splits
    method = METHODS[args.tableau]
    if getattr(args, "switching", ""):
        method = "per-cell %s / %s" % ({"rkf45": "RKF45", "w": "ROS2W"}[args.switching], method)
    return {"workload": wl, "mechanism": mech_name, "species": spec["ns"],
            "reactions": len(spec["reactions"]), "cells": n_cells, "recipe": recipe,
            "state_seed": seed, "dt_s": dt, "split_steps_per_step": splits,
            "method": method, "cuda_graph": splits > 1, "rtol": args.rtol,
            "atol": args.atol, "l2": "flushed (512 MiB write) between steps",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on the host cores; each step integrates a
    bounded, evenly strided sample of the workload's cells (sized to ~60 s / steps of CPU work)
    and the step's value is the sample's cells x split steps per second."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from paper_2205_05681_gb300 import synth
    from oracle import oracle as O
    O.build()
    wl = args.workload
    mech_name, n_cells, recipe, seed, dt, splits = synth.WORKLOADS[wl]
    path = synth.mechanism_file(mech_name, MECH_DIR)
    runs = []
    kw = dict(tableau=args.tableau, rtol=args.rtol, atol=args.atol)
    for _ in range(args.warmup):
        cpu_oracle_rate(path, wl, budget_s=3.0, **kw)
    for _ in range(args.steps):
        runs.append(cpu_oracle_rate(path, wl, budget_s=max(3.0, 60.0 / max(args.steps, 1)), **kw))
    vals = [r["value"] for r in runs]
    v = statistics.median(vals)
    r0 = runs[len(runs) // 2]
    cfg = workload_config(wl, args, world)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            # the measured time of one step: the sample that step integrated
            "ms_per_step": statistics.median(r["seconds"] for r in runs) * 1e3,
            "ms_per_step_extrapolated_to_workload": cfg["cells"] * splits / v * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": r0["cores"],
                             "kind": "oracle", "sample": r0["sample"]},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def work_precision(args, chem, synth, torch, np, dev):
    """Work-precision study of the four Rosenbrock methods, in the manner of the paper's solver
    verification (Sec. 3.1): rtol = atol = tol for tol in 1e-4 .. 1e-12; per IVP the error norm
    of Eq. (e:ivp_norm), sqrt(mean_i (|y°_i - y_i| / (1e-10 + 1e-6 |y°_i|))^2) over [T, Y_k],
    and its maximum over the IVPs, Eq. (e:error_norm).  y° is RODAS4 at rtol = atol = 1e-14 on
    the same cells (the paper used CVODEs; a reference from the same integrator at a much tighter
    tolerance, whose agreement with the CPU oracle the parity tests establish).
    Time: CUDA events around one chem_integrate call over all `cells` cells."""
    mech_name, n_all, recipe, seed, dt, _ = synth.WORKLOADS["ch4_53_fwd"]
    path = synth.mechanism_file(mech_name, MECH_DIR)
    n = min(args.cells or 4096, n_all)
    st = synth.make_states(synth.mechanism(mech_name), n, recipe, seed)
    m = chem.Mechanism(path)
    T0 = torch.tensor(st.T, device=dev)
    P = torch.tensor(st.P, device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(st.Y.T), device=dev)
    att = torch.zeros(n, dtype=torch.int32, device=dev)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    o = m.opts(attempts=att, tableau=3)
    ws = m.workspace(n, o, device=dev)
    Tr, Yr = T0.clone(), Y0.clone()
    t0 = time.perf_counter()
    m.integrate(Tr, P, Yr, dt, rtol=1e-14, atol=1e-14, status=status, opts=o, workspace=ws)
    torch.cuda.synchronize()
    ref_s = time.perf_counter() - t0
    ref_ok = status == 0
    ref = np.concatenate([Tr.cpu().numpy()[:, None], Yr.cpu().numpy().T], axis=1)
    del ws
    rows = []
    for tab, name in enumerate(METHODS[:4]):
        o = m.opts(attempts=att, tableau=tab)
        ws = m.workspace(n, o, device=dev)
        for e in range(4, 13):
            tol = 10.0 ** -e
            times = []
            for rep in range(2):  # the first run also compiles the method's module
                T, Y = T0.clone(), Y0.clone()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.integrate(T, P, Y, dt, rtol=tol, atol=tol, status=status, opts=o, workspace=ws)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            got = np.concatenate([T.cpu().numpy()[:, None], Y.cpu().numpy().T], axis=1)
            ej = np.sqrt(np.mean((np.abs(ref - got) / (1e-10 + 1e-6 * np.abs(ref))) ** 2, axis=1))
            ok = (ref_ok & (status == 0)).cpu().numpy()
            rows.append({"method": name, "tol": tol, "error": float(ej[ok].max()),
                         "ms": float(times[-1]), "attempts_mean": float(att.float().mean()),
                         "ok_cells": int((status == 0).sum())})
        del ws
    return {"metric": "work-precision (Eqs. e:ivp_norm, e:error_norm) of ROS4/ROS3/RODAS3/RODAS4",
            "value": None, "unit": "error norm vs ms", "n_gpus": 1, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "ch4_53_fwd", "cells": n, "error_cells": int(ref_ok.sum()),
                       "dt_s": dt,
                       "reference": "RODAS4, rtol = atol = 1e-14, same cells (%.1f s)" % ref_s},
            "work_precision": rows}


DEFAULT_WORKLOAD = "ch4_111_batched"


def prepare_inputs(m, synth, torch, np, dev, wl, cells=0):
    """Device copies of the workload's seeded states (T0, P, Y0 [Ns, C]); for the flame-front
    workload the product cells are first relaxed (untimed)."""
    mech_name, n_cells, recipe, seed, dt, splits = synth.WORKLOADS[wl]
    st = synth.make_states(synth.mechanism(mech_name), n_cells, recipe, seed)
    if cells:
        n_cells = min(n_cells, cells)
        st = synth.States(st.T[:n_cells], st.P[:n_cells], st.Y[:n_cells])
    T0 = torch.tensor(st.T, device=dev)
    P = torch.tensor(st.P, device=dev)
    Y0 = torch.tensor(np.ascontiguousarray(st.Y.T), device=dev)
    prep = {}
    if recipe == "ch4_front":
        prep = relax_products(m, st, T0, P, Y0, torch, np)
    return T0, P, Y0, prep


def forward_run(m, chem, torch, np, dev, T0, P, Y0, dt, splits, steps, warmup, rtol, atol,
                tableau=0, clocks_index=None, world=1, plain=True, plain_runs=1, cost_order=False,
                switching=False, light_precapture=False):
    """Times `steps` bench steps (each: restore inputs, flush L2, `splits` split steps, graph-
    captured when splits > 1) after `warmup` untimed ones; optionally the plain driver on the
    same inputs.  cost_order: from the second split step on, the work queue hands out the cells
    by decreasing attempts of the previous split step (chem_cost_order, inside the graph).
    switching: per-cell switching between RKF45 and the Rosenbrock method, the method array
    carried from split step to split step (reset with the inputs).  light_precapture: the
    untimed run before graph capture (which loads every module the graph launches) integrates
    only the first 256 cells.  Returns a dict of times (s), attempts per cell, the cells that
    ended on the explicit method, and the clock summary."""
    n_cells = T0.shape[0]
    T, Y = T0.clone(), Y0.clone()
    h = torch.zeros(n_cells, dtype=torch.float64, device=dev)
    status = torch.zeros(n_cells, dtype=torch.int32, device=dev)
    att = torch.zeros(n_cells, dtype=torch.int32, device=dev)
    att_total = torch.zeros(n_cells, dtype=torch.int32, device=dev)
    meth = torch.zeros(n_cells, dtype=torch.int32, device=dev)
    # the W-method's factorisation cache (the W-method itself, or the W-method as the switching
    # alternative)
    alt = 5 if switching == "w" else 4
    jc = m.jac_cache(n_cells, device=dev) if (tableau == 5 or alt == 5) else None
    opts = m.opts(attempts=att, tableau=tableau, cell_method=meth if switching else None,
                  jac_cache=jc, alt_tableau=alt if switching else 0)
    ws = m.workspace(n_cells, opts, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def restore():
        T.copy_(T0)
        Y.copy_(Y0)
        h.zero_()
        meth.zero_()
        if jc is not None:
            jc.zero_()
        flush.fill_(1.0)  # evict the inputs from L2 (512 MiB > 129 MB)

    def one_split(o=opts, w=ws):
        m.integrate(T, P, Y, dt, rtol=rtol, atol=atol, h=h, status=status, opts=o, workspace=w)

    order = torch.arange(n_cells, dtype=torch.int32, device=dev)
    ows = torch.empty(int(m._lib.chem_cost_order_workspace()) + 256, dtype=torch.uint8, device=dev)
    ows = ows[(256 - ows.data_ptr() % 256) % 256:]
    oopts = m.opts(attempts=att, tableau=tableau, order=order,
                   cell_method=meth if switching else None, jac_cache=jc,
                   alt_tableau=alt if switching else 0)

    if splits > 1:
        # consecutive split steps (h carried) captured once as a CUDA graph and replayed
        def splits_body():
            att_total.zero_()
            for sp in range(splits):
                one_split(oopts if (cost_order and sp > 0) else opts)
                att_total.add_(att)
                if cost_order and sp + 1 < splits:
                    m.cost_order(att, order, ows)

        restore()
        s_cap = torch.cuda.Stream()
        s_cap.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s_cap):
            if light_precapture:  # load the modules on a few cells
                k = min(256, n_cells)
                Tk, Pk, Yk = T0[:k].clone(), P[:k].clone(), Y0[:, :k].contiguous()
                mk = torch.zeros(k, dtype=torch.int32, device=dev)
                jk = m.jac_cache(k, device=dev) if jc is not None else None
                ok = m.opts(tableau=tableau, cell_method=mk if switching else None, jac_cache=jk,
                            alt_tableau=alt if switching else 0)
                m.integrate(Tk, Pk, Yk, dt, rtol=rtol, atol=atol, opts=ok,
                            workspace=m.workspace(k, ok, device=dev))
                if switching:  # and the alternative method's module
                    mk.fill_(64)
                    m.integrate(Tk, Pk, Yk, dt, rtol=rtol, atol=atol, opts=ok,
                                workspace=m.workspace(k, ok, device=dev))
                m.cost_order(att[:k].contiguous())
            else:
                splits_body()  # eager run on the capture stream before capture
        torch.cuda.current_stream().wait_stream(s_cap)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            splits_body()

        def one_step():
            graph.replay()
    else:
        if switching:  # load the alternative method's module before timing
            mk = torch.full((min(256, n_cells),), 64, dtype=torch.int32, device=dev)
            k = mk.shape[0]
            jk = m.jac_cache(k, device=dev) if jc is not None else None
            ok = m.opts(tableau=tableau, cell_method=mk, jac_cache=jk,
                        alt_tableau=alt if switching else 0)
            m.integrate(T0[:k].clone(), P[:k].clone(), Y0[:, :k].contiguous(), dt, rtol=rtol,
                        atol=atol, opts=ok, workspace=m.workspace(k, ok, device=dev))

        def one_step():
            one_split()
            att_total.copy_(att)

    for _ in range(warmup):
        restore()
        one_step()
    torch.cuda.synchronize()
    times = []
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(clocks_index if clocks_index is not None else 0) as clk:
        for _ in range(steps):
            restore()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) * 1e-3)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # this library's kernels per bench step: the integrator per split step; with switching also
    # the routing and fall-back kernels and the alternative method's integrator; with the cost
    # order the three sorting kernels between split steps
    per_split = 4 if switching else 1
    launches = splits * per_split + (3 * (splits - 1) if (cost_order and splits > 1) else 0)
    res = {"times": times, "attempts": att_total.cpu().numpy(),
           "ok_cells": int((status == 0).sum().item()), "clocks": clk.summary(),
           "explicit_cells": int((meth > 0).sum().item()) if switching else 0,
           "launches_per_step": launches}
    if plain:
        # the plain one-launch-per-attempt driver on the same inputs (split steps run eagerly: its
        # host polling cannot be captured in a graph); one run, its kernels are already loaded
        po = m.opts(mode=chem.MODE_PLAIN, tableau=tableau)
        pws = m.workspace(n_cells, po, device=dev)
        pt = []
        for _ in range(plain_runs):
            restore()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(splits):
                one_split(po, pws)
            e1.record(stream)
            e1.synchronize()
            pt.append(e0.elapsed_time(e1) * 1e-3)
        res["plain_s"] = min(pt)
        del pws
    del ws, flush, ows, meth, jc
    return res


def roofline(spec, tableau, total_attempts, sec, probe, dgemm, sm_mhz, n_sm, wl, full_size,
             n_cells, launches):
    """FP64-ALU roofline of chem_integrate_k over the timed region."""
    fl, trans = algorithmic_flops_per_attempt(spec, tableau)
    achieved = fl * total_attempts / sec / 1e12
    folded = (fl + 2.0 * (trans["exp"] * probe["exp_cost"] + trans["log"] * probe["log_cost"]))
    achieved_t = folded * total_attempts / sec / 1e12
    peak = probe["dfma_tflops"]
    N = spec["ns"]
    traffic = measured_traffic(wl, full_size and tableau == 0)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_source": "FMA-chain probe (chem_fp64_probe) on this GPU in this run",
            "peak_dgemm": dgemm, "frac_vs_dgemm": achieved / dgemm,
            "peak_derived_from_clock": (n_sm * 4.0 * sm_mhz * 1e6 / 1e12) if sm_mhz else None,
            "peak_derived_note": "SMs x 2 FP64 lanes per clock x 2 flops x median SM clock",
            "achieved_with_transcendentals": achieved_t,
            "frac_with_transcendentals": achieved_t / peak,
            "transcendental_cost_fma": {"exp": probe["exp_cost"], "log": probe["log_cost"]},
            "traffic": traffic,
            "traffic_source": ("ncu single-pass capture summarised in profiles/, device-source "
                               "hash matched" if traffic is not None else None),
            "traffic_unit": "bytes per launch (one split step)",
            "algorithmic_bytes_per_launch": int(8 * n_cells * (2 * (N + 1) + 3)),
            "kernel": "chem_integrate_k", "launches": launches,
            "flops_per_attempt": fl, "transcendentals_per_attempt": trans,
            "note": ("W-method: the Jacobian and factorisation are counted on every attempt, "
                     "an upper bound (attempts that reuse the cached factorisation skip them)"
                     if tableau == 5 else None)}


def attempts_summary(a, ok):
    return {"total": int(a.sum()), "mean": float(a.mean()), "p50": float(np.percentile(a, 50)),
            "p99": float(np.percentile(a, 99)), "max": int(a.max()),
            "max_over_p50": float(a.max() / max(np.percentile(a, 50), 1)), "ok_cells": ok}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--team", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-kernel comparison")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 53-species forward and the two adjoint legs")
    ap.add_argument("--cells", type=int, default=0,
                    help="use only the first CELLS cells of the workload (small profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default kernel configuration instead of autotuning")
    ap.add_argument("--tape-capacity", type=int, default=4096, help="adjoint workloads: steps/cell")
    ap.add_argument("--interval", type=int, default=16, help="adjoint workloads: checkpoint interval")
    ap.add_argument("--tableau", type=int, default=0,
                    help="method: 0 ROS4 (default), 1 ROS3, 2 RODAS3, 3 RODAS4, 4 RKF45 (explicit), "
                         "5 ROS2W (W-method with factorisation reuse)")
    ap.add_argument("--rtol", type=float, default=1e-6)
    ap.add_argument("--atol", type=float, default=1e-10)
    ap.add_argument("--splits", type=int, default=0,
                    help="override the workload's split steps per bench step (graph-captured)")
    ap.add_argument("--switching", default="", choices=["", "rkf45", "w"],
                    help="per-cell switching on the timed leg between the Rosenbrock method and "
                         "RKF45 (stiffness rule) or the W-method ROS2 (quiescent cells)")
    ap.add_argument("--cost-order", action="store_true",
                    help="cost-ordered work queue on the timed leg (split steps after the first)")
    ap.add_argument("--work-precision", action="store_true",
                    help="error vs time of the four Rosenbrock methods over tolerances 1e-4..1e-12")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2205_05681_gb300 import chem, synth
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    wl = args.workload
    if args.work_precision:
        if rank == 0:
            print(json.dumps(work_precision(args, chem, synth, torch, np, dev)), flush=True)
        return 0
    if wl.endswith("_adjoint"):
        res = adjoint_leg(chem, synth, torch, np, dev, wl=wl, cells=args.cells,
                          cap=args.tape_capacity, interval=args.interval)
        if rank == 0:
            line = {"metric": "adjoint/forward time (discrete adjoint, ROS4, FP64)",
                    "value": res["adjoint_over_fwd"], "unit": "x", "n_gpus": world,
                    "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                    "config": {"workload": wl}, "adjoint": res}
            print(json.dumps(line), flush=True)
        return 0
    mech_name, n_all, recipe, seed, dt, splits = synth.WORKLOADS[wl]
    if args.splits:
        splits = args.splits
    path = synth.mechanism_file(mech_name, MECH_DIR + ("" if world == 1 else "_r%d" % rank))
    t0 = time.perf_counter()
    m = chem.Mechanism(path, team=args.team, block=args.block)
    load_s = time.perf_counter() - t0
    T0, P, Y0, prep = prepare_inputs(m, synth, torch, np, dev, wl, args.cells)
    n_cells = T0.shape[0]

    tuned = None
    if not args.no_autotune and not args.team:
        t0 = time.perf_counter()
        tuned = m.autotune(T0, P, Y0, dt)
        tuned["autotune_wall_s"] = time.perf_counter() - t0

    run = forward_run(m, chem, torch, np, dev, T0, P, Y0, dt, splits, args.steps, args.warmup,
                      args.rtol, args.atol, tableau=args.tableau, clocks_index=local,
                      world=world, plain=not args.no_plain, switching=args.switching,
                      cost_order=args.cost_order)
    sec = reduce_max_seconds(sum(run["times"]) / len(run["times"]), world, dev)
    value = whole_job_value(n_cells, splits, world, sec)
    attempts = run["attempts"]

    # end to end: pinned host arrays through chem_integrate_host (H2D copies of T, P, Y, h, the
    # integration and D2H copies of T, Y, h, status inside the timed region; one host call per
    # split step, h carried on the host), same inputs as the device-resident leg
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    srcT, srcY = T0.cpu().numpy(), Y0.cpu().numpy()
    Th, Ph, Yh = pinned(srcT), pinned(P.cpu().numpy()), pinned(srcY)
    hh = pinned(np.zeros(n_cells))
    sh = pinned(np.zeros(n_cells, dtype=np.int32))
    ho = m.opts(tableau=args.tableau)
    e2e_t = []
    n_e2e = 0 if args.no_e2e else (max(1, min(args.steps, 3)) if splits == 1 else 1)
    for i in range(n_e2e + 1 if n_e2e else 0):
        Th[:] = srcT
        Yh[:] = srcY
        hh[:] = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(splits if i else 1):  # the untimed first pass sizes the library's buffers
            m.integrate_host(Th, Ph, Yh, dt, rtol=args.rtol, atol=args.atol, h=hh, status=sh,
                             opts=ho)
        el = time.perf_counter() - t0
        if i:
            e2e_t.append(el)
    e2e_sec = statistics.median(e2e_t) if e2e_t else float("nan")

    extra = {}
    full = not args.cells and world == 1
    if full and not args.no_extra and splits > 1 and not (args.switching or args.cost_order):
        if args.tableau < 4:
            # quiescent cells moved to the W-method, whose factorisation serves their next split
            # steps (stiffness-aware switching; ROS4 keeps the reacting cells)
            rs = forward_run(m, chem, torch, np, dev, T0, P, Y0, dt, splits, 1, 0, args.rtol,
                             args.atol, tableau=args.tableau, clocks_index=local, plain=False,
                             switching="w", light_precapture=True)
            s_s = statistics.median(rs["times"])
            extra["method_switching"] = {"alternative": "ROS2W with factorisation reuse",
                                         "value": n_cells * splits / s_s, "unit": "cells/s",
                                         "ms_per_step": s_s * 1e3,
                                         "speedup_over_single_method": sec / s_s,
                                         "cells_on_alternative_at_end": rs["explicit_cells"],
                                         "attempts_mean": float(rs["attempts"].mean()), "steps": 1,
                                         "ok_cells": rs["ok_cells"]}
    if full and not args.no_extra and wl == DEFAULT_WORKLOAD and args.tableau == 0:
        # the 53-species forward workload (one split step over 65,536 cells)
        wl2 = "ch4_53_fwd"
        mn2, _, _, _, dt2, sp2 = synth.WORKLOADS[wl2]
        m2 = chem.Mechanism(synth.mechanism_file(mn2, MECH_DIR))
        a0, p2, b0, _ = prepare_inputs(m2, synth, torch, np, dev, wl2)
        r2 = forward_run(m2, chem, torch, np, dev, a0, p2, b0, dt2, sp2, 3, 1, args.rtol,
                         args.atol, clocks_index=local)
        s2 = statistics.median(r2["times"])
        extra["forward_53"] = {"workload": wl2, "cells": a0.shape[0], "value": a0.shape[0] / s2,
                               "unit": "cells/s", "ms_per_step": s2 * 1e3,
                               "plain_value": a0.shape[0] / r2["plain_s"],
                               "speedup_over_plain": r2["plain_s"] / s2,
                               "kernel": m2.kernel_config(),
                               "attempts": attempts_summary(r2["attempts"], r2["ok_cells"]),
                               "_spec": read_spec_counts(m2.spec_path), "_sec": s2}
        del a0, p2, b0, m2
        torch.cuda.empty_cache()
        extra["adjoint"] = adjoint_leg(chem, synth, torch, np, dev, wl="ch4_53_adjoint",
                                       cap=args.tape_capacity, interval=args.interval)
        torch.cuda.empty_cache()
        extra["adjoint_111"] = adjoint_leg(chem, synth, torch, np, dev, wl="ch4_111_adjoint",
                                           cap=1024, interval=args.interval, hbm_budget_gib=64)
        torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    spec = read_spec_counts(path)
    probe = chem.fp64_probe()
    dgemm = fp64_peak_tflops(torch, dev)
    props = torch.cuda.get_device_properties(dev)
    clk = run["clocks"]
    rl = roofline(spec, args.tableau, float(attempts.sum()), sec, probe, dgemm, clk.get("sm_mhz"),
                  props.multi_processor_count, wl, full, n_cells, splits)
    if args.switching:
        # the attempts mix two methods (an attempt of the alternative is not a Rosenbrock attempt)
        # and the integrator launches cover subsets of the cells: no flop rate or traffic applies
        for k in ("achieved", "frac", "frac_vs_dgemm", "achieved_with_transcendentals",
                  "frac_with_transcendentals", "traffic", "traffic_source"):
            rl[k] = None
        rl["note"] = ("per-cell switching: attempts of two methods, no flop rate derived; the "
                      "single-method run carries the roofline")
    if "forward_53" in extra:
        f53 = extra["forward_53"]
        r53 = roofline(f53.pop("_spec"), 0, float(f53["attempts"]["total"]), f53.pop("_sec"),
                       probe, dgemm, clk.get("sm_mhz"), props.multi_processor_count, "ch4_53_fwd",
                       True, f53["cells"], 1)
        f53["roofline"] = {k: r53[k] for k in ("achieved", "peak", "frac", "frac_vs_dgemm",
                                                "frac_with_transcendentals", "traffic",
                                                "traffic_source")}
    cpu = None
    if not args.no_cpu:
        from oracle import oracle as O
        O.build()
        r = cpu_oracle_rate(path, wl, tableau=args.tableau, rtol=args.rtol, atol=args.atol)
        cpu = {"value": r["value"], "unit": "cells/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"]}
    N = spec["ns"]
    cfg = workload_config(wl, args, world)
    kcfg = m.kernel_config(m.opts(tableau=args.tableau))
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "kernel": {"team": kcfg["team"], "block": kcfg["block"], "smem_bytes": kcfg["smem"],
                   "regs": kcfg["regs"], "autotuned": tuned is not None},
        "roofline": rl,
        "attempts": attempts_summary(attempts, run["ok_cells"]),
        "plain_gpu": None if "plain_s" not in run else {
            "value": n_cells * splits / run["plain_s"], "unit": "cells/s",
            "ms_per_step": run["plain_s"] * 1e3, "speedup_of_persistent": run["plain_s"] / sec},
        "autotuned": tuned,
        "input_prep": prep or None,
        "e2e": None if not e2e_t else {
            "value": n_cells * splits / e2e_sec, "unit": "cells/s",
            "h2d_bytes_per_step": int(splits * 8 * n_cells * (2 + N + 1)),
            "d2h_bytes_per_step": int(splits * (8 * n_cells * (1 + N + 1) + 4 * n_cells)),
            "host_memory": "pinned", "host_calls_per_step": splits},
        "cpu_baseline": cpu,
        "gpu_launches": args.steps * run["launches_per_step"],
        "clocks": clk,
        "mech_load_s": load_s,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
