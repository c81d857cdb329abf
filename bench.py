#!/usr/bin/env python
"""Benchmark of the EOFA hot path on GB300.

Workload: the paper-shaped lattice 24^3 x 64, Ls = 24 (the 24ID volume of
Table 1), Moebius alpha = 2 (c = 1, d = 1/2), M5 = 1.8, synthetic
strange-like mass pair m1 = 0.0362, m2 = 1.0, seeded synthetic SU(3) links
exp(i 0.7 sum_a h_a lambda_a) (seed 3) and a Gaussian pseudofermion.

One step = one EOFA pseudofermion force evaluation (Sec. 3.3, Eq. (7)),
the operation that dominates an EOFA trajectory (Table 4): the two
Cayley / even-odd preconditioned solves of Eq. (8) for chi_L and chi_R in
mixed precision (FP32 inner CG, FP64 reliable updates) to a true residual of
1e-10, the action value of Eq. (5) and the force kernel.

value = whole-job dslash bandwidth: algorithmic bytes of every even-odd
dslash (hop) launched in the timed steps, summed over ranks, divided by the
slowest rank's time.  The roofline object reports the hop kernel itself
(average duration from CUDA events recorded around each launch on its
stream during the timed steps).  "solve" compares the same chi_L solve in
mixed precision and in plain FP64 on the GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DWF dslash GB/s (% HBM roofline); EOFA solve time mixed vs FP64 at 1e-10"
WORKLOAD = dict(dims=(24, 24, 24, 64), Ls=24, alpha=2.0, M5=1.8, m1=0.0362, m2=1.0, eps=0.7, seed=3, bc=-1)
SMALL = dict(dims=(8, 8, 8, 8), Ls=8, alpha=2.0, M5=1.8, m1=0.0362, m2=1.0, eps=0.7, seed=3, bc=-1)
FALLBACK_HBM_GBS = 6800.0


def hop_bytes_per_site(prec: int, Ls: int) -> float:
    """Algorithmic bytes per output 5D site of one even-odd hop: one input and one
    output spinor plus 8 links amortised over Ls (FP16: FP32 per-site scale, FP32 links)."""
    if prec == 0:
        return 192 + 192 + 8 * 144 / Ls
    if prec == 1:
        return 96 + 96 + 8 * 72 / Ls
    return (48 + 4) + (48 + 4) + 8 * 72 / Ls


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    v = d[key]
                    return float(v["burst"] if isinstance(v, dict) and "burst" in v else v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [ln.strip().split(", ") for ln in open(self.f.name) if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(U, wl, cg_iters=2):
    """The oracle (plain FP64 C restatement of D_w, D_DWF and CGNR, oracle/c) on the host cores.

    Timed: one D_w on the whole lattice with every core, the same on a 2-slice
    sample with one core, and cg_iters CGNR iterations on D_DWF (Eq. (3)) with
    every core, reported per iteration.  GB/s counts the same algorithmic
    bytes per 5D site as the GPU's FP64 hop."""
    import numpy as np

    from oracle import c_oracle
    from paper_1611_00298_gb300 import inputs

    X, Y, Z, T = wl["dims"]
    Ls = wl["Ls"]
    V = X * Y * Z * T
    bps = hop_bytes_per_site(0, Ls)
    cores = c_oracle.threads()
    psi = inputs.fermion5d(wl["dims"], Ls, wl["seed"], stream=9)
    t0 = time.perf_counter()
    c_oracle.wilson(U, psi, wl["M5"], wl["bc"])
    t_all = time.perf_counter() - t0
    c_oracle.set_threads(1)
    try:
        sample = np.ascontiguousarray(psi[:2])
        t0 = time.perf_counter()
        c_oracle.wilson(U, sample, wl["M5"], wl["bc"])
        t_one = time.perf_counter() - t0
    finally:
        c_oracle.set_threads(cores)
    _, it, _, t_cg = c_oracle.cgnr_dwf(U, psi, wl["alpha"], wl["M5"], wl["m1"], wl["bc"], tol=1e-30,
                                       maxiter=cg_iters, timing=True)
    del np
    return {"value": round(V * Ls * bps / t_all / 1e9, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "single_core_GBs": round(V * 2 * bps / t_one / 1e9, 4),
            "cg_iteration_seconds": round(t_cg / max(1, it), 3), "cg_iterations_timed": it,
            "sample": f"C oracle (oracle/c/dwf_oracle.c, gcc -O2, OpenMP): D_w on the whole {X}x{Y}x{Z}x{T} x "
                      f"Ls={Ls} lattice with {cores} threads ({t_all:.2f} s); the same on 2 of {Ls} s-slices "
                      f"with 1 thread ({t_one:.2f} s); {it} CGNR iterations on D_DWF (m_f={wl['m1']}) with "
                      f"{cores} threads, {t_cg:.2f} s in total; bytes counted as for the FP64 hop"}


def run_reference(args, wl, rank):
    """The oracle on the host cores, per step one D_w on the whole lattice (all cores)."""
    if rank != 0:
        return 0
    from oracle import c_oracle
    from paper_1611_00298_gb300 import inputs
    U = inputs.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    psi = inputs.fermion5d(wl["dims"], wl["Ls"], wl["seed"], stream=9)
    X, Y, Z, T = wl["dims"]
    nbytes = X * Y * Z * T * wl["Ls"] * hop_bytes_per_site(0, wl["Ls"])
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        c_oracle.wilson(U, psi, wl["M5"], wl["bc"])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = nbytes * len(times) / sum(times) / 1e9
    cores = c_oracle.threads()
    cb = {"value": round(v, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
          "sample": f"C oracle D_w on the whole {X}x{Y}x{Z}x{T} x Ls={wl['Ls']} lattice per step, {cores} threads"}
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * sum(times) / len(times), 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl), "cpu_baseline": cb,
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fp64_peak_bench(args, wl):
    """FP64 FMA rate of the GPU (probe kernel, CUDA events) and the FP64 hop's flop rate against it."""
    import torch

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    peak = eofa.probe_fp64_fma()
    U = inputs.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    lat = eofa.Lattice(wl["dims"], wl["Ls"], bc_t=wl["bc"])
    lat.gauge_load(U)
    del U
    canon = torch.randn(lat.V * wl["Ls"] * 24, dtype=torch.float64, device="cuda")
    nb = lat.field_bytes(0)
    e = torch.empty(nb, dtype=torch.uint8, device="cuda")
    o = torch.empty_like(e)
    out = torch.empty_like(e)
    lat.pack_dev(0, canon, e, o)
    del canon
    for _ in range(3):
        lat.hop_dev(0, 0, 0, o, out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.hop_reps):
        lat.hop_dev(0, 0, 0, o, out)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.hop_reps
    n5h = lat.V // 2 * wl["Ls"]
    tf = 1320.0 * n5h / (ms / 1000) / 1e12
    print(json.dumps({"fp64_fma_tflops": round(peak, 3), "fp64_hop_ms": round(ms, 3), "fp64_hop_tflops": round(tf, 3),
                      "fp64_hop_frac_of_measured_fma": round(tf / peak, 3),
                      "lattice": "x".join(map(str, wl["dims"])), "Ls": wl["Ls"],
                      "flops_per_site": 1320}), flush=True)
    lat.close()
    return 0


def hop_only(args, wl):
    """Launch the even-odd hop alone on a random field (profiling target)."""
    import torch

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    prec = {"f64": 0, "f32": 1, "f16": 2}[args.hop_precision or args.precision]
    U = inputs.gauge_field(wl["dims"], wl["eps"], wl["seed"])
    lat = eofa.Lattice(wl["dims"], wl["Ls"], bc_t=wl["bc"])
    lat.gauge_load(U)
    canon = torch.randn(lat.V * wl["Ls"] * 24, dtype=torch.float64, device="cuda")
    nb = lat.field_bytes(prec)
    e = torch.empty(nb, dtype=torch.uint8, device="cuda")
    o = torch.empty_like(e)
    out = torch.empty_like(e)
    lat.pack_dev(prec, canon, e, o)
    del canon

    def one():
        if args.schur:
            lat.schur_hop_dev(prec, 0, 0, o, out, wl["alpha"], wl["M5"], wl["m1"])
        else:
            lat.hop_dev(prec, 0, 0, o, out)
    one()  # the first launch runs the tile autotuner
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.hop_reps):
        one()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.hop_reps
    n5h = lat.V // 2 * wl["Ls"]
    gbs = hop_bytes_per_site(prec, wl["Ls"]) * n5h / (ms / 1000) / 1e9
    print(json.dumps({"hop_only": True, "schur": args.schur, "dims": wl["dims"], "Ls": wl["Ls"],
                      "precision": args.hop_precision or args.precision,
                      "avg_ms": round(ms, 4), "GBs": round(gbs, 1), "kernel_version": kernel_version()}))
    lat.close()
    return 0


MD_WORKLOAD = dict(dims=(16, 16, 16, 32), Ls=12, eps=0.5, seed=4, alpha=2.0, M5=1.8, m1=0.04, m2=1.0, bc=-1)


def heatbath_bench(args):
    """phi = f(M_EOFA) eta, 12-pole Zolotarev f ~ x^-1/2 on [1e-3, 20], mixed F32 solves to 1e-10."""
    import torch

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    w = MD_WORKLOAD
    lat = eofa.Lattice(w["dims"], w["Ls"], bc_t=w["bc"])
    lat.gauge_load(inputs.gauge_field(w["dims"], w["eps"], w["seed"]))
    eta = torch.from_numpy(inputs.fermion4d(w["dims"], 9)).cuda()
    phi = torch.empty_like(eta)
    a0, al, be, err = eofa.rational_inv_sqrt(12, 1e-3, 20.0)
    out = {"heatbath": True, "lattice": "x".join(map(str, w["dims"])), "Ls": w["Ls"], "poles": 12,
           "interval": [1e-3, 20.0], "rational_max_rel_err": err}
    for forecast in (False, True):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = lat.heatbath_dev(eta, phi, w["alpha"], w["M5"], w["m1"], w["m2"], a0, al, be,
                                precision=eofa.PREC_MIXED_F32, tol=1e-10, forecast=forecast)
        torch.cuda.synchronize()
        key = "forecast" if forecast else "zero_guess"
        out[key] = {"seconds": round(time.perf_counter() - t0, 3), "iters": sum(i.iters for i in info),
                    "iters_per_solve": [i.iters for i in info]}
    out["iteration_ratio"] = round(out["forecast"]["iters"] / out["zero_guess"]["iters"], 3)
    print(json.dumps(out), flush=True)
    lat.close()
    return 0


def hmc_bench(args):
    """One trajectory (tau = 1) of H = tr P^2 + S_g(beta 5.7) + S_EOFA, nested QPQPQ, mixed F32 solves."""
    import torch

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    w = MD_WORKLOAD
    U = inputs.gauge_field(w["dims"], w["eps"], w["seed"])
    P0 = inputs.momenta(w["dims"], 5)
    phi = torch.from_numpy(inputs.fermion4d(w["dims"], 6)).cuda()
    lat = eofa.Lattice(w["dims"], w["Ls"], bc_t=w["bc"])
    out = {"hmc": True, "lattice": "x".join(map(str, w["dims"])), "Ls": w["Ls"], "beta": 5.7, "tau": 1.0,
           "integrator": "force-gradient QPQPQ"}
    kw = dict(alpha=w["alpha"], M5=w["M5"], m1=w["m1"], m2=w["m2"], precision=eofa.PREC_MIXED_F32, tol=1e-10,
              beta=5.7, integrator=eofa.INT_FG_QPQPQ, tau=1.0)
    lat.gauge_load(U)
    FL = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    FR = torch.empty_like(FL)
    lat.force_parts_dev(phi, FL, FR, w["alpha"], w["M5"], w["m1"], w["m2"], precision=eofa.PREC_MIXED_F32, tol=1e-10)
    # size of the two EOFA force terms (the L / R asymmetry behind split integration)
    rms = lambda F: float(torch.sqrt((F.abs() ** 2).sum(dim=(-1, -2)).mean()))  # noqa: E731
    out["force_rms"] = {"L": rms(FL), "R": rms(FR)}
    out["force_max"] = {"L": float(FL.abs().amax()), "R": float(FR.abs().amax())}
    for name, extra in (("nested", dict(nsteps=4, n_inner=2)),
                        ("split_R_outer", dict(nsteps=4, n_middle=1, n_inner=2, split_lr=1)),
                        ("split_L_outer", dict(nsteps=4, n_middle=1, n_inner=2, split_lr=2))):
        lat.gauge_load(U)
        P = torch.from_numpy(P0).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = lat.hmc_trajectory_dev(P, phi, None, **kw, **extra)
        torch.cuda.synchronize()
        out[name] = dict(extra, seconds=round(time.perf_counter() - t0, 3), dH=info["dH"],
                         fermion_forces=info["fermion_forces"], gauge_forces=info["gauge_forces"],
                         solver_iters=info["solver_iters"])
    print(json.dumps(out), flush=True)
    lat.close()
    return 0


def hmc_chain_bench(args):
    """HMC Markov chain: pure-gauge thermalisation, then EOFA trajectories with heatbath refresh
    and Metropolis; acceptance and <exp(-dH)> (Sec. 3, Sec. 5; Table 3 analogue)."""
    import numpy as np
    import torch

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    dims, Ls, beta = (8, 8, 8, 8), 8, 5.7
    # the random start relaxes over a few hundred pure-gauge trajectories (cheap); the
    # plaquette must have stopped drifting before <exp(-dH)> means anything
    n_therm, n_traj = 600, args.chain_traj
    U = inputs.gauge_field(dims, 0.5, 41)
    lat = eofa.Lattice(dims, Ls, bc_t=-1)
    lat.gauge_load(U)
    Pth = torch.from_numpy(np.stack([inputs.momenta(dims, 42, stream=10 + k) for k in range(n_therm)])).cuda()
    uth = inputs.uniform(inputs.stream_key(42, 1), n_therm)
    t0 = time.perf_counter()
    th = lat.hmc_dev(Pth, None, uth, beta=beta, integrator=eofa.INT_FG_QPQPQ, nsteps=4, tau=1.0)
    t_therm = time.perf_counter() - t0
    dHg = np.array([i["dH"] for i in th[n_therm // 2:]])
    del Pth
    a0, al, be, err = eofa.rational_inv_sqrt(12, 1e-3, 20.0)
    kw = dict(alpha=2.0, M5=1.8, m1=0.04, m2=1.0, precision=eofa.PREC_MIXED_F32, tol=1e-10, beta=beta,
              integrator=eofa.INT_FG_QPQPQ, nsteps=4, tau=1.0, n_inner=2)

    def draws(n, seed):
        # momenta with density exp(-tr P^2); heatbath noise with density exp(-eta^+ eta), i.e. real and
        # imaginary parts N(0, 1/2) (fermion4d draws N(0, 1) parts), so that phi = f(M) eta has density
        # exp(-phi^+ M phi)
        Ps = torch.from_numpy(np.stack([inputs.momenta(dims, seed, stream=10 + k) for k in range(n)])).cuda()
        etas = torch.from_numpy(np.stack([inputs.fermion4d(dims, seed + 1, stream=10 + k) for k in range(n)])
                                / np.sqrt(2.0)).cuda()
        return Ps, etas, inputs.uniform(inputs.stream_key(seed + 2, 1), n)
    # the fermion changes the equilibrium: thermalise with it before measuring
    n_therm_f = args.chain_therm
    t0 = time.perf_counter()
    thf = lat.hmc_dev(*draws(n_therm_f, 50), rational=(a0, al, be), **kw)
    t_therm_f = time.perf_counter() - t0
    Ps, etas, us = draws(n_traj, 43)
    t0 = time.perf_counter()
    info = lat.hmc_dev(Ps, etas, us, rational=(a0, al, be), **kw)
    t_chain = time.perf_counter() - t0
    e = np.array([i["exp_minus_dH"] for i in info])
    dH = np.array([i["dH"] for i in info])
    out = {"hmc_chain": True, "lattice": "x".join(map(str, dims)), "Ls": Ls, "beta": beta, "m1": 0.04, "m2": 1.0,
           "alpha": 2.0, "integrator": "nested force-gradient QPQPQ (4 EOFA steps, 2 gauge steps each), tau = 1",
           "heatbath": f"12-pole Zolotarev x^-1/2 on [1e-3, 20], max rel err {err:.1e}",
           "thermalisation": {"trajectories": n_therm, "acceptance": float(np.mean([i["accepted"] for i in th])),
                              "plaquette_end": th[-1]["plaquette"],
                              "plaquette_last_100_mean": float(np.mean([i["plaquette"] for i in th[-100:]])),
                              "second_half_exp_minus_dH": float(np.exp(-dHg).mean()),
                              "second_half_exp_minus_dH_err": float(np.exp(-dHg).std(ddof=1) / np.sqrt(len(dHg))),
                              "second_half_dH_mean": float(dHg.mean()),
                              "seconds": round(t_therm, 2)},
           "thermalisation_with_eofa": {"trajectories": n_therm_f,
                                        "acceptance": float(np.mean([i["accepted"] for i in thf])),
                                        "dH": [round(i["dH"], 4) for i in thf], "seconds": round(t_therm_f, 2)},
           "trajectories": n_traj, "acceptance": float(np.mean([i["accepted"] for i in info])),
           "dH": [round(i["dH"], 4) for i in info],
           "exp_minus_dH_mean": float(e.mean()), "exp_minus_dH_err": float(e.std(ddof=1) / np.sqrt(len(e))),
           "dH_mean": float(dH.mean()), "dH_rms": float(np.sqrt(np.mean(dH ** 2))),
           "plaquette_mean": float(np.mean([i["plaquette"] for i in info])),
           "plaquette_halves": [float(np.mean([i["plaquette"] for i in info[:n_traj // 2]])),
                                float(np.mean([i["plaquette"] for i in info[n_traj // 2:]]))],
           "plaquette_eofa_thermalisation_halves": [float(np.mean([i["plaquette"] for i in thf[:n_therm_f // 2]])),
                                                    float(np.mean([i["plaquette"] for i in thf[n_therm_f // 2:]]))],
           "S_start_over_eta2": float(np.mean([i["S_eofa_start"] / i["eta_norm2"] for i in info])),
           "seconds_per_trajectory": round(t_chain / n_traj, 3),
           "solver_iters_per_trajectory": float(np.mean([i["solver_iters"] for i in info]))}
    print(json.dumps(out), flush=True)
    lat.close()
    return 0


def batched(args):
    """Three lattices x (3 mass pairs x {L, R} EOFA systems + 2 D_DWF systems) = 24 solves."""
    import numpy as np

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    lats, params, bs = [], [], []
    for dims, Ls, seed in (((8, 8, 8, 8), 8, 5), ((12, 12, 12, 12), 12, 6), ((16, 16, 16, 32), 16, 7)):
        lat = eofa.Lattice(dims, Ls)
        lat.gauge_load(inputs.gauge_field(dims, 0.5, seed))
        for m1, m2 in ((0.04, 0.2), (0.2, 0.6), (0.6, 1.0)):
            for system, shift in ((eofa.SYS_EOFA_L, 0.0), (eofa.SYS_EOFA_R, -1.0)):
                lats.append(lat)
                params.append(dict(system=system, alpha=2.0, M5=1.8, m1=m1, m2=m2, shift=shift))
                bs.append(inputs.fermion5d(dims, Ls, seed, stream=60 + len(bs)))
        for mf in (0.04, 0.2):
            lats.append(lat)
            params.append(dict(system=eofa.SYS_DWF, alpha=2.0, M5=1.8, mf=mf))
            bs.append(inputs.fermion5d(dims, Ls, seed, stream=60 + len(bs)))
    xs = [np.zeros_like(b) for b in bs]

    def run_batched(prec):
        ps = [lat.solve_params(precision=prec, tol=1e-10, **kw) for lat, kw in zip(lats, params)]
        t0 = time.perf_counter()
        info = eofa.solve_batched(lats, ps, bs, xs)
        return time.perf_counter() - t0, info

    def run_sequential(prec):
        t0 = time.perf_counter()
        its = []
        for lat, kw, b in zip(lats, params, bs):
            _, inf = lat.solve(b, precision=prec, tol=1e-10, **kw)
            its.append(inf.iters)
        return time.perf_counter() - t0, its

    for _ in range(max(1, args.warmup)):
        run_batched(eofa.PREC_MIXED_F32)
    tb = []
    for _ in range(args.steps):
        t, info = run_batched(eofa.PREC_MIXED_F32)
        tb.append(t)
    ts32, _ = run_sequential(eofa.PREC_MIXED_F32)
    ts64, its64 = run_sequential(eofa.PREC_F64) if not args.no_fp64 else (float("nan"), [])
    worst = max(i.true_resid for i in info)
    out = {"metric": "batched EOFA/DWF solves per second (24 solves, 3 lattices, true residual 1e-10)",
           "value": round(len(bs) / statistics.mean(tb), 3), "unit": "solves/s", "n_gpus": 1,
           "batched_mixed_f32_seconds": round(statistics.mean(tb), 4),
           "sequential_mixed_f32_seconds": round(ts32, 4), "sequential_fp64_seconds": round(ts64, 4),
           "fp64_sequential_over_batched": round(ts64 / statistics.mean(tb), 2) if not args.no_fp64 else None,
           "worst_true_resid": worst, "iters": [i.iters for i in info], "fp64_iters": its64,
           "config": {"workload": "8^4x8, 12^4x12, 16^3x32x16 (eps 0.5, seeds 5, 6, 7); mass pairs (0.04,0.2), "
                                  "(0.2,0.6), (0.6,1.0) x {L, R} + D_DWF at m_f 0.04, 0.2 per lattice"}}
    print(json.dumps(out), flush=True)
    return 0


def workload_config(wl):
    X, Y, Z, T = wl["dims"]
    return {"workload": f"EOFA force evaluation, {X}^3x{T} Ls={wl['Ls']} Moebius alpha={wl['alpha']} "
                        f"M5={wl['M5']} m1={wl['m1']} m2={wl['m2']}, synthetic links eps={wl['eps']} seed {wl['seed']}",
            "lattice": f"{X}x{Y}x{Z}x{T}", "Ls": wl["Ls"], "global_batch": 1,
            "what": "dslash GB/s: algorithmic bytes of the even-odd Wilson hops (one input and one output spinor "
                    "per 5D site, links once per 4D site) per second",
            "l2": "inputs larger than L2 (each FP32 half-checkerboard field is 1.02 GB)",
            "parallelism": "replicas (one independent lattice per GPU)"}


def replica_seed(seed, rank):
    """Each rank integrates its own independent lattice (replicas, no data-path collective)."""
    return seed + 100 * rank


def replica_totals(dist, elapsed, nbytes, device):
    """Whole-job figures over the ranks: the slowest rank's time and the summed bytes."""
    if dist is None:
        return elapsed, nbytes
    import torch
    t = torch.tensor([elapsed], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([nbytes], device=device, dtype=torch.float64)
    dist.all_reduce(b)
    return float(t.item()), float(b.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f16"])
    ap.add_argument("--cg-form", default="auto", choices=["auto", "five", "six"],
                    help="CG iteration form (auto: timed on the first solve)")
    ap.add_argument("--small", action="store_true", help="8^4 x 8 lattice (quick check)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 solve comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-cg-iters", type=int, default=2, help="CGNR iterations of the CPU oracle baseline")
    ap.add_argument("--hop-only", action="store_true",
                    help="only launch the even-odd hop kernel (for ncu captures); see --dims, --hop-reps")
    ap.add_argument("--dims", default=None, help="X,Y,Z,T override for --hop-only")
    ap.add_argument("--hop-reps", type=int, default=4)
    ap.add_argument("--schur", action="store_true", help="with --hop-only: the fused G^-1 D_hop kernel")
    ap.add_argument("--hop-precision", default=None, choices=["f64", "f32", "f16"])
    ap.add_argument("--heatbath", action="store_true",
                    help="EOFA heatbath (Eq. (6)) at 16^3x32, Ls=12: solver iterations and time with and without "
                         "chronological initial guesses")
    ap.add_argument("--hmc", action="store_true",
                    help="one nested force-gradient QPQPQ trajectory at 16^3x32, Ls=12 (EOFA + Wilson gauge), "
                         "one level and split L/R")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="measured FP64 FMA rate (the ALU roofline of the FP64 hop) and the FP64 hop against it")
    ap.add_argument("--hmc-chain", action="store_true",
                    help="HMC chain at 8^4, Ls=8: pure-gauge thermalisation, then EOFA trajectories with heatbath "
                         "refresh and Metropolis; acceptance and <exp(-dH)>")
    ap.add_argument("--chain-traj", type=int, default=24)
    ap.add_argument("--chain-therm", type=int, default=24, help="EOFA trajectories before the measured ones")
    ap.add_argument("--batched", action="store_true",
                    help="24 solves on three lattices (8^4x8, 12^4x12, 16^3x32x16): one batched, graph-captured "
                         "mixed-precision call vs sequential FP64 solves")
    args = ap.parse_args()
    wl = dict(SMALL if args.small else WORKLOAD)
    if args.dims:
        wl["dims"] = tuple(int(v) for v in args.dims.split(","))
    if args.hop_only:
        return hop_only(args, wl)
    if args.batched:
        return batched(args)
    if args.heatbath:
        return heatbath_bench(args)
    if args.hmc:
        return hmc_bench(args)
    if args.hmc_chain:
        return hmc_chain_bench(args)
    if args.fp64_peak:
        return fp64_peak_bench(args, wl)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, wl, rank)

    import numpy as np
    import torch

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    from paper_1611_00298_gb300 import build, eofa, inputs
    if not os.path.exists(eofa.LIB_PATH):
        build.build()
    eofa.load_library()

    prec = eofa.PREC_MIXED_F32 if args.precision == "f32" else eofa.PREC_MIXED_F16
    Ls = wl["Ls"]
    U = inputs.gauge_field(wl["dims"], wl["eps"], replica_seed(wl["seed"], rank))
    phi_np = inputs.fermion4d(wl["dims"], replica_seed(wl["seed"], rank))
    lat = eofa.Lattice(wl["dims"], Ls, bc_t=wl["bc"])
    lat.gauge_load(U)
    if args.cg_form != "auto":
        lat.set_cg_form(prec, eofa.CG_FORM_FIVE if args.cg_form == "five" else eofa.CG_FORM_SIX)
    phi = torch.from_numpy(phi_np).cuda()
    F = torch.empty(lat.shapeU, dtype=torch.complex128, device="cuda")
    kw = dict(alpha=wl["alpha"], M5=wl["M5"], m1=wl["m1"], m2=wl["m2"], precision=prec, tol=1e-10)
    n5h = lat.V // 2 * Ls

    def step():
        S, info = lat.force_dev(phi, F, **kw)
        return S, [info[0].as_dict(), info[1].as_dict()]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    clocks = ClockSampler(local_rank)
    l0 = eofa.kernel_launches()
    lat.profile_start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos, actions = [], []
    for _ in range(args.steps):
        S, inf = step()
        infos.append(inf)
        actions.append(S)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    launches = eofa.kernel_launches() - l0
    hop_launches, kind_ms, kind_bytes = lat.profile_stop()
    clk = clocks.stop()

    # algorithmic bytes counted per launch by the library (each spinor read /
    # written once, links once per 4D site, the axpy input when present)
    hop_bytes = sum(kind_bytes[p] for p in range(3))
    t_max, total_bytes = replica_totals(dist, elapsed, hop_bytes, "cuda")
    value = total_bytes / t_max / 1e9

    inner = 1 if prec == eofa.PREC_MIXED_F32 else 2
    avg_ms = kind_ms[inner] / max(1, hop_launches[inner])
    avg_bytes = kind_bytes[inner] / max(1, hop_launches[inner])
    achieved = avg_bytes / (avg_ms / 1000.0) / 1e9
    peak, peak_src = hbm_peak()
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "hop_traffic.json")
    if os.path.exists(tpath):
        try:
            td = json.load(open(tpath))
            key = f"{'fp32' if inner == 1 else 'fp16'}_solver_24x24x24x64_Ls24"
            if key in td and td[key].get("kernel_version") == kernel_version():
                traffic = td[key]["bytes_per_launch"]
        except Exception:
            traffic = None

    result = None
    if rank == 0:
        # end to end through the public host API: pinned host phi in, host F out
        phi_h = torch.from_numpy(phi_np.copy()).pin_memory()
        F_h = torch.empty(lat.shapeU, dtype=torch.complex128).pin_memory()
        lat.profile_start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lat.force(phi_h.numpy(), alpha=wl["alpha"], M5=wl["M5"], m1=wl["m1"], m2=wl["m2"], precision=prec,
                      tol=1e-10, out=F_h.numpy())
        torch.cuda.synchronize()
        e2e_t = (time.perf_counter() - t0) / args.steps
        _, _, b2 = lat.profile_stop()
        e2e_bytes = sum(b2[p] for p in range(3)) / args.steps
        e2e = {"value": round(e2e_bytes / e2e_t / 1e9, 2), "unit": "GB/s",
               "h2d_bytes_per_step": int(phi_np.nbytes), "d2h_bytes_per_step": int(F_h.numel() * 16 + 8),
               "seconds_per_step": round(e2e_t, 4)}

        mixed_s = statistics.mean(i[0]["seconds"] for i in infos)
        solve = {"system": "chi_L = H(m1)^-1 Omega_- P_- phi (Eq. (8), a = 0)",
                 f"mixed_{args.precision}_seconds": round(mixed_s, 4),
                 "mixed_iters": infos[-1][0]["iters"], "mixed_reliable_updates": infos[-1][0]["reliable_updates"],
                 "mixed_fp32_updates": infos[-1][0]["low_updates"],
                 "mixed_true_resid": infos[-1][0]["true_resid"]}
        if not args.no_fp64:
            b = torch.empty(lat.V * Ls * 12, dtype=torch.complex128, device="cuda")
            x = torch.zeros_like(b)
            # same right-hand side as chi_L: Omega_- P_- phi
            k, Op, Om = eofa.coefficients(Ls, wl["alpha"], wl["m1"], wl["m2"])
            bm = np.zeros(lat.shape5, dtype=np.complex128)
            bm[..., 2:, :] = Om[:, None, None, None, None, None, None] * phi_np[None, ..., 2:, :]
            b.copy_(torch.from_numpy(bm.reshape(-1)))
            info64 = lat.solve_dev(b, x, system=eofa.SYS_EOFA_L, alpha=wl["alpha"], M5=wl["M5"], m1=wl["m1"],
                                   m2=wl["m2"], shift=0.0, precision=eofa.PREC_F64, tol=1e-10)
            solve.update({"fp64_seconds": round(info64.seconds, 4), "fp64_iters": info64.iters,
                          "fp64_true_resid": info64.true_resid,
                          "fp64_over_mixed": round(info64.seconds / mixed_s, 3)})
        hop_share = kind_ms[inner] / 1000.0 / elapsed
        names = ["dslash_fp64", "dslash_fp32", "dslash_fp16", "local5_fp64", "local5_fp32", "local5_fp16"]
        by_kind = {names[k]: {"launches": hop_launches[k], "ms_per_step": round(kind_ms[k] / args.steps, 2),
                              "avg_launch_ms": round(kind_ms[k] / hop_launches[k], 4),
                              "GB/s": round(kind_bytes[k] / (kind_ms[k] / 1000.0) / 1e9, 1) if kind_bytes[k] else None}
                   for k in range(6) if hop_launches[k]}
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "kernel": f"fused even-odd dslash (hop + 5D-local + axpy), {'FP32' if inner == 1 else 'FP16'} "
                              "storage, all Ls slices",
                    "bytes_per_launch": int(avg_bytes), "avg_launch_ms": round(avg_ms, 4),
                    "launches_timed": hop_launches[inner], "share_of_step": round(hop_share, 4),
                    "peak_source": f"{peak_src} ({'of measured' if peak_src == 'measured' else 'of fallback'})"}
        result = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * t_max / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded SU(3) links and Gaussian pseudofermion; no ensemble)",
            "config": workload_config(wl),
            "solver": f"mixed {args.precision.upper()} inner CG, FP64 reliable updates, "
                      f"{ {0: 'five', 1: 'six'}.get(lat.cg_form(prec), 'undecided') }-launch iteration "
                      f"({'timed' if args.cg_form == 'auto' else 'forced'})",
            "roofline": roofline, "e2e": e2e, "solve": solve, "clocks": clk, "gpu_launches": int(launches),
            "timed_kernels": by_kind,
            "hop_launches_by_precision": {"fp64": hop_launches[0], "fp32": hop_launches[1], "fp16": hop_launches[2]},
            "action": actions[-1],
        }
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(U, wl, args.cpu_cg_iters)
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    lat.close()
    return 0


def kernel_version():
    """Hash of the dslash kernel sources, to invalidate stored ncu traffic when they change."""
    import hashlib
    h = hashlib.sha256()
    for f in ("dslash_impl.cuh", "dslash_bulk.cuh", "dslash_pipe.cuh", "field.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1611_00298_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
