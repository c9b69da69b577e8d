"""Benchmark of the HGKS hot path on one B300 (replicas on N GPUs).

Default workload: the jittered density-wave mesh of 48^3 cubes x 6 tetrahedra
(663,552 cells), inviscid, FP64, CFL 0.4.  One bench "step" is one full S2O4
step (time step, two stages of reconstruction, flux and update) of the whole
mesh.  Metric: cell-updates/s = cells x steps / device time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hgks|reference]
                    [--precision fp64|mixed]
                    [--workload densityN | densityNv | sphere | sphereN | transonic | transonicN
                                | hybrid | hybridN | prismN]
                    [--no-cpu-baseline] [--no-serve] [--serve]

densityN: N^3 x 6 tets (densityNv with mu = 1e-3, Pr = 0.72); sphere: the
1.51M-cell hex shell at Ma 0.2535, Re 300; sphereN: a 6 x N^2 x 1.3N shell;
transonic, transonicN: the same shells at Ma 1.5, Re 300; hybrid: the
1.46M-cell hex/prism shell 6 x 50^2 x 75 with 30% of its columns cut into
prisms, Ma 0.2535, Re 300; hybridN: 6 x N^2 x 1.3N likewise; prismN: the
density wave on N^3 x 2 jittered prisms.

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank advances its
own replica of the workload: the path has no exchange step on one GPU per
problem, so the job is weak-scaled replicas with no data-path collective.
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

# Executed operations per unit of the dominant kernels as built, from ncu
# operation counts (the profile summary of the flux and reconstruction counts
# under profiles/ gives the commands), and
# DRAM bytes per unit where a capture measured them.  "sha" is the digest of
# the kernel's sources (kernel_source_digest) that the counts were taken on:
# when they have changed since, the line carries "counts_stale": true and no
# traffic.
# Flops: binary64 2 dfma + dadd + dmul (FP64 path), binary32 2 ffma + fadd +
# fmul (mixed path), per launch divided by the units of the launch.
ROOF_TABLE = {
    ("k_flux", "fp64", 3, False): dict(unit="face", flop=4498, dram=478.5, sha="cffb70417c18",
                                       src="ncu operation counts and DRAM bytes on 48^3 x 6 tets"),
    ("k_flux", "fp64", 4, True): dict(unit="face", flop=12636, dram=541.9, sha="cffb70417c18",
                                      src="ncu operation counts and DRAM bytes on the 6 x 40^2 x 52 hex shell"),
    ("k_flux", "mixed", 3, False): dict(unit="face", flop=4368, dram=247.3, sha="cffb70417c18",
                                        src="ncu operation counts and DRAM bytes on 48^3 x 6 tets"),
    ("k_flux", "mixed", 4, True): dict(unit="face", flop=11739, dram=279.0, sha="cffb70417c18",
                                       src="ncu operation counts and DRAM bytes on the 6 x 40^2 x 52 hex shell"),
}
# DRAM bytes per cell of k_recon_rs as built, keyed by stencil shape (K, M,
# KM), for the traffic of its roofline
RECON_RS_DRAM = {
    (14, 4, 6): dict(bytes_per_cell=1118.7, sha="1f4f31a54f24", src="ncu DRAM bytes on 48^3 x 6 tets"),
    (24, 8, 3): dict(bytes_per_cell=1520.3, sha="1f4f31a54f24", src="ncu DRAM bytes on the 6 x 40^2 x 52 hex shell"),
}
# Algorithmic bytes per cell of one binary32 reconstruction launch (k_recon_rs):
# the cell's share of its block's binary32 record (pseudo-inverse rows
# 9K + 3 M KM, second moments and 1/h 7, sub-stencil positions M KM / 4 rows of
# 4 bytes per cell), stencil indices 4K, the cell's own 32-byte state record,
# and the 50 binary32 coefficients written.  Neighbour records are gathered
# through L2 and not counted.
def recon_rs_bytes_per_cell(K: int, M: int = 4, KM: int = 6) -> int:
    return (9 * K + 7 + M * KM // 4 + 3 * M * KM) * 4 + 4 * K + 32 + 50 * 4


FP64_PEAK_TFLOPS = 148 * 2 * 2 * 2.032e9 / 1e12  # SMs x DFMA/clk x 2 flop x max SM clock
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock


def kernel_source_digest(kernel: str = "k_flux") -> str:
    """Digest of the sources a kernel is built from (its device header, the
    shared device helpers and its host launcher)."""
    import hashlib

    files = {"k_flux": ("hgks_dev_common.cuh", "erfcx_table.h", "hgks_dev_flux.cuh", "hgks_flux.cu"),
             "k_recon_rs": ("hgks_dev_common.cuh", "hgks_dev_recon.cuh", "hgks_recon.cu")}[kernel]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2407_00656_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def recon_roofline(K: int, M: int, KM: int, cells: int, ms_per_launch: float, with_ghosts: bool):
    """roofline object of the binary32 reconstruction (k_recon_rs) from its
    algorithmic bytes; with_ghosts: the time includes the ghost fill that
    precedes each launch on meshes with boundaries (a lower bound on frac)."""
    per_launch = recon_rs_bytes_per_cell(K, M, KM) * cells
    ach = per_launch / (ms_per_launch * 1e-3) / 1e9
    r = {"bound": "hbm", "kernel": f"k_recon_rs<{K}, {M}, {KM}> (binary32)", "achieved": ach,
         "peak": HBM_PEAK_GBS, "unit": "GB/s", "frac": ach / HBM_PEAK_GBS, "bytes_per_launch": per_launch,
         "bytes_per_cell": recon_rs_bytes_per_cell(K, M, KM), "ms_per_launch": ms_per_launch,
         "peak_source": "MEASURED_PEAKS.json hbm_gbs", "traffic": None}
    if with_ghosts:
        r["time_includes"] = "the ghost fill before each launch"
    e = RECON_RS_DRAM.get((K, M, KM))
    if e and e["bytes_per_cell"] and e["sha"] == kernel_source_digest("k_recon_rs"):
        r["traffic"] = e["bytes_per_cell"] * cells
        r["traffic_source"] = e["src"]
    return r


def flux_roofline(precision: str, G: int, viscous: bool, faces: int, ms_per_launch: float):
    """roofline object of the flux kernel from the operation table."""
    peak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    r = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
         "kernel": f"k_flux ({'binary64' if precision == 'fp64' else 'binary32'}, {G} Gauss points, "
                   f"{'viscous' if viscous else 'inviscid'})",
         "peak_source": ("derived: 148 SMs x 2 DFMA/clk x 2 flop x 2.032 GHz" if precision == "fp64" else
                         "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz"),
         "achieved": None, "frac": None, "traffic": None, "ms_per_launch": ms_per_launch}
    e = ROOF_TABLE.get(("k_flux", precision, G, viscous))
    if e is None or not ms_per_launch:
        return r
    ach = e["flop"] * faces / (ms_per_launch * 1e-3) / 1e12
    r.update({"achieved": ach, "frac": ach / peak, "flop_per_launch": e["flop"] * faces,
              "flop_per_face": e["flop"], "counts_source": e["src"]})
    stale = e["sha"] != kernel_source_digest()
    r["counts_stale"] = stale
    if e["dram"] and not stale:
        r["traffic"] = e["dram"] * faces
        r["traffic_source"] = "ncu dram bytes per face of one launch, times the faces"
    return r


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6400.0  # fallback figure


HBM_PEAK_GBS = _hbm_peak()


def workload(name: str):
    from paper_2407_00656_b300 import inputs as I

    # densityN: the N^3 x 6 tet density wave, inviscid; densityNv: the same
    # with constant viscosity mu = 1e-3, Pr = 0.72
    body = name[len("density"):] if name.startswith("density") else ""
    visc = body.endswith("v")
    if body and body.rstrip("v").isdigit():
        n = int(body.rstrip("v"))
        jit = 0.15 if n != 8 else 0.0
        xyz, cells, per = I.kuhn_cube(n, jitter=jit, seed=0)
        q = I.density_wave_state(xyz, cells, 0.0)
        params = dict(mu_ref=1e-3, Pr=0.72, visc_exp=0.0, T_ref=1.0, tau_num_c=0.0) if visc else {}
        return dict(xyz=xyz, cells=cells, periods=per, q=q, params=params,
                    desc=f"density wave, {n}^3 x 6 tets" + (", jitter 0.15h seed 0" if jit else "") +
                    (", mu 1e-3 Pr 0.72" if visc else ", inviscid"))
    # prismN: the density wave on N^3 x 2 prisms, jittered, inviscid
    if name.startswith("prism") and name[len("prism"):].isdigit():
        n = int(name[len("prism"):])
        xyz, cells, per = I.prism_cube(n, jitter=0.15, seed=0)
        q = I.random_smooth_state(xyz, cells, seed=0)
        return dict(xyz=xyz, cells=cells, periods=per, q=q, params={},
                    desc=f"smooth state, {n}^3 x 2 prisms, jitter 0.15h seed 0, inviscid")
    # hybrid: the hex/prism shell of ~1.5M cells (30% of the columns cut into
    # prisms), Ma 0.2535, Re 300; hybridN: 6 x N^2 x round(1.3 N) columns
    if name == "hybrid" or (name.startswith("hybrid") and name[len("hybrid"):].isdigit()):
        size = name[len("hybrid"):]
        n, nr = (50, 75) if size == "" else (int(size), max(2, round(1.3 * int(size))))
        xyz, cells, bfn, bft = I.sphere_shell(n, nr, seed=0, prism_frac=0.3)
        qinf = I.free_stream(0.2535)
        q = np.tile(qinf, (len(cells), 1))
        return dict(xyz=xyz, cells=cells, periods=None, bfn=bfn, bft=bft, q=q,
                    params=dict(q_inf=qinf, mu_ref=0.2535 / 300, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
                                tau_num_c=1.0),
                    desc=f"hex/prism shell 6x{n}^2x{nr} columns, 30% cut into prisms, Ma 0.2535 Re 300, "
                         "wall + far field")
    # sphere: the 1.51M-cell shell 6 x 58^2 x 75 at Ma 0.2535, Re 300;
    # sphereN: 6 x N^2 x round(1.3 N); transonic, transonicN: the same shells
    # at Ma 1.5, Re 300 (the transonic sphere of Section 5.2)
    for base, mach in (("sphere", 0.2535), ("transonic", 1.5)):
        size = name[len(base):] if name.startswith(base) else None
        if size == "" or (size and size.isdigit()):
            n, nr = (58, 75) if size == "" else (int(size), max(2, round(1.3 * int(size))))
            xyz, cells, bfn, bft = I.sphere_shell(n, nr, seed=0)
            qinf = I.free_stream(mach)
            q = np.tile(qinf, (len(cells), 1))
            return dict(xyz=xyz, cells=cells, periods=None, bfn=bfn, bft=bft, q=q,
                        params=dict(q_inf=qinf, mu_ref=mach / 300, Pr=0.72, visc_exp=0.7, T_ref=1 / 1.4,
                                    tau_num_c=1.0),
                        desc=f"sphere shell 6x{n}^2x{nr} hex, Ma {mach} Re 300, wall + far field")
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.rows.append([x.strip() for x in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of x over the ranks: a job's time is its slowest rank's.
    dist is torch.distributed (or None for one process); device holds the
    reduction tensor ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(cells: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job cell-updates/s of `world` replicas that each advance `cells`
    cells by `steps` steps, timed by the slowest replica."""
    return cells * steps * world / seconds


def cpu_baseline(w, H=None, budget_steps: int = 3):
    """The CPU oracle as it stands, all host cores, on `budget_steps` steps of
    the same mesh.  With the library H, the GPU FP64 and mixed paths take the
    same steps from the same state and their differences from the oracle's
    state are reported (the parity metric of the GPU tests: max |gpu - oracle|
    over cells / max |oracle|, per variable; and the volume-weighted L1)."""
    import oracle

    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    o = oracle.Oracle(w["xyz"], w["cells"], w["periods"], w.get("bfn"), w.get("bft"),
                      **{{"tau_num_c": "tau_c", "q_inf": "qinf"}.get(k, k): v for k, v in w["params"].items()})
    o.set_state(w["q"])
    t0 = time.perf_counter()
    o.step(budget_steps)
    dt = time.perf_counter() - t0
    nc = len(w["cells"])
    res = {"value": nc * budget_steps / dt, "unit": "cell-updates/s", "cores": oracle.get_threads(),
           "kind": "oracle", "sample": f"{budget_steps} S2O4 step(s) of the full {nc}-cell mesh, FP64, "
                                       f"{oracle.get_threads()} OpenMP threads ({dt:.1f} s)"}
    if H is not None:
        qo, to, no = o.get_state()
        vol = o.geometry()[0]
        names = (("rho", 0), ("rhoU", 1), ("rhoV", 2), ("rhoW", 3), ("rhoE", 4))
        for prec, key in ((H.HGKS_FP64, "fp64_vs_oracle"), (H.HGKS_FP32_MIXED, "mixed_vs_oracle")):
            s = H.Solver(H.Mesh(w["xyz"], w["cells"], w["periods"], w.get("bfn"), w.get("bft")), w["q"],
                         precision=prec, **w["params"])
            s.step(budget_steps)
            qg, tg, ng = s.read()
            s.close()
            res[key] = {"steps": ng, "time_rel_diff": abs(tg - to) / to,
                        "max_rel": {k: float(np.abs(qg[:, v] - qo[:, v]).max() / np.abs(qo[:, v]).max())
                                    for k, v in names},
                        "l1_rel": {k: float((np.abs(qg[:, v] - qo[:, v]) * vol).sum() /
                                            (np.abs(qo[:, v]) * vol).sum()) for k, v in names}}
    return res


def run_reference(args, rank, world):
    """The CPU oracle as it stands on the host cores (rank 0 only).  Each
    timed step is one S2O4 step of a bounded sample of the workload: the
    24^3 x 6 jittered mesh for the density-wave workloads, the 6 x 24^2 x 31
    shell at the workload's Mach number for the sphere workloads, the 6 x 20^2
    x 26 hybrid shell and the 24^3 x 2 prism cube for those workloads."""
    if rank != 0:
        return
    import oracle

    w = workload(args.workload)
    ws = w
    if args.workload.startswith("density"):
        ws = workload("density24v" if args.workload.endswith("v") else "density24")
    elif args.workload.startswith("sphere"):
        ws = workload("sphere24")
    elif args.workload.startswith("transonic"):
        ws = workload("transonic24")
    elif args.workload.startswith("hybrid"):
        ws = workload("hybrid20")
    elif args.workload.startswith("prism"):
        ws = workload("prism24")
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    o = oracle.Oracle(ws["xyz"], ws["cells"], ws["periods"], ws.get("bfn"), ws.get("bft"),
                      **{{"tau_num_c": "tau_c", "q_inf": "qinf"}.get(k, k): v for k, v in ws["params"].items()})
    o.set_state(ws["q"])
    o.step(min(args.warmup, 1))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    nc = len(ws["cells"])
    val = nc * args.steps / dt
    line = {"impl": "reference", "metric": "cell-updates/s", "value": val, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "sample": f"{nc}-cell mesh per timed step"},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{args.steps} S2O4 steps of the {nc}-cell mesh"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def mixed_vs_fp64(H, w, stream, K, W, error_steps: int = 20):
    """FP32-mixed throughput on the same workload, and its L1 difference from
    the FP64 path after `error_steps` steps of the same fixed dt from the same
    state."""
    nc = len(w["cells"])
    base = H.Mesh(w["xyz"], w["cells"], w["periods"], w.get("bfn"), w.get("bft"))
    nf, kst = base.n_faces, base.stencil_size
    s = H.Solver(base.clone(), w["q"], precision=H.HGKS_FP32_MIXED, stream=stream.cuda_stream, **w["params"])
    ms = timed_steps(s, stream, K, W)
    prof = s.profile(K)
    s.close()
    # precision: both paths from the initial state with the FP64 path's first dt
    dts = []
    out = {}
    for prec in (H.HGKS_FP64, H.HGKS_FP32_MIXED):
        t = H.Solver(base.clone(), w["q"], precision=prec, **w["params"])
        if not dts:
            t.step(1)
            dts.append(t.read()[1])
            t.write(w["q"], 0.0)
        t.step(error_steps, dt_fixed=dts[0])
        out[prec] = t.read()[0]
        t.close()
    vol = base.geometry()[0]
    a, b = out[H.HGKS_FP32_MIXED], out[H.HGKS_FP64]
    l1 = {name: float((np.abs(a[:, v] - b[:, v]) * vol).sum() / (np.abs(b[:, v]) * vol).sum())
          for name, v in (("rho", 0), ("rhoU", 1), ("rhoE", 4))}
    linf = {name: float(np.abs(a[:, v] - b[:, v]).max() / np.abs(b[:, v]).max())
            for name, v in (("rho", 0), ("rhoU", 1), ("rhoE", 4))}
    G = 3 if len(w["cells"][0]) == 4 else 4
    viscous = bool(w["params"].get("mu_ref", 0.0) or w["params"].get("tau_num_c", 0.0))
    res = {"value": nc * K / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms / K, "dtype": "f32-mixed",
           "kernel_ms_per_step": {"ghost+recon": prof[1], "flux": prof[2], "update": prof[3]},
           "error_vs_fp64": {"steps": error_steps, "l1_rel": l1, "linf_rel": linf, "dt": dts[0]},
           "roofline_flux": flux_roofline("mixed", G, viscous, nf, prof[2] / 2.0)}
    if len(w["cells"][0]) == 4:
        # two reconstruction launches per step
        res["roofline_recon"] = recon_roofline(kst, 4, 6, nc, prof[1] / 2, w["periods"] is None)
    return res


def timed_steps(solver, stream, K, W):
    """Device time (ms) of K graph-replayed steps after W warm-up steps, CUDA
    events on the solver's stream."""
    import torch

    solver.step(W)
    solver.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    solver.step(K)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def c3_run(H, K, W, error_steps):
    """The laminar sphere of Section 5.2 on the 1.51M-cell hex shell (6 x 58^2
    x 75, wall spacing 0.0049, growth 1.08, Ma 0.2535, Re 300): FP64 and
    FP32-mixed throughput, per-kernel times, the flux roofline of both, and
    the mixed-vs-FP64 difference after `error_steps` steps of one fixed dt."""
    import torch

    w = workload("sphere")
    nc = len(w["cells"])
    base = H.Mesh(w["xyz"], w["cells"], None, w["bfn"], w["bft"])
    nf = base.n_faces
    stream = torch.cuda.Stream()
    out = {"workload": w["desc"], "cells": nc, "faces": nf}
    dt0 = None
    finals = {}
    for prec, name in ((H.HGKS_FP64, "fp64"), (H.HGKS_FP32_MIXED, "mixed")):
        s = H.Solver(base.clone(), w["q"], precision=prec, stream=stream.cuda_stream, **w["params"])
        ms = timed_steps(s, stream, K, W)
        prof = s.profile(K)
        s.close()
        out[name] = {"value": nc * K / (ms * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms / K,
                     "kernel_ms_per_step": {"finalize": prof[0], "ghost+recon": prof[1], "flux": prof[2],
                                            "update": prof[3]},
                     "roofline": flux_roofline(name, 4, True, nf, prof[2] / 2.0)}
        if name == "mixed":
            out[name]["roofline_recon"] = recon_roofline(base.stencil_size, 8, 3, nc, prof[1] / 2, True)
        # both precisions from the initial state with the FP64 path's first dt
        t = H.Solver(base.clone(), w["q"], precision=prec, **w["params"])
        if dt0 is None:
            t.step(1)
            dt0 = t.read()[1]
            t.write(w["q"], 0.0)
        t.step(error_steps, dt_fixed=dt0)
        finals[name] = t.read()[0]
        t.close()
    vol = base.geometry()[0]
    a, b = finals["mixed"], finals["fp64"]
    out["mixed"]["error_vs_fp64"] = {
        "steps": error_steps, "dt": dt0,
        "l1_rel": {k: float((np.abs(a[:, v] - b[:, v]) * vol).sum() / (np.abs(b[:, v]) * vol).sum())
                   for k, v in (("rho", 0), ("rhoU", 1), ("rhoE", 4))},
        "linf_rel": {k: float(np.abs(a[:, v] - b[:, v]).max() / np.abs(b[:, v]).max())
                     for k, v in (("rho", 0), ("rhoU", 1), ("rhoE", 4))}}
    out["mixed_speedup"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def serve_run(H, small: bool, capacity=None):
    """Serving stream, FP32-mixed.  small: 48 requests of 5e3..1e5 cells (the
    default line); otherwise the full 256 requests of 5e3..2e6 cells.  The
    Poisson rate offers 0.8 x the measured mixed throughput."""
    from paper_2407_00656_b300 import serve as S

    import torch

    n, hi = (48, 1e5) if small else (256, 2e6)
    lo, steps = 5e3, 200
    classes = 4 if small else 8
    cache = S.MeshCache()
    t0 = time.perf_counter()
    cache.warm(S.c5_requests(n=n, lo=lo, hi=hi, steps=steps, rate=1.0, seed=0, classes=classes))
    warm_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    budget = int(0.7 * free)
    # capacity of this request mix: every request present at t = 0 (closed loop)
    burst = S.c5_requests(n=n, lo=lo, hi=hi, steps=steps, rate=1e9, seed=0, classes=classes)
    S.Server(mem_budget=budget, precision=H.HGKS_FP32_MIXED, chunk_steps=10, cache=cache).run(burst, time_limit=1800)
    cap = S.summarize(burst)["cell_updates_per_s"]
    # open loop: Poisson arrivals offering 0.8 x that capacity
    mean_work = np.mean([r.cells for r in burst]) * steps
    rate = 0.8 * cap / mean_work
    reqs = S.c5_requests(n=n, lo=lo, hi=hi, steps=steps, rate=rate, seed=0, classes=classes)
    server = S.Server(mem_budget=budget, precision=H.HGKS_FP32_MIXED, chunk_steps=10, cache=cache)
    server.run(reqs, time_limit=1800)
    st = S.summarize(reqs)
    st.update({"capacity_cell_updates_per_s": cap, "offered_rate_per_s": rate, "steps_per_request": steps,
               "cells_range": [lo, hi],
               "peak_resident_solves": server.peak_active, "peak_device_bytes": server.peak_used,
               "mesh_cache_build_s": warm_s, "precision": "f32-mixed",
               "mix": "half jittered density-wave cubes, half sphere shells at Re U[100,300]"})
    return st


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hgks", choices=["hgks", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="density48")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving stream of the default line")
    ap.add_argument("--serve-small", action="store_true",
                    help="serve the small stream (48 requests of 5e3..1e5 cells) instead of the full one")
    ap.add_argument("--no-c3", action="store_true", help="skip the sphere-shell sub-line of the default line")
    ap.add_argument("--error-steps", type=int, default=None,
                    help="steps of the mixed-vs-FP64 comparison (default: the --steps value)")
    ap.add_argument("--serve", action="store_true", help="run the full serving stream (256 requests, up to 2M cells)")
    ap.add_argument("--no-graph", action="store_true", help="launch each step's kernels one by one (no CUDA graph)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.serve:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2407_00656_b300 import hgks as H

        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            st = serve_run(H, small=False)
        if rank == 0:
            print(json.dumps({"metric": "serve p50/p99 latency (s) and aggregate cell-updates/s", "value": st["p99_s"],
                              "unit": "s (p99)", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
                              "dtype": "f32-mixed", "config": {"workload": "serving stream, 256 requests"},
                              "serve": st, "clocks": clk.summary()}), flush=True)
        return

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2407_00656_b300 import hgks as H

    H.lib()
    prec = H.HGKS_FP64 if args.precision == "fp64" else H.HGKS_FP32_MIXED
    w = workload(args.workload)
    nc = len(w["cells"])
    stream = torch.cuda.Stream()
    mesh = H.Mesh(w["xyz"], w["cells"], w["periods"], w.get("bfn"), w.get("bft"))
    mesh_nf = mesh.n_faces
    solver = H.Solver(mesh, w["q"], precision=prec, stream=stream.cuda_stream, use_graph=0 if args.no_graph else 1,
                      **w["params"])
    W, K = max(args.warmup, 3), args.steps
    solver.step(W)
    solver.sync()
    launches_per_step = 7 + (2 if w.get("bfn") is not None else 0)

    # ---- device-timed region: K steps, inputs resident in HBM (graph replay)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            e0.record(stream)
            solver.step(K)
            e1.record(stream)
        e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    value = replica_throughput(nc, K, world, ms * 1e-3)

    # ---- per-kernel-group times (separate profiled pass of K steps, events
    # around each group on the solver's stream)
    prof = solver.profile(K)
    flux_ms = prof[2] / 2.0  # two flux launches per step
    nf = mesh_nf
    G = 3 if len(w["cells"][0]) == 4 else 4
    viscous = bool(w["params"].get("mu_ref", 0.0) or w["params"].get("tau_num_c", 0.0))
    roof = flux_roofline(args.precision, G, viscous, nf, flux_ms)
    roof["kernel_ms_per_step"] = {"finalize": prof[0], "ghost+recon": prof[1], "flux": prof[2], "update": prof[3]}

    # ---- end to end through the C ABI with host buffers: per step the state
    # goes host -> device, one step runs, the state comes back
    qh = torch.from_numpy(np.ascontiguousarray(w["q"])).pin_memory().numpy()
    out = torch.empty((nc, 5), dtype=torch.float64).pin_memory().numpy()
    e2e_steps = max(2, min(K, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.write(qh, 0.0)
        solver.step(1)
        solver.read(out)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": replica_throughput(nc, e2e_steps, world, t_e2e), "unit": "cell-updates/s",
           "h2d_bytes_per_step": int(qh.nbytes), "d2h_bytes_per_step": int(out.nbytes)}

    extra = {}
    if args.precision == "fp64":
        extra["mixed"] = mixed_vs_fp64(H, w, stream, K, W, args.error_steps or K)
    solo = world == 1
    if solo and args.workload == "density48" and not args.no_c3:
        extra["c3"] = c3_run(H, K, W, args.error_steps or K)
    if solo and not args.no_serve:
        extra["serve"] = serve_run(H, small=args.serve_small)

    if rank == 0:
        line = {"metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == H.HGKS_FP64 else "f32-mixed", "data": "synthetic",
                "config": {"workload": w["desc"], "cells": nc, "faces": nf, "precision": args.precision,
                           "cuda_graph": not args.no_graph,
                           "l2": "inputs larger than L2 (pseudo-inverses alone exceed 126 MB)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "e2e": e2e, "gpu_launches": K * launches_per_step + 1,
                "clocks": clk.summary()}
        line.update(extra)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(w, H)
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
