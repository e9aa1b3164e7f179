#!/usr/bin/env python
"""Throughput benchmark: FP64 DOF-updates/s of the H-M-H Strang step.

Headline workload: the MHD blast wave on a 1024 x 1024 periodic mesh of
[-1/2,1/2]^2, DGSEM degree p = 3, magnetic degree k = 3, gamma = 1.4, every
stabilisation map on (hydro OE, positivity limiter, artificial resistivity,
velocity OE), synthetic analytic initial state, CFL 0.4 time step fixed at
its t = 0 value.  One "step" is one full Strang step
S^dt = Phi_H^{dt/2} o Phi_M^{dt} o Phi_H^{dt/2}.  DOFs per element:
5 (p+1)^2 + 3 (k+1)^2 = 128.  Side legs: the Orszag-Tang vortex 256 x 256
(stabilised throughput), the reduced 2D2V stage, other (p, k), the adjoint
and the batch of independent runs.

  python bench.py --gpus N --steps K --warmup W [--impl ours|reference]

N > 1 runs under torchrun: every rank runs an independent replica (the
method has no data-path collective; weak scaling), the timed region is
bracketed by a barrier and synchronisation and the max over ranks is used.
--impl reference times the CPU oracle on the host cores (its OpenMP timing
build, bitwise equal to the serial oracle) on a bounded sample of the same
workload.
"""
import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FP64 DOF-updates/s per Strang step at p=3"
UNIT = "DOF-updates/s"
NOMINAL_FP64_TFLOPS = 1.25  # B300 dense FP64, nominal
FALLBACK_HBM_GBS = 6400.0   # profiling recipe's fallback copy bandwidth
# The stabilised workloads: OE (both stages), positivity limiter, artificial
# resistivity and velocity filter active, with the paper's constants.
STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)
WORKLOADS = {"blast": ("blast", 1024), "orszag_tang": ("orszag_tang", 256)}
# DRAM bytes (read + write) per element of one launch group of a kernel
# class, from the ncu captures of the current kernels on the 256 x 256 blast
# (profiles/kernels_blast_256_full.md: 65,536 elements; traffic grows in
# proportion to the elements, so it is scaled by K).  stab_hydro: k_stats
# (45.368 MB) + k_oe_pp (61.970 MB); k_lines and k_global move a few KB.
# vol: k_vol (69.970 MB).  Remove an entry whenever its kernels change.
NCU_TRAFFIC_BYTES_PER_ELEMENT = {"stab_hydro": (45367552 + 61970176) / 65536, "vol": (63017728 + 6952448) / 65536}


def workload_config(stab, name="orszag_tang", mesh=None):
    wl_name, default_mesh = WORKLOADS[name]
    mesh = mesh or default_mesh
    if name == "blast":
        return dict(workload=f"blast_{mesh}x{mesh}_p3k3", mesh=[mesh, mesh], domain=[-0.5, 0.5, -0.5, 0.5], p=3,
                    k=3, gamma=1.4, dofs_per_element=128, cfl=0.4, stabilization=stab,
                    l2="working set per step >> 126 MB L2 (state + stage buffers ~7 GB), no flush needed")
    return dict(workload=f"orszag_tang_{mesh}x{mesh}_p3k3", mesh=[mesh, mesh], domain=[0.0, 1.0, 0.0, 1.0], p=3,
                k=3, gamma=5.0 / 3.0, dofs_per_element=128, cfl=0.4, stabilization=stab,
                l2="working set per step > 126 MB L2 (state + stage buffers ~0.5 GB), no flush needed")


def max_over_ranks(ms, dist, device):
    """Slowest rank's time (ms): every rank gets the maximum (replicas, weak scaling)."""
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, dofs_per_rank, steps, ms):
    """DOF-updates/s of the whole job: every rank advances its own replica."""
    return world * dofs_per_rank * steps / (ms * 1e-3)


def dofs_per_element(p, k):
    return 5 * (p + 1) ** 2 + 3 * (k + 1) ** 2


def vol_flops_per_element_pairs(p):
    """Algorithmic work of one volume-kernel launch per element: ~117 FP64
    op-equivalents per unique entropy-conservative pair (means 12, two log means 2 x 22, p-hat 9, h-hat
    21, flux 6, accumulation into both nodes 20; FMA = 2, division = 8) times
    the p (p+1)^2 unique pairs of an element (48 at p = 3: 5,616)."""
    return 117 * p * (p + 1) ** 2


def vol_flops_per_element_minimal(p):
    """Algorithmic FP64 flops of one launch of the volume kernel per element
    (FMA = 2, add/mul/reciprocal = 1): 52 per entropy-conservative pair
    (p (p+1)^2 pairs), 16 per node for the primitives, 5 (4p + 3) per node for
    the gather with D, 8 per face node for the end terms, 4 per node-component
    for the stage combination and 2 per node-component for the raw average."""
    n = p + 1
    n2 = n * n
    return 52 * p * n2 + 16 * n2 + 5 * n2 * (4 * p + 3) + 5 * 4 * n * 2 + 5 * n2 * 4 + 5 * n2 * 2 + 8


def stats_flops(p, nc):
    """OE statistics of nc DG fields per element (k_stats): the weighted
    average (one FMA per node), and per direction the jump measures J_r of the
    lower face: r = 0 the traces (4 flops per face node), r >= 1 the r-th
    derivative of both traces (2 (p+1) FMAs per face node) and the squared
    jump (4), each order closed by a scale and a square root."""
    n = p + 1
    per_dir = 4 * n + 1 + p * (n * (4 * n + 4) + 2)
    return nc * (2 * n * n + 2 * per_dir)


def b_nodes_flops(p, k):
    """B_x, B_y, B_z at all (p+1)^2 DG nodes of an element, sum-factorised:
    an x-pass over the rows, then a y-pass (2 flops per FMA).  A node family
    that coincides with the DG nodes (GLL(k+1) at k = p - 1, GLL(k) at k = p)
    needs no interpolation: its passes are copies."""
    n, mm, mL = p + 1, k + 1, k + 2
    lid, mid = mL == n, mm == n
    bx = (0 if lid else mm * n * mL) + n * n * mm
    by = mL * n * mm if lid else mm * n * mL + n * n * mm  # columns to the DG y-nodes first
    bz = 0 if mid else mm * n * mm + n * n * mm
    return 2 * (bx + by + bz)


def ar_elem_flops(p, k):
    """The A.R. partials of one element (k_ar_elem): the exact integrals of
    B_x, B_y, B_z (weight rows, x-pass then y-pass), per lower face the two
    tangential traces of both elements with the normal direction collapsed
    first, their values, jumps and squared sums at the k + 2 face points and a
    square root per component, and B at the DG nodes with |B|^2 / rho, a
    square root and the speeds per node."""
    n, mm, mL = p + 1, k + 1, k + 2
    n2 = n * n
    integrals = 2 * (mm * mL + mm) + 2 * (mL * mm + mL) + 2 * (mm * mm + mm) + 3
    traces = 2 * (2 * mL * mm + 2 * mm * mm)
    per_point = 2 * (2 * mL + 2 * mm) + 2 + 2 + 2 * 2
    face = traces + (k + 2) * per_point + 2
    nodes = b_nodes_flops(p, k) + n2 * (5 + 1 + 1 + 1 + 4)
    return integrals + 2 * face + nodes


def step_work(p, k):
    """Algorithmic FP64 flops and DRAM bytes per element of each kernel class
    for one Strang step with every stabilisation map on and a resistive A.R.,
    counted from the kernels' loop bounds (FMA = 2 flops; add, multiply,
    reciprocal, square root = 1; index arithmetic, reductions of maxima and
    table products not counted).  Bytes: every array the class must read and
    write once from DRAM (no reuse across kernels assumed).  Classes are those
    of the library's event profiler; a Strang step has 6 hydro stages, 3
    magnetic stages and 2 nodal exchanges.  The resistive Ohm load and the
    Ohmic heating run only in elements with eta_K > 0 and are not counted (a
    lower bound)."""
    n = p + 1
    n2, mm, mL = n * n, k + 1, k + 2
    NX = NY = mm * mL
    NW, NZ = mL * mL, mm * mm
    d8 = 8
    work = {}
    # LLF on the 2 (p+1) face nodes an element owns: ~70 flops each; reads
    # both traces, writes the flux (5 components)
    work["face"] = (6 * 2 * n * 70, 6 * 2 * n * 15 * d8)
    # volume + SSP combination + raw average; stage input, U^n (stages 2, 3),
    # output and the face fluxes of the element's own faces
    work["vol"] = (6 * vol_flops_per_element_minimal(p), 2 * (8 * 5 * n2 + 3 * 2 * 5 * n) * d8)
    # hydro OE + limiter per stage: statistics of 5 fields, the rate (20), the
    # sensor (2 n sigma items) and factors (n exponentials), the damping as
    # three sum-factorised passes per component (forward y, the x-filter of
    # each y-mode, backward y: 2 n^3 FMAs each) after building the x-filters
    # once per element (n^3 (n+1) / 2 FMAs), the limiter (~35 per node:
    # average, pressures, scalings)
    oe = (20 + 2 * n * (5 + 2) + n * (2 * n + 3) + 5 * 3 * n2 * n * 2 + 2 * (n ** 3 * (n + 1) // 2)
          + 35 * n2)
    work["stab_hydro"] = (6 * (stats_flops(p, 5) + oe), 6 * 3 * 5 * n2 * d8)
    # nodal exchange (u = m/rho, e; and back): ~10 flops per node each way
    work["exchange"] = (2 * 10 * n2, (5 + 4 + 4 + 1 + 5) * n2 * d8)
    # magnetic stage (J, E, curl) x 3 stages
    fJ = 2 * (2 * mm * mL * mL + 2 * NZ * mm + 2 * mm * NW + (NX + NY) * mm) + 3 * NW + 2 * (NX + NY)
    assemble = 4 * NW + 2 * (NX + NY)
    # at k = p - 1 the GLL(k+1) nodes are the DG nodes: every pass between them is a copy
    lid = mL == n
    # velocity: u_x rows to GLL(k+1) x and u_y columns to GLL(k+1) y (shared by two families
    # each), u_z rows to Gauss x and columns to Gauss y, then one second pass per family value
    fE = (assemble
          + 2 * (2 * n * mm * n + (0 if lid else 2 * n * mL * n) + NW * mm + NZ * mm + mm * mL * mm)  # first passes
          + 2 * ((NX + NY + (0 if lid else NX + NY + 2 * NW)) * n + (NX + NY + NW) * mm)              # second passes
          + 10 * (NX + NY + NW)                                                              # Ohm loads, Lorentz
          + (2 * 2 * n * mm * mL if lid else 2 * (4 * n * mm * mL + 2 * n * mL * mL))        # transposed first passes
          + n2 * (2 * ((0 if lid else 2 * mL) + 2 * mm) + 27))                               # second passes, rates, SSP
    fB = assemble + 2 * (NZ * mL + mL * mm * mm) + 3 * NZ * (2 * mL + 6) + NZ * 2 * mm
    loads = (NX + NY + NW) * d8
    bJ = 3 * NZ * d8 + loads
    bE = loads + 3 * NZ * d8 + (3 + 1 + 1) * n2 * d8 + (3 + 1) * n2 * d8 * 2 + loads
    bB = loads + 3 * NZ * d8 * 3
    work["mag_stage"] = (3 * (fJ + fE + fB), 3 * (bJ + bE + bB))
    # A.R. coefficient once per magnetic substep: element integrals, face jumps
    # of the tangential traces, and B at the DG nodes for the directional speeds
    work["stab_eta"] = (ar_elem_flops(p, k), (3 * NZ + 3 * n2 + 16) * d8)
    # velocity OE: projectors once (rho-weighted Gram matrix, Cholesky, the
    # rows of Psi = Phi L^-T), then per stage the statistics of 3 fields and the
    # map (B at the nodes, coefficients and shell sums: 2 n2^2 FMAs per component)
    prep = (2 * n2 + 2 * n * (n * (n + 1) // 2) * n + 2 * (n2 * (n2 + 1) // 2) * n
            + 2 * n2 ** 3 // 3 + n2 ** 3)
    voe = b_nodes_flops(p, k) + 10 * n2 + 3 * 2 * 2 * n2 * n2 + 3 * 3 * n
    work["stab_vel"] = (prep + 3 * (stats_flops(p, 3) + 20 + 2 * n * 5 + n * (2 * n + 3) + voe),
                        (n2 + n2 * n2) * d8 + 3 * (3 * n2 + 3 * n2 + n2 + 3 * NZ + n2 * n2 + 4 * n2 + n2) * d8)
    return work


def measured_hbm_gbs():
    """Copy bandwidth of the B300s (MEASURED_PEAKS.json), else the
    recipe's fallback; returns (GB/s, source)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_rooflines(kt, K, steps, p, k, p64_tflops, bw_gbs):
    """Per-class roofline from the live CUDA-event times of `steps` Strang
    steps: algorithmic flops and bytes per step (step_work) against the FP64
    issue peak and the copy bandwidth; the bound is the larger of the two
    times; frac = that time / the measured time.  Also the step-level bound
    sum_k max(flops_k / P64, bytes_k / BW)."""
    work = step_work(p, k)
    out, bound_ms = {}, 0.0
    for cls, (ms, groups) in kt.items():
        if cls not in work:
            continue
        fl, by = work[cls]
        fl_step, by_step = fl * K, by * K
        t_ms = ms / steps
        t_fl = fl_step / (p64_tflops * 1e12) * 1e3
        t_by = by_step / (bw_gbs * 1e9) * 1e3
        bound = "fp64" if t_fl >= t_by else "hbm"
        bound_ms += max(t_fl, t_by)
        out[cls] = {"ms_per_step": t_ms, "launch_groups_per_step": groups / steps,
                    "flops_per_step": fl_step, "bytes_per_step": by_step,
                    "achieved_tflops": fl_step / (t_ms * 1e-3) / 1e12,
                    "achieved_gbs": by_step / (t_ms * 1e-3) / 1e9,
                    "bound": bound, "frac": max(t_fl, t_by) / t_ms}
    return out, bound_ms


def make_solver(name, mesh, stab_params, p=3, k=3):
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.WORKLOADS[WORKLOADS[name][0]]()
    s = Solver(mesh, mesh, p, k, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    s.set_primitive(np.ascontiguousarray(rho), np.ascontiguousarray(np.stack([ux, uy, uz])),
                    np.ascontiguousarray(pr))
    del X, Y, rho, ux, uy, uz, pr
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_B_from_potential(np.ascontiguousarray(wl["Az"](XW, YW)), *wl["B0"],
                           np.ascontiguousarray(wl["fields"](XZ, YZ)[5]))
    if stab_params:
        s.set_params(cfl=0.4, **stab_params)
    return s


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def oracle_for(name, n, parallel):
    """The oracle (serial, or its bitwise-equal OpenMP build) on an n x n mesh
    of the same workload and physics as the GPU run."""
    import oracle
    from paper_2609_10849_b300 import workloads
    wl = workloads.WORKLOADS[WORKLOADS[name][0]]()
    cls = oracle.ParallelOracle if parallel else oracle.Oracle
    o = cls(n, n, 3, 3, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = o.coords("w")
    XZ, YZ = o.coords("bz")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW), *wl["B0"])
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, wl["fields"](XZ, YZ)[5])
    o.set_params(cfl=0.4, **STAB)
    return o


def cpu_baseline(name="blast", n=64, steps_serial=2, steps_parallel=8):
    """The oracle as it stands on a bounded sample of the same workload (the
    same physics on an n x n mesh, p = k = 3): single-threaded, and its OpenMP
    timing build on every host core (bitwise equal results)."""
    cores = host_cores()
    res = {}
    for parallel, steps in ((False, steps_serial), (True, steps_parallel)):
        o = oracle_for(name, n, parallel)
        used = o.set_threads(cores) if parallel else 1
        dt = o.cfl_dt()
        o.strang_step(dt)  # warm-up
        t0 = time.perf_counter()
        for _ in range(steps):
            o.strang_step(dt)
        el = time.perf_counter() - t0
        res[parallel] = (dofs_per_element(3, 3) * n * n * steps / el, used, steps, el)
    v1, _, s1, e1 = res[False]
    vN, used, sN, eN = res[True]
    return dict(value=vN, unit=UNIT, cores=used, kind="oracle", value_1_thread=v1, cpu_model=cpu_model(),
                host_cores=cores,
                sample=f"same {name} physics on a {n}x{n} mesh (p=k=3, all stabilisation on): {sN} Strang steps on "
                       f"{used} threads (OpenMP timing build of the oracle, bitwise equal to the serial one, "
                       f"{eN:.1f} s) and {s1} steps single-threaded ({e1:.1f} s)")


def run_reference(args, rank):
    if rank != 0:
        return
    n = 64
    o = oracle_for(args.workload, n, parallel=True)
    used = o.set_threads(host_cores())
    dt = o.cfl_dt()
    for _ in range(args.warmup):
        o.strang_step(dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.strang_step(dt)
    el = time.perf_counter() - t0
    value = dofs_per_element(3, 3) * n * n * args.steps / el
    sample = (f"each step: one Strang step of the {args.workload} workload's physics on a {n}x{n} sample mesh "
              f"(p=k=3), the oracle's OpenMP timing build on {used} host threads ({cpu_model()})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(STAB, args.workload, args.mesh),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def batch_leg(nruns, steps):
    """Batched workload: nruns independent Orszag-Tang variants with seeded
    uneven meshes and degrees, all stabilisation on, advanced by one CUDA-graph
    launch per call, against the same runs advanced one at a time."""
    import torch
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.mhd import Batch
    specs = workloads.batch_specs(nruns)
    wls = [workloads.orszag_tang_variant(i) for i in range(len(specs))]
    full = [(N, N, p, p, wl["gamma"], wl["domain"]) for (N, p), wl in zip(specs, wls)]
    t0 = time.perf_counter()
    batch = Batch(full)
    for r, wl in zip(batch.runs, wls):
        X, Y = r.coords("dg")
        rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
        r.set_primitive(np.ascontiguousarray(rho), np.ascontiguousarray(np.stack([ux, uy, uz])), np.ascontiguousarray(pr))
        XW, YW = r.coords("w")
        XZ, YZ = r.coords("bz")
        r.set_B_from_potential(np.ascontiguousarray(wl["Az"](XW, YW)), *wl["B0"],
                               np.ascontiguousarray(wl["fields"](XZ, YZ)[5]))
        r.set_params(cfl=0.4, **STAB)
    dts = np.array([r.compute_dt() for r in batch.runs])
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch.autotune()  # per-run tiles, used by the batched and the sequential runs alike
    tune = time.perf_counter() - t0
    dofs = sum(dofs_per_element(p, p) * N * N for N, p in specs)
    batch.step(dts, steps)  # capture + warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    batch.step(dts, steps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    for r, dt in zip(batch.runs, dts):  # sequential: one run at a time through the plain path
        r.strang_steps(dt, steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, dt in zip(batch.runs, dts):
        r.strang_steps(dt, steps)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    out = {
        "metric": "FP64 DOF-updates/s, batched vs sequential", "unit": UNIT, "runs": len(specs),
        "elements": int(sum(N * N for N, _ in specs)), "steps": steps,
        "batched": dofs * steps / tb, "sequential": dofs * steps / ts, "speedup": ts / tb,
        "setup_s": setup, "autotune_s": tune, "degrees": {str(p): sum(1 for _, q in specs if q == p) for p in (2, 3, 4)},
        "config": {"workload": "orszag_tang_variants_batch", "stabilization": STAB, "seed": workloads.SEED}}
    batch.close()
    return out


def gll_weights(p):
    """GLL(p) quadrature weights 2/(p(p+1) P_p(x_i)^2) (nodes: +-1 and the roots
    of P_p'), for the objective's mass weights."""
    from numpy.polynomial import legendre as L
    x = np.concatenate([[-1.0], np.sort(L.Legendre.basis(p).deriv().roots().real), [1.0]])
    return 2.0 / (p * (p + 1) * L.legval(x, [0] * p + [1]) ** 2)


def adjoint_leg(steps=20, every=20, n=128, p=4):
    """Adjoint workload: the advected MHD vortex (§4.2) on n x n elements of
    [-5,5]^2, p = k = 4, fixed dt (CFL at t = 0), stabilisation off.  Times
    `steps` forward Strang steps and the checkpointed backward pass of the
    objective 1/2 sum_q M_q (rho_q(T) - rho*_q(T))^2 (a seeded perturbed run
    gives rho*), against the plain forward of the same steps."""
    import torch
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.adjoint import pack_primitive, strang_steps
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.balsara_vortex()
    s = Solver(n, n, p, p, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
    dt = s.compute_dt()
    x = torch.zeros(s.state_size(), dtype=torch.float64, device="cuda")
    s.get_packed(x)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    B, r0, u0, p0 = x[5 * s.N:].clone(), dev(rho), dev(np.stack([ux, uy, uz])), dev(pr)
    rs = dev(workloads.vortex_target_density(X, Y))
    with torch.no_grad():
        target = strang_steps(s, pack_primitive(s, rs, u0, p0, B), dt, steps, every)[:s.N].clone()
    Mq = dev(np.tile(np.outer(gll_weights(p), gll_weights(p)).ravel() * (10.0 / n) ** 2 / 4, s.K))

    def forward_backward():
        rho_v = r0.clone().requires_grad_(True)
        u_v = u0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xT = strang_steps(s, pack_primitive(s, rho_v, u_v, p0, B), dt, steps, every)
        J = 0.5 * (Mq * (xT[:s.N] - target) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        return t1 - t0, time.perf_counter() - t1

    forward_backward()  # warm-up: first-use costs and the adjoint's tape allocation
    tf, tb = forward_backward()
    s.set_packed(x)
    s.strang_steps(dt, steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.strang_steps(dt, steps)
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    dofs = dofs_per_element(p, p) * s.K
    return {"workload": f"balsara_vortex_{n}x{n}_p{p}k{p}", "steps": steps, "checkpoint_every": every, "dt": dt,
            "plain_ms_per_step": 1e3 * tp / steps, "forward_ms_per_step": 1e3 * tf / steps,
            "backward_ms_per_step": 1e3 * tb / steps, "backward_over_plain": tb / tp,
            "plain_dof_updates_per_s": dofs * steps / tp, "adjoint_dof_updates_per_s": dofs * steps / tb,
            "note": "backward = one mhd_adjoint_segment per checkpoint segment (recomputes the segment once, "
                    "recording every stage state, then the step adjoints); forward includes checkpoint copies; "
                    "second of two forward/backward passes"}


def timed_steps(s, dt, steps, stream):
    """CUDA-event time (ms) of `steps` graph-replayed Strang steps on `stream`."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.strang_steps(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def reduced_2d2v_leg(s, dt, steps, stream, dofs, full_ms_per_step):
    """The same workload with the reduced 2D2V magnetic stage (the state has
    u_z = B_z = 0, which every step keeps exactly; the result equals the full
    stage bitwise).  Same DOF count, timed like the headline."""
    import torch
    s.set_params(reduced_2d2v=1)
    s.strang_steps(dt, 3)
    torch.cuda.synchronize()
    ms = timed_steps(s, dt, steps, stream)
    s.set_params(reduced_2d2v=0)
    return {"ms_per_step": ms / steps, "value": dofs * steps / (ms * 1e-3), "unit": UNIT,
            "speedup_vs_full": full_ms_per_step / (ms / steps),
            "note": "reduced_2d2v=1: in-plane E_h, J_h and u_z, B_z are not formed (all identically zero)"}


def throughput_leg(name, mesh, p, k, steps, stream=None):
    """Stabilised throughput of a workload at (p, k), tile-autotuned."""
    import torch
    s = make_solver(name, mesh, STAB, p, k)
    stream = stream or torch.cuda.Stream()
    s.set_stream(stream.cuda_stream)
    tiles = s.autotune()
    dt = s.compute_dt()
    s.strang_steps(dt, 3)
    torch.cuda.synchronize()
    ms = timed_steps(s, dt, steps, stream) / steps
    s.close()
    return {"ms_per_step": ms, "value": dofs_per_element(p, k) * mesh * mesh / (ms * 1e-3), "unit": UNIT,
            "tiles": list(tiles), "steps": steps}


def degree_leg(pairs=((3, 2), (4, 4), (2, 2), (4, 3)), mesh=256, steps=10):
    """The Orszag-Tang workload (all stabilisation on) at other (p, k): the
    even-m family the paper recommends, (3,2) and (4,4), and two neighbours.
    Each pair is tile-autotuned; DOFs per element 5 (p+1)^2 + 3 (k+1)^2."""
    return {"workload": f"orszag_tang_{mesh}x{mesh}", "steps": steps,
            "pairs": {f"p{p}k{k}": throughput_leg("orszag_tang", mesh, p, k, steps) for p, k in pairs}}


def run_batch(args):
    print(json.dumps(batch_leg(args.batch, args.steps)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="blast", choices=list(WORKLOADS))
    ap.add_argument("--mesh", type=int, default=0, help="elements per direction (0: the workload's own)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0, help="run the batched workload with this many runs instead")
    ap.add_argument("--no-side-legs", action="store_true", help="skip the side measurements")
    ap.add_argument("--tiles", default="", help="VOL,MAG tile variants instead of the autotuner (VOL 0 default, 1, "
                    "2; MAG 0..2 for all magnetic kernels or the code vE + 3 vJ + 9 vB), for runs under a profiler, "
                    "whose serialised launches distort the autotuner's timings")
    ap.add_argument("--leg", default="", choices=["", "adjoint"], help="run only this side measurement")
    ap.add_argument("--reduced-2d2v", action="store_true",
                    help="time the reduced 2D2V magnetic stage in the main measurement (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.mesh = args.mesh or WORKLOADS[args.workload][1]

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.batch:
        run_batch(args)
        return
    if args.leg == "adjoint":
        print(json.dumps(adjoint_leg()), flush=True)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2609_10849_b300 import mhd
    s = make_solver(args.workload, args.mesh, STAB)
    stream = torch.cuda.Stream()  # a capturable stream (the legacy default stream is not)
    torch.cuda.set_stream(stream)
    s.set_stream(stream.cuda_stream)
    if args.reduced_2d2v:
        s.set_params(reduced_2d2v=1)
    if args.tiles:  # fixed variants; elements per CTA of p = 3 (csrc: vol_tile_eb, mag_tile_eb)
        tv, tm = (int(x) for x in args.tiles.split(","))
        s.set_tiles(tv, tm)
        tiles = ((8, 4, 16)[tv], (16, 8, 32)[tm % 3])
    else:
        tiles = s.autotune()  # elements per CTA of the volume and magnetic kernels
    dt = s.compute_dt()
    dofs = dofs_per_element(3, 3) * s.K

    s.strang_steps(dt, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        s.strang_steps(dt, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - l0
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    ms_per_step = ms / args.steps
    value = whole_job_value(world, dofs, args.steps, ms)

    # per-class CUDA-event timing of the same number of steps (separate, eager
    # pass on the same stream) for the rooflines
    s.profile_kernels(True)
    s.strang_steps(dt, args.steps)
    kt = s.kernel_times()
    s.profile_kernels(False)
    p64 = mhd.fp64_peak_tflops()
    bw, bw_src = measured_hbm_gbs()
    per_class, bound_ms = kernel_rooflines(kt, s.K, args.steps, 3, 3, p64, bw)
    events_ms = sum(v[0] for v in kt.values()) / args.steps
    top = max(per_class, key=lambda c: per_class[c]["ms_per_step"])
    vol_ms = kt["vol"][0] / kt["vol"][1]
    top_r = per_class[top]
    traffic = NCU_TRAFFIC_BYTES_PER_ELEMENT.get(top)
    roofline = {
        "bound": "alu", "kernel_class": top, "achieved": top_r["achieved_tflops"], "peak": p64,
        "unit": "TFLOP/s", "frac": top_r["achieved_tflops"] / p64,
        "traffic": None if traffic is None else traffic * s.K,
        "traffic_algorithmic": top_r["bytes_per_step"] / top_r["launch_groups_per_step"],
        "traffic_unit": "DRAM bytes per launch group (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
        "peak_source": "FP64 FMA issue rate measured in this run (mhd_fp64_peak: DFMA probe, all lanes)",
        "peak_nominal_tflops": NOMINAL_FP64_TFLOPS,
        "frac_of_nominal": top_r["achieved_tflops"] / NOMINAL_FP64_TFLOPS,
        "flops_definition": "algorithmic FP64 flops counted from the kernels' loop bounds (bench.step_work: "
                            "FMA = 2, add/mul/rcp/sqrt = 1)",
        "hbm_gbs": bw, "hbm_source": bw_src,
        "per_kernel_class": per_class,
        "step_bound_ms": bound_ms, "step_ms_events": events_ms, "step_frac": bound_ms / ms_per_step,
        "vol": {"avg_launch_ms": vol_ms,
                "tflops_117_per_pair": vol_flops_per_element_pairs(3) * s.K / (vol_ms * 1e-3) / 1e12,
                "tflops_minimal": vol_flops_per_element_minimal(3) * s.K / (vol_ms * 1e-3) / 1e12},
    }

    # end-to-end through the public API with pinned host buffers
    U, Bx, By, Bz = (torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
                     for n in (5 * s.N, s.G, s.G, s.Z))
    host = (U.reshape(5, s.N), Bx, By, Bz)
    s.get_state(host)
    e2e_steps = max(5, args.steps // 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state(*host)
        s.strang_step(dt)
        s.get_state(host)
    e2e_el = time.perf_counter() - t0
    nbytes = 8 * (5 * s.N + 2 * s.G + s.Z)
    e2e = {"value": world * dofs * e2e_steps / e2e_el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    del U, Bx, By, Bz, host

    side = {}
    if not args.no_side_legs and world == 1 and not args.reduced_2d2v:
        side["reduced_2d2v"] = reduced_2d2v_leg(s, dt, args.steps, stream, dofs, ms_per_step)
    s.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": f"synthetic (analytic {args.workload} initial state)",
            "config": dict(workload_config(STAB, args.workload, args.mesh), parallelism=f"replicas{world}", dt=dt,
                           magnetic_stage="reduced 2D2V" if args.reduced_2d2v else "full",
                           tiles={"vol_elements_per_cta": tiles[0], "mag_elements_per_cta": tiles[1]}),
            "roofline": roofline, "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
        }
        line.update(side)
        if not args.no_side_legs and world == 1:
            if args.workload != "orszag_tang":
                line["orszag_tang_256"] = throughput_leg("orszag_tang", 256, 3, 3, args.steps)
            line["degrees"] = degree_leg()
            line["adjoint"] = adjoint_leg()
            line["batched"] = batch_leg(256, 5)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
