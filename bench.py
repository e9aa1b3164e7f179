#!/usr/bin/env python
"""Throughput benchmark: FP64 DOF-updates/s of the H-M-H Strang step.

Workload: the Orszag-Tang vortex on a 256 x 256 periodic mesh of [0,1]^2,
DGSEM degree p = 3, magnetic degree k = 3, gamma = 5/3, synthetic analytic
initial state, CFL 0.4 time step fixed at its t = 0 value.  One "step" is one
full Strang step S^dt = Phi_H^{dt/2} o Phi_M^{dt} o Phi_H^{dt/2}.
DOFs per element: 5 (p+1)^2 + 3 (k+1)^2 = 128.

  python bench.py --gpus N --steps K --warmup W [--impl ours|reference]

N > 1 runs under torchrun: every rank runs an independent replica (the
method has no data-path collective; weak scaling), the timed region is
bracketed by a barrier and synchronisation and the max over ranks is used.
--impl reference times the CPU oracle (plain FP64, one core) on a bounded
sample of the same workload.
"""
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

METRIC = "FP64 DOF-updates/s per Strang step at p=3"
UNIT = "DOF-updates/s"
NOMINAL_FP64_TFLOPS = 1.25  # B300 dense FP64, nominal
# DRAM bytes (read + write) of one k_vol<3> launch, mean over the three SSP stages (stage 1
# does not read U^n), from the ncu capture summarised in
# profiles/kvol_dram_orszag_tang_256.md (same kernel source as this bench); reset to None
# whenever the volume kernel changes until it is captured again.
K_VOL_TRAFFIC_BYTES = (63016704 + 7692032 + 104972544 + 16648192 + 105055488 + 7912192) / 3.0
# The stabilised benchmark workload: OE (both stages), positivity limiter, artificial
# resistivity and velocity filter active, with the paper's constants.
STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def workload_config(stab, mesh=256):
    return dict(workload=f"orszag_tang_{mesh}x{mesh}_p3k3", mesh=[mesh, mesh], domain=[0.0, 1.0, 0.0, 1.0], p=3, k=3,
                gamma=5.0 / 3.0, dofs_per_element=128, cfl=0.4, stabilization=stab,
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


def make_solver(stab_params, mesh=256):
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.orszag_tang()
    s = Solver(mesh, mesh, 3, 3, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, p, _ = wl["fields"](X, Y)
    s.set_primitive(np.ascontiguousarray(rho), np.ascontiguousarray(np.stack([ux, uy, uz])),
                    np.ascontiguousarray(p))
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


def cpu_baseline(steps=3, n=64):
    """The oracle as it stands, single-threaded, on a bounded sample of the same
    workload: the Orszag-Tang vortex on an n x n mesh, p = k = 3."""
    import oracle
    from paper_2609_10849_b300 import workloads
    wl = workloads.orszag_tang()
    o = oracle.Oracle(n, n, 3, 3, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = o.coords("w")
    XZ, YZ = o.coords("bz")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW), *wl["B0"])
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, wl["fields"](XZ, YZ)[5])
    o.set_params(cfl=0.4, **STAB)
    dt = o.cfl_dt()
    o.strang_step(dt)  # warm-up
    t0 = time.perf_counter()
    for _ in range(steps):
        o.strang_step(dt)
    el = time.perf_counter() - t0
    return dict(value=dofs_per_element(3, 3) * n * n * steps / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"{steps} Strang steps of the same Orszag-Tang workload on a {n}x{n} mesh (p=k=3), "
                       f"serial C++ oracle, {el:.1f} s")


def run_reference(args, rank):
    if rank != 0:
        return
    stab = STAB
    n = 32
    import oracle
    from paper_2609_10849_b300 import workloads
    wl = workloads.orszag_tang()
    o = oracle.Oracle(n, n, 3, 3, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = o.coords("w")
    XZ, YZ = o.coords("bz")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW), *wl["B0"])
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, wl["fields"](XZ, YZ)[5])
    o.set_params(cfl=0.4, **STAB)
    dt = o.cfl_dt()
    for _ in range(args.warmup):
        o.strang_step(dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.strang_step(dt)
    el = time.perf_counter() - t0
    value = dofs_per_element(3, 3) * n * n * args.steps / el
    sample = (f"each step: one Strang step of the Orszag-Tang workload on a {n}x{n} sample mesh (p=k=3), serial "
              f"C++ oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(stab, args.mesh),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
        target = strang_steps(s, pack_primitive(rs, u0, p0, s.gamma, B), dt, steps, every)[:s.N].clone()
    Mq = dev(np.tile(np.outer(gll_weights(p), gll_weights(p)).ravel() * (10.0 / n) ** 2 / 4, s.K))
    def forward_backward():
        rho_v = r0.clone().requires_grad_(True)
        u_v = u0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xT = strang_steps(s, pack_primitive(rho_v, u_v, p0, s.gamma, B), dt, steps, every)
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


def reduced_2d2v_leg(s, dt, steps, stream, dofs, full_ms_per_step):
    """The same workload with the reduced 2D2V magnetic stage (the Orszag-Tang
    state has u_z = B_z = 0, which every step keeps exactly; the result equals
    the full stage bitwise).  Same DOF count, timed like the headline."""
    import torch
    s.set_params(reduced_2d2v=1)
    s.strang_steps(dt, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.strang_steps(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    s.set_params(reduced_2d2v=0)
    return {"ms_per_step": ms / steps, "value": dofs * steps / (ms * 1e-3), "unit": UNIT,
            "speedup_vs_full": full_ms_per_step / (ms / steps),
            "note": "reduced_2d2v=1: in-plane E_h, J_h and u_z, B_z are not formed (all identically zero)"}


def degree_leg(pairs=((3, 2), (4, 4), (2, 2), (4, 3)), mesh=256, steps=10):
    """The benchmark workload (Orszag-Tang, all stabilisation on) at other
    (p, k): the even-m family the paper recommends, (3,2) and (4,4), and two
    neighbours.  Each pair is tile-autotuned; DOFs per element 5 (p+1)^2 + 3 (k+1)^2."""
    import torch
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.mhd import Solver
    out = {}
    wl = workloads.orszag_tang()
    for p, k in pairs:
        s = Solver(mesh, mesh, p, k, wl["gamma"], wl["domain"])
        X, Y = s.coords("dg")
        rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
        s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
        XW, YW = s.coords("w")
        XZ, YZ = s.coords("bz")
        s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
        s.set_params(cfl=0.4, **STAB)
        stream = torch.cuda.Stream()
        s.set_stream(stream.cuda_stream)
        tiles = s.autotune()
        dt = s.compute_dt()
        s.strang_steps(dt, 3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.strang_steps(dt, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[f"p{p}k{k}"] = {"ms_per_step": ms, "value": dofs_per_element(p, k) * s.K / (ms * 1e-3), "unit": UNIT,
                            "tiles": list(tiles)}
        s.close()
    return {"workload": f"orszag_tang_{mesh}x{mesh}", "steps": steps, "pairs": out}


def run_batch(args):
    print(json.dumps(batch_leg(args.batch, args.steps)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mesh", type=int, default=256, help="elements per direction (256 is the benchmark workload)")
    ap.add_argument("--batch", type=int, default=0, help="run the batched workload with this many runs instead")
    ap.add_argument("--no-side-legs", action="store_true", help="skip the adjoint and batched side measurements")
    ap.add_argument("--leg", default="", choices=["", "adjoint"], help="run only this side measurement")
    ap.add_argument("--reduced-2d2v", action="store_true",
                    help="time the reduced 2D2V magnetic stage in the main measurement (for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

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
    stab = STAB
    s = make_solver(stab, args.mesh)
    stream = torch.cuda.Stream()  # a capturable stream (the legacy default stream is not)
    torch.cuda.set_stream(stream)
    s.set_stream(stream.cuda_stream)
    if args.reduced_2d2v:
        s.set_params(reduced_2d2v=1)
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

    # per-kernel event timing of the same steps (separate pass) for the roofline
    s.profile_kernels(True)
    s.strang_steps(dt, args.steps)
    kt = s.kernel_times()
    s.profile_kernels(False)
    vol_ms = kt["vol"][0] / kt["vol"][1]
    vol_flops = vol_flops_per_element_pairs(3) * s.K
    achieved = vol_flops / (vol_ms * 1e-3) / 1e12
    measured_peak = mhd.fp64_peak_tflops()
    step_ms_sum = sum(v[0] for v in kt.values())
    roofline = {"bound": "alu", "kernel": "k_vol<3> (entropy-conservative volume term + SSP stage)",
                "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / NOMINAL_FP64_TFLOPS, "traffic": K_VOL_TRAFFIC_BYTES,
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": "nominal B300 dense FP64 (1.25 TFLOP/s)",
                "peak_measured_dfma_tflops": measured_peak, "frac_of_measured_dfma": achieved / measured_peak,
                "flops_per_launch": vol_flops, "avg_launch_ms": vol_ms,
                "flops_definition": "117 op-equivalents per unique EC pair x p(p+1)^2 pairs per element "
                                    "(FMA = 2, div = 8)",
                "frac_minimal_count": vol_flops_per_element_minimal(3) * s.K / (vol_ms * 1e-3) / 1e12
                / NOMINAL_FP64_TFLOPS,
                "fp64_pipe_busy_ncu": 0.877,
                "kernel_share_of_step": {k: v[0] / step_ms_sum for k, v in kt.items()}}

    # end-to-end through the public API with pinned host buffers
    U, Bx, By, Bz = (torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
                     for n in (5 * s.N, s.G, s.G, s.Z))
    host = (U.reshape(5, s.N), Bx, By, Bz)
    s.get_state(host)
    e2e_steps = max(5, args.steps // 5)
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

    reduced = None
    if not args.no_side_legs and world == 1 and not args.reduced_2d2v:
        reduced = reduced_2d2v_leg(s, dt, args.steps, stream, dofs, ms_per_step)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic Orszag-Tang initial state)",
            "config": dict(workload_config(stab, args.mesh), parallelism=f"replicas{world}", dt=dt,
                           magnetic_stage="reduced 2D2V" if args.reduced_2d2v else "full",
                           tiles={"vol_elements_per_cta": tiles[0], "mag_elements_per_cta": tiles[1]}),
            "roofline": roofline, "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
        }
        if reduced is not None:
            line["reduced_2d2v"] = reduced
        if not args.no_side_legs and world == 1:
            line["degrees"] = degree_leg()
            line["adjoint"] = adjoint_leg()
            line["batched"] = batch_leg(256, 2)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
