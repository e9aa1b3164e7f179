"""Child process of test_gpu_debug_bounds: drives the library built with index
checks (MHD_DEBUG_BUILD=1 selects libmhd_debug.so) through every path of the
step on small and one-element-wide meshes and prints the number of
out-of-range indices the checked kernels met (JSON on the last line)."""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2609_10849_b300 import mhd, workloads  # noqa: E402

assert os.path.basename(mhd.LIB_PATH) == "libmhd_debug.so"
STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)
PK = [(1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 3), (4, 4)]


def start(s, wl):
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])


def main():
    lib = mhd.lib()
    lib.mhd_debug_oob(1)
    runs = 0
    for wl_name in ("orszag_tang", "blast"):
        wl = workloads.WORKLOADS[wl_name]()
        for p, k in PK:
            for nx, ny in ((1, 1), (1, 3), (3, 1), (2, 2), (5, 3)):
                s = mhd.Solver(nx, ny, p, k, wl["gamma"], wl["domain"])
                start(s, wl)
                s.set_params(cfl=0.4, **STAB)
                for _ in range(2):
                    s.strang_step(s.compute_dt())
                s.diagnostics()
                U, Bx, By, Bz = s.get_state()
                s.hydro_rhs(U)
                s.hydro_stage_map(U, 1e-3)
                s.set_params(reduced_2d2v=1 if wl_name == "blast" else 0)
                s.strang_steps(s.compute_dt(), 2)
                s.close()
                runs += 1
    wl = workloads.rotor()
    for walls, cond in ((1, 0), (2, 2), (3, 2)):
        for p, k in ((2, 2), (3, 2)):
            s = mhd.Solver(3, 2, p, k, wl["gamma"], wl["domain"], walls=walls, conducting=cond)
            start(s, wl)
            s.mirror_fill()
            s.set_params(cfl=0.4, **STAB)
            s.strang_step(s.compute_dt())
            s.diagnostics()
            s.close()
            runs += 1
    specs = [(4, 3, 2, 2, 5 / 3, (0.0, 1.0, 0.0, 1.0)), (1, 1, 3, 3, 5 / 3, (0.0, 1.0, 0.0, 1.0)),
             (3, 5, 1, 0, 5 / 3, (0.0, 1.0, 0.0, 1.0))]
    b = mhd.Batch(specs)
    wl = workloads.orszag_tang()
    for r in b.runs:
        start(r, wl)
        r.set_params(cfl=0.4, **STAB)
    b.step(np.array([r.compute_dt() for r in b.runs]), 2)
    b.close()
    runs += 1
    print(json.dumps({"runs": runs, "oob": int(lib.mhd_debug_oob(0))}))


if __name__ == "__main__":
    main()
