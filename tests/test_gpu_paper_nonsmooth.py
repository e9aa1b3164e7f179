"""The CUDA path against the numbers the paper quotes for its periodic
nonsmooth tests, (p, m) = (2, 2), OE on both stages with s_H = s_M = 0.02,
the positivity limiter, and A.R. (C_eta = 0.2, C_s = 5) off or on, at the CFL
number 0.8 of the field loop with the CFL reading R2.

* Field loop (§4.3; 256 x 128, t = 1): retained magnetic energy (99.87 % and
  96.45 %) and the maximum field (1.412 A0 and 1.018 A0) to their printed
  digits, the transport error e_B^tr (0.11827, 0.11839) within 0.5 %, the
  A.R. current extrema [-0.0537, 0.119] within 3 %.
* Oblique blast (§4.6; 256^2, t = 0.2): final-step maximum A.R. coefficient
  3.18e-4 and magnetic-pressure maxima 2.25 -> 1.77 within 3 %.
* Orszag-Tang (§4.4; 256^2, t = 3): density maxima 6.1604 and 6.1594 within
  0.1 %, and the common contour limits of the density minimum (1.066) and of
  the magnetic-pressure maximum (5.060) within 0.5 %.

Maxima of |B| and of the magnetic pressure are taken over the DG nodes (the
library's diagnostics), the transport error and the current on 8 x 8 Gauss
points per element (the oracle's sampling).  The paper measures the
divergence in L2 (1e-15 to 1e-11); the library's metric R16 is held at
1e-12 of max |B| instead.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads

pytestmark = pytest.mark.gpu

STAB = dict(oe_hydro=1, oe_vel=1, pp=1, s_H=0.02, s_M=0.02, C_s=5.0, cfl=0.8)


def nonsmooth_solver(wl, nx, ny, ar):
    from paper_2609_10849_b300.mhd import Solver
    s = Solver(nx, ny, 2, 2, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    XW, YW = s.coords("w")
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], np.zeros(s.Z))
    s.set_params(**STAB, ar=int(ar), C_eta=0.2 if ar else 0.0)
    return s


def run_to(s, tf):
    """CFL-limited steps, the last one shortened to land on t_f."""
    t = 0.0
    while t < tf * (1.0 - 1e-14):
        st, taken = s.strang_step(min(s.compute_dt(), tf - t))
        assert st == 0
        t += taken


def close(got, want, rel):
    return abs(got / want - 1.0) <= rel


def test_field_loop():
    wl = workloads.field_loop()
    out = {}
    for ar in (0, 1):
        s = nonsmooth_solver(wl, 256, 128, ar)
        e0 = s.diagnostics()["E_mag"]
        run_to(s, 1.0)
        d = s.diagnostics()
        o = Oracle(256, 128, 2, 2, wl["gamma"], wl["domain"])
        o.set_state(*s.get_state())
        F = {c: o.sample(c, 8) for c in ("Bx", "By", "Bz", "Jz")}
        X, Y, W = F["Bx"][1], F["Bx"][2], F["Bx"][3]
        ex = wl["exact_B"](X, Y, 1.0)
        num = sum(np.sum(W * (F[c][0] - e) ** 2) for c, e in zip(("Bx", "By", "Bz"), ex))
        den = sum(np.sum(W * e ** 2) for e in ex)
        out[ar] = dict(energy=d["E_mag"] / e0, bmax=d["B_max"] / wl["A0"], etr=math.sqrt(num / den),
                       jz=(F["Jz"][0].min(), F["Jz"][0].max()), div=d["div_B"] / d["B_max"])
    for ar, energy, bmax, etr in ((0, 0.9987, 1.412, 0.11827), (1, 0.9645, 1.018, 0.11839)):
        r = out[ar]
        assert abs(r["energy"] - energy) <= 1e-4, (ar, r)  # printed to 0.01 %
        assert close(r["bmax"], bmax, 1e-3), (ar, r)
        assert close(r["etr"], etr, 5e-3), (ar, r)
        assert r["div"] <= 1e-12, (ar, r)
    assert close(out[1]["jz"][0], -0.0537, 0.03) and close(out[1]["jz"][1], 0.119, 0.03), out[1]
    # A.R. removes most of the grid-scale current (printed extrema -0.349, 0.482 without it)
    assert out[0]["jz"][1] > 3 * out[1]["jz"][1] and out[0]["jz"][0] < 3 * out[1]["jz"][0], out


def test_oblique_blast():
    wl = workloads.blast_oblique()
    pm = {}
    for ar in (0, 1):
        s = nonsmooth_solver(wl, 256, 256, ar)
        run_to(s, 0.2)
        d = s.diagnostics()
        pm[ar] = 0.5 * d["B_max"] ** 2
        assert d["div_B"] <= 1e-12 * d["B_max"]
        if ar:
            assert close(s.eta().max(), 3.18e-4, 0.03), s.eta().max()
    assert close(pm[0], 2.25, 0.03) and close(pm[1], 1.77, 0.03), pm


def test_orszag_tang():
    wl = workloads.orszag_tang_2pi()
    rho_max, rho_min, pm = {}, {}, {}
    for ar in (0, 1):
        s = nonsmooth_solver(wl, 256, 256, ar)
        run_to(s, 3.0)
        U = s.get_state()[0]
        d = s.diagnostics()
        rho_max[ar], rho_min[ar], pm[ar] = U[0].max(), U[0].min(), 0.5 * d["B_max"] ** 2
        assert d["div_B"] <= 1e-12 * d["B_max"]
    assert close(rho_max[0], 6.1604, 1e-3) and close(rho_max[1], 6.1594, 1e-3), rho_max
    assert rho_max[1] < rho_max[0]  # A.R. lowers the maximum slightly, as printed
    # contour limits common to both rows: min density, max magnetic pressure
    assert close(min(rho_min.values()), 1.066, 5e-3), rho_min
    assert close(max(pm.values()), 5.060, 5e-3), pm
