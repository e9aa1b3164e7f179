"""The CUDA path against the numbers the paper prints: Table 1 (the reduced
Alfven wave of the magnetic stage, §4.1) and, for the advected MHD vortex
(§4.2), Table 4 (spatial convergence without and with stabilisation), Table 3
(temporal self-convergence) and Table 2 (spatial convergence by
magnetic-degree parity).  Errors are evaluated on the oracle's Gauss-point
sampling of the GPU states.

* Table 1 (8 (p, m) pairs, N = 16 ... 128, Delta t = 1e-4, t_f = 1, magnetic
  substeps only; initial B_z the L2 projection onto V_h^m, reading R10): all
  128 errors to their four printed digits, except the (4, 4), N = 128 row,
  whose errors (~1e-11) are at the level of rounding after 10^4 steps.

Vortex errors and Cauchy differences are L2 norms over the central region
[-5, 5]^2 of the periodic box [-10, 10]^2; velocity and pressure are formed at
the Gauss points from the interpolated conserved fields, and E_z carries the
resistive part eta_K J_h with the coefficient of the last magnetic substep
(reading R22).

* Table 4 ((p, m) = (2, 2), N = 16 ... 128, Delta t = 1e-4, t_f = 1, H-M-H):
  all 24 entries of the unstabilised and the OE + limiter configurations, and
  the OE + A.R. rows at N = 64 and 128, are reproduced to their four printed
  digits; the OE + A.R. rows at N = 16 and 32 within 1.5 % (E_z within 7 %),
  and the final-step A.R. maximum at N = 16 within 3 %.
* Table 3 ((p, m) = (2, 2), 64^2, t_f = 1): with the M-H-M composition
  (reading R20) the printed Cauchy differences of rho, u, p and B are
  reproduced to their four printed digits (E_z and J_z to 0.5 %); the H-M-H
  composition of eq. strang-composition gives the same second order with
  smaller fluid constants.
* Table 2 (Delta t = 1e-4, t_f = 1): the velocity, magnetic field, E_z and
  J_z errors agree within 3 %; the density and pressure errors are of the same
  size.  Table 2's (2, 2) row disagrees with Table 4's unstabilised row for
  the same configuration, which we match (reading R21).
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads

pytestmark = pytest.mark.gpu


def vortex_solver(p, m, N, order=0):
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.balsara_vortex(L=10.0)
    s = Solver(N, N, p, m, wl["gamma"], wl["domain"])
    s.set_params(strang_order=order)
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
    return s, wl


def advance(s, dt, tf, chunk=500):
    n = int(round(tf / dt))
    done = 0
    while done < n:
        k = min(chunk, n - done)
        assert s.strang_steps(dt, k) == k
        done += k


GROUPS = {"rho": ("rho",), "u": ("ux", "uy", "uz"), "p": ("p",), "B": ("Bx", "By", "Bz"), "Ez": ("Ez",),
          "Jz": ("Jz",)}
ORDER = ("rho", "u", "p", "B", "Ez", "Jz")


def sampled(o, state, nq=6, eta=None):
    """Fields at nq x nq Gauss points per element: rho, B, E_z and J_z from
    their own representations, u and p from the conserved fields at the
    points.  ``eta``: element resistivity for the E_h of E_z (zero if None)."""
    o.set_state(*state)
    o.set_eta(np.zeros(o.K) if eta is None else eta)
    out = {}
    for f in ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "Ez", "Jz"):
        out[f], X, Y, W = o.sample(f, nq)
    r = out["rho"]
    for c, mc in (("ux", "mx"), ("uy", "my"), ("uz", "mz")):
        out[c] = out[mc] / r
    out["p"] = (o.gamma - 1.0) * (out["E"] - 0.5 * r * (out["ux"] ** 2 + out["uy"] ** 2 + out["uz"] ** 2))
    msk = (np.abs(X) <= 5 + 1e-9) & (np.abs(Y) <= 5 + 1e-9)
    return out, X, Y, W, msk


def vortex_errors(wl, vals, X, Y, W, msk, tf=1.0):
    """L2(Omega_e) errors of the groups of ``GROUPS`` against the exact vortex at t_f."""
    ex = wl["fields"](X, Y, t=tf)
    exB = wl["exact_B"](X, Y, t=tf)
    Xd = X - tf - 20.0 * np.round((X - tf) / 20.0)
    Yd = Y - tf - 20.0 * np.round((Y - tf) / 20.0)
    g = np.exp(0.5 * (1.0 - Xd * Xd - Yd * Yd))
    exact = {"rho": ex[0], "ux": ex[1], "uy": ex[2], "uz": ex[3], "p": ex[4], "Bx": exB[0], "By": exB[1],
             "Bz": exB[2], "Ez": g / (2 * np.pi) * (-Yd - Xd), "Jz": g * (2.0 - Xd * Xd - Yd * Yd) / (2 * np.pi)}
    return {gname: math.sqrt(sum(np.sum(W[msk] * (vals[f][msk] - exact[f][msk]) ** 2) for f in fields))
            for gname, fields in GROUPS.items()}


TABLE1 = {  # Table 1: e_u, e_B, e_E, e_J at N = 16, 32, 64, 128
    (1, 0): [(5.367e-2, 8.803e-2, 5.782e-2, 8.042e-2), (2.467e-2, 4.372e-2, 2.620e-2, 3.686e-2),
             (1.204e-2, 2.182e-2, 1.272e-2, 1.797e-2), (5.981e-3, 1.091e-2, 6.312e-3, 8.923e-3)],
    (2, 2): [(6.337e-4, 9.094e-4, 4.242e-4, 1.654e-2), (6.800e-5, 1.334e-4, 5.287e-5, 5.030e-3),
             (6.690e-6, 1.362e-5, 5.464e-6, 9.559e-4), (1.215e-6, 2.006e-6, 8.721e-7, 3.057e-4)],
    (3, 2): [(8.536e-5, 1.486e-4, 9.856e-5, 2.819e-4), (1.070e-5, 1.847e-5, 1.231e-5, 4.922e-5),
             (1.340e-6, 2.300e-6, 1.537e-6, 8.551e-6), (1.659e-7, 2.872e-7, 1.908e-7, 1.691e-6)],
    (4, 4): [(3.417e-7, 4.384e-7, 2.631e-7, 1.482e-5), (9.945e-9, 1.123e-8, 7.422e-9, 7.646e-7),
             (2.977e-10, 3.614e-10, 2.115e-10, 4.449e-8), (9.345e-12, 1.018e-11, 6.704e-12, 2.682e-9)],
    (1, 1): [(7.512e-2, 7.792e-2, 4.259e-2, 6.176e-1), (3.770e-2, 3.914e-2, 2.109e-2, 6.184e-1),
             (1.887e-2, 1.959e-2, 1.052e-2, 6.186e-1), (9.436e-3, 9.799e-3, 5.258e-3, 6.186e-1)],
    (2, 1): [(5.901e-4, 4.549e-3, 2.583e-3, 8.284e-3), (1.224e-4, 1.116e-3, 6.420e-4, 2.169e-3),
             (2.663e-5, 2.769e-4, 1.601e-4, 5.454e-4), (6.140e-6, 6.923e-5, 3.999e-5, 2.640e-4)],
    (3, 3): [(7.826e-5, 1.028e-4, 4.782e-5, 1.856e-3), (9.723e-6, 1.287e-5, 5.848e-6, 4.636e-4),
             (1.213e-6, 1.610e-6, 7.322e-7, 1.158e-4), (1.514e-7, 2.013e-7, 9.156e-8, 2.893e-5)],
    (4, 3): [(1.271e-6, 3.662e-6, 2.135e-6, 9.514e-6), (7.306e-8, 2.276e-7, 1.319e-7, 7.156e-7),
             (4.467e-9, 1.420e-8, 8.221e-9, 7.365e-8), (2.769e-10, 8.880e-10, 5.134e-10, 1.022e-8)]}


def alfven_stage_errors(p, m, N, dt=1e-4, tf=1.0, nq_init=8):
    """Table 1 run: the reduced Alfven wave advanced by magnetic substeps of
    the CUDA path; L2(Omega) errors of u, B, E_h and J_h at t_f."""
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.alfven_diagonal()
    s = Solver(N, N, p, m, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    XW, YW = s.coords("w")
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], np.zeros(s.Z))
    XQ, YQ = s.quad_coords(nq_init)
    s.set_Bz_projected(wl["fields"](XQ, YQ)[5], nq_init)
    for _ in range(int(round(tf / dt))):
        s.substep("M", dt)
    o = Oracle(N, N, p, m, wl["gamma"], wl["domain"])
    o.set_state(*s.get_state())
    nq = max(p, m) + 3
    err = {}
    for name, comps in (("u", ("ux", "uy", "uz")), ("B", ("Bx", "By", "Bz")), ("E", ("Ex", "Ey", "Ez")),
                        ("J", ("Jx", "Jy", "Jz"))):
        tot = 0.0
        for ci, c in enumerate(comps):
            v, Xq, Yq, W = o.sample(c, nq)
            a = wl["exact"](Xq, Yq, t=tf)
            if name in ("u", "B"):
                ref = a[c]
            elif name == "E":  # E = -u x B
                ref = [-(a["uy"] * a["Bz"] - a["uz"] * a["By"]), -(a["uz"] * a["Bx"] - a["ux"] * a["Bz"]),
                       -(a["ux"] * a["By"] - a["uy"] * a["Bx"])][ci]
            else:  # J = curl B of the wave
                th = Xq + Yq - wl["omega"] * tf
                ref = [0.1 * np.cos(th), -0.1 * np.cos(th), -math.sqrt(2.0) * 0.1 * np.sin(th)][ci]
            tot += np.sum(W * (v - ref) ** 2)
        err[name] = math.sqrt(tot)
    return err


@pytest.mark.parametrize("pm", list(TABLE1))
def test_table1_alfven_magnetic_stage(pm):
    """Table 1: (p, m) as given, N = 16 ... 128, Delta t = 1e-4, t_f = 1."""
    for N, printed in zip((16, 32, 64, 128), TABLE1[pm]):
        err = alfven_stage_errors(*pm, N)
        for key, want in zip("uBEJ", printed):
            # four printed digits (rounding <= 5e-4 relative); the (4,4), N = 128
            # errors of ~1e-11 are at the rounding level of 10^4 steps
            tol = 5e-2 if (pm == (4, 4) and N == 128) else 6e-4
            assert abs(err[key] / want - 1.0) <= tol, (pm, N, key, err[key], want)


TABLE4 = {  # Table 4: e_rho, e_u, e_p, e_B, e_Ez, e_Jz at N = 16, 32, 64, 128
    "none": {16: (9.863e-3, 3.668e-2, 1.345e-2, 8.791e-2, 1.607e-2, 4.256e-1),
             32: (1.522e-3, 4.669e-3, 2.587e-3, 7.262e-3, 2.071e-3, 7.411e-2),
             64: (2.829e-4, 8.723e-4, 4.998e-4, 4.224e-4, 1.719e-4, 8.737e-3),
             128: (5.596e-5, 1.442e-4, 1.004e-4, 5.054e-5, 1.852e-5, 2.152e-3)},
    "oe": {16: (1.107e-2, 1.679e-1, 2.105e-2, 8.840e-2, 1.627e-2, 4.283e-1),
           32: (4.056e-3, 4.371e-2, 7.408e-3, 7.590e-3, 2.289e-3, 7.695e-2),
           64: (8.301e-4, 7.828e-3, 1.517e-3, 5.855e-4, 3.607e-4, 9.626e-3),
           128: (9.504e-5, 6.243e-4, 1.685e-4, 6.440e-5, 3.720e-5, 2.271e-3)},
    "oe_ar": {16: (8.579e-3, 1.666e-1, 2.257e-2, 7.196e-2, 5.343e-2, 2.496e-1),
              32: (3.522e-3, 4.366e-2, 7.420e-3, 9.542e-3, 8.639e-3, 6.628e-2),
              64: (7.957e-4, 7.828e-3, 1.497e-3, 7.238e-4, 5.544e-4, 9.625e-3),
              128: (9.353e-5, 6.244e-4, 1.674e-4, 6.891e-5, 4.572e-5, 2.269e-3)}}
TABLE4_PARAMS = {"none": {},
                 "oe": dict(oe_hydro=1, oe_vel=1, pp=1, s_H=0.02, s_M=0.02),
                 "oe_ar": dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)}


@pytest.mark.parametrize("config", ["none", "oe", "oe_ar"])
def test_table4_stabilised_vortex_errors(config):
    """Table 4: (p, m) = (2, 2), Delta t = 1e-4, t_f = 1, H-M-H; the OE
    configurations use s_H = s_M = 0.02 and the positivity limiter, the last
    one A.R. with C_eta = 0.2, C_s = 5."""
    eta_max = {}
    for N, printed in TABLE4[config].items():
        s, wl = vortex_solver(2, 2, N)
        if TABLE4_PARAMS[config]:
            s.set_params(**TABLE4_PARAMS[config])
        advance(s, 1e-4, 1.0)
        eta = s.eta()
        eta_max[N] = eta.max()
        o = Oracle(N, N, 2, 2, wl["gamma"], wl["domain"])
        err = vortex_errors(wl, *sampled(o, s.get_state(), nq=8, eta=eta))
        for gname, want in zip(ORDER, printed):
            # four printed digits (rounding <= 5e-4 relative); the A.R. rows on
            # the two coarsest meshes within 1.5 %, E_z there within 7 %
            tol = 1e-3
            if config == "oe_ar" and N <= 32:
                tol = 7e-2 if gname == "Ez" else 1.5e-2
            assert abs(err[gname] / want - 1.0) <= tol, (config, N, gname, err[gname], want)
    if config == "oe_ar":
        # final-step maximum A.R. coefficient: 6.46e-2 at N = 16 (the sensor is
        # saturated there), then a rapid monotone decay (Table 4 discussion)
        assert abs(eta_max[16] / 6.46e-2 - 1.0) <= 0.03, eta_max
        rates = [math.log2(eta_max[a] / eta_max[2 * a]) for a in (16, 32, 64)]
        assert all(r > 2.5 for r in rates) and 3.5 < rates[-1] < 4.6, (eta_max, rates)
    else:
        assert max(eta_max.values()) == 0.0


@pytest.mark.parametrize("order", [1, 0])
def test_table3_temporal_cauchy_differences(order):
    """Table 3: (p, m) = (2, 2), 64^2 mesh, t_f = 1, Delta t = 1e-2 2^-l."""
    printed = {  # Delta t = 1e-2 and 5e-3 rows of Table 3
        "rho": (2.882e-6, 7.189e-7), "u": (3.526e-6, 8.682e-7), "p": (4.776e-6, 1.190e-6),
        "B": (1.277e-6, 3.128e-7), "Ez": (1.690e-6, 4.159e-7), "Jz": (6.982e-6, 1.588e-6)}
    o = Oracle(64, 64, 2, 2, 5 / 3, (-10.0, 10.0, -10.0, 10.0))
    samples = []
    for l in range(3):
        s, _ = vortex_solver(2, 2, 64, order)
        advance(s, 1e-2 * 2.0 ** (-l), 1.0, chunk=200)
        samples.append(sampled(o, s.get_state()))
    W, msk = samples[0][3], samples[0][4]
    d = {}
    for g, fields in GROUPS.items():
        d[g] = [math.sqrt(sum(np.sum(W[msk] * (samples[l][0][f][msk] - samples[l + 1][0][f][msk]) ** 2)
                              for f in fields)) for l in range(2)]
    for g in GROUPS:
        rate = math.log2(d[g][0] / d[g][1])
        if order == 1:  # the paper's numbers: rho, u, p, B to their four printed digits; E_z, J_z to 0.5 %
            assert 1.95 < rate < 2.2, (g, d[g])
            tol = 1.5e-3 if g in ("rho", "u", "p", "B") else 5e-3
            for got, want in zip(d[g], printed[g]):
                assert abs(got - want) <= tol * want, (g, got, want)
        else:  # at least second order (E_z, J_z still pre-asymptotic on the first pair)
            assert rate > 1.95, (g, d[g])
            if g in ("rho", "u", "p"):
                assert d[g][0] < printed[g][0], (g, d[g])


@pytest.mark.parametrize("p,m,N,printed", [
    (1, 0, 32, dict(rho=1.140e-2, u=9.312e-2, p=2.116e-2, B=1.410e-1, Ez=1.249e-1, Jz=2.372e-1)),
    (1, 1, 32, dict(rho=1.232e-2, u=9.285e-2, p=2.043e-2, B=5.372e-2, Ez=1.214e-2, Jz=2.786e-1)),
    (2, 2, 32, dict(rho=1.436e-3, u=4.671e-3, p=2.385e-3, B=7.290e-3, Ez=2.065e-3, Jz=7.441e-2)),
    (3, 3, 16, dict(rho=1.301e-3, u=6.320e-3, p=2.229e-3, B=7.851e-3, Ez=2.704e-3, Jz=7.654e-2)),
    (4, 4, 16, dict(rho=4.438e-4, u=9.424e-4, p=6.053e-4, B=3.994e-3, Ez=2.880e-4, Jz=4.626e-2)),
])
def test_table2_vortex_errors(p, m, N, printed):
    s, wl = vortex_solver(p, m, N)
    advance(s, 1e-4, 1.0)
    o = Oracle(N, N, p, m, wl["gamma"], wl["domain"])
    err = vortex_errors(wl, *sampled(o, s.get_state(), nq=8))
    for gname in ("u", "B", "Ez", "Jz"):
        assert abs(err[gname] / printed[gname] - 1.0) <= 0.03, (gname, err[gname], printed[gname])
    for gname in ("rho", "p"):
        assert 0.5 <= err[gname] / printed[gname] <= 2.0, (gname, err[gname], printed[gname])
