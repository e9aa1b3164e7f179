"""The CUDA path against the numbers the paper prints for the advected MHD
vortex (§4.2): Table 3 (temporal self-convergence) and Table 2 (spatial
convergence).  Errors and Cauchy differences are L2 norms over the central
region [-5, 5]^2 of the periodic box [-10, 10]^2, evaluated on the oracle's
Gauss-point sampling of the GPU states.

* Table 3 ((p, m) = (2, 2), 64^2, t_f = 1): with the M-H-M composition
  (reading R20) the printed Cauchy differences of rho, u, p and B are
  reproduced to their four printed digits (E_z and J_z to 0.3 %); the H-M-H
  composition of eq. strang-composition gives the same second order with
  smaller fluid constants.
* Table 2 (Delta t = 1e-4, t_f = 1): the velocity, magnetic field, E_z and
  J_z errors agree within 3 %; the density and pressure errors are of the same
  size (reading R21).
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


def sampled(o, state, nq=6):
    o.set_state(*state)
    out = {}
    for fields in GROUPS.values():
        for f in fields:
            v, X, Y, W = o.sample(f, nq)
            out[f] = v
    msk = (np.abs(X) <= 5 + 1e-9) & (np.abs(Y) <= 5 + 1e-9)
    return out, X, Y, W, msk


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
    vals, X, Y, W, msk = sampled(o, s.get_state(), nq=8)
    tf = 1.0
    ex = wl["fields"](X, Y, t=tf)
    exB = wl["exact_B"](X, Y, t=tf)
    Xd = X - tf - 20.0 * np.round((X - tf) / 20.0)
    Yd = Y - tf - 20.0 * np.round((Y - tf) / 20.0)
    g = np.exp(0.5 * (1.0 - Xd * Xd - Yd * Yd))
    exact = {"rho": ex[0], "ux": ex[1], "uy": ex[2], "uz": ex[3], "p": ex[4], "Bx": exB[0], "By": exB[1],
             "Bz": exB[2], "Ez": g / (2 * np.pi) * (-Yd - Xd), "Jz": g * (2.0 - Xd * Xd - Yd * Yd) / (2 * np.pi)}
    err = {gname: math.sqrt(sum(np.sum(W[msk] * (vals[f][msk] - exact[f][msk]) ** 2) for f in fields))
           for gname, fields in GROUPS.items()}
    for gname in ("u", "B", "Ez", "Jz"):
        assert abs(err[gname] / printed[gname] - 1.0) <= 0.03, (gname, err[gname], printed[gname])
    for gname in ("rho", "p"):
        assert 0.5 <= err[gname] / printed[gname] <= 2.0, (gname, err[gname], printed[gname])
