"""Helpers shared by the tests: oracle states built from the workload module."""
import numpy as np

from oracle import Oracle
from paper_2609_10849_b300 import workloads


def oracle_state(wl, nx, ny, p, m, t=0.0):
    """Oracle with the nodal initial state of workload dict ``wl`` (reading R10)."""
    o = Oracle(nx, ny, p, m, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    kw = {"t": t} if t else {}
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y, **kw)
    XW, YW = o.coords("w")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW, **kw), *wl["B0"])
    XZ, YZ = o.coords("bz")
    Bz = wl["fields"](XZ, YZ, **kw)[5]
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, Bz)
    return o


def prim_from_cons(U, gamma):
    rho = U[0]
    u = U[1:4] / rho
    e = (U[4] - 0.5 * rho * (u ** 2).sum(axis=0)) / rho
    return rho, u, e
