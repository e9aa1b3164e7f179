"""Pins of the oracle's diagnostics (mass, momentum, energies, entropy, field
extrema) by closed forms on states where the quadratures are exact.

The fluid integrals use the DG-GLL(p) quadrature (the mass matrix of §3.2,
exact for polynomials of degree 2p - 1 per direction) and the magnetic energy
the exact magnetic product (eq. magnetic-inner-product).  On a uniform state
every integrand is a constant; on a state with linear density and B_z every
integrand that the tests use is a polynomial the rules integrate exactly.  A
dropped factor 1/2, a wrong gamma - 1 or a wrong weight fails one of them.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from tests.util import oracle_state
from paper_2609_10849_b300 import workloads

DOM = (0.0, 1.2, 0.0, 0.7)
AREA = 1.2 * 0.7


def _set(o, rho, u, p, Bx0, By0, Bz):
    Bx, By = o.b_from_potential(np.zeros(o.G), Bx0, By0)
    o.set_primitive(rho, u, p, Bx, By, Bz)


@pytest.mark.parametrize("pm", [(1, 1), (2, 2), (3, 2), (4, 4)])
def test_uniform_state_closed_forms(pm):
    g = 1.4
    o = Oracle(5, 3, *pm, g, DOM)
    N = o.K * o.n2
    rho, u, p = 1.7, np.array([0.3, -0.2, 0.45]), 0.9
    B = np.array([0.6, -0.25, 0.35])
    _set(o, np.full(N, rho), np.repeat(u[:, None], N, axis=1), np.full(N, p), B[0], B[1], np.full(o.Z, B[2]))
    d = o.diagnostics()
    want = {
        "mass": rho * AREA, "mom_x": rho * u[0] * AREA, "mom_y": rho * u[1] * AREA, "mom_z": rho * u[2] * AREA,
        "E_kin": 0.5 * rho * (u @ u) * AREA, "E_int": p / (g - 1.0) * AREA, "E_mag": 0.5 * (B @ B) * AREA,
        "entropy": rho * (math.log(p) - g * math.log(rho)) * AREA, "B_max": math.sqrt(B @ B),
        "rho_min": rho, "p_min": p}
    for key, v in want.items():
        assert d[key] == pytest.approx(v, rel=1e-13), key
    assert abs(d["div_B"]) <= 1e-14 and d["eta_max"] == 0.0


@pytest.mark.parametrize("pm", [(1, 0), (2, 2), (3, 3)])
def test_linear_density_and_bz_closed_forms(pm):
    """rho = 1 + 0.4 x, constant u and p, B_z = 0.2 + 0.3 x (linear on every
    element, so its nodal interpolant is exact; V_h^m holds it for m >= 1, and
    for m = 0 B_z is the constant of each element, whose integral is then the
    midpoint sum)."""
    g = 5 / 3
    o = Oracle(6, 2, *pm, g, DOM)
    X, Y = o.coords("dg")
    XZ, _ = o.coords("bz")
    u = np.array([0.5, 0.1, -0.2])
    p = 0.6
    rho = 1.0 + 0.4 * X
    Bz = 0.2 + 0.3 * XZ  # for m = 0: one GLL(0) node per element, at its centre
    _set(o, rho, np.repeat(u[:, None], X.size, axis=1), np.full(X.size, p), 0.4, 0.1, Bz)
    d = o.diagnostics()
    Lx, Ly = 1.2, 0.7
    mass = (Lx + 0.2 * Lx ** 2) * Ly
    assert d["mass"] == pytest.approx(mass, rel=1e-13)
    for i, key in enumerate(("mom_x", "mom_y", "mom_z")):
        assert d[key] == pytest.approx(u[i] * mass, rel=1e-13)
    assert d["E_kin"] == pytest.approx(0.5 * (u @ u) * mass, rel=1e-13)
    assert d["E_int"] == pytest.approx(p / (g - 1.0) * Lx * Ly, rel=1e-13)
    if pm[1] == 0:
        h = Lx / 6
        int_bz2 = sum((0.2 + 0.3 * (h * (e + 0.5))) ** 2 for e in range(6)) * h * Ly
    else:
        int_bz2 = Ly * ((0.2 + 0.3 * Lx) ** 3 - 0.2 ** 3) / (3 * 0.3)
    assert d["E_mag"] == pytest.approx(0.5 * ((0.4 ** 2 + 0.1 ** 2) * Lx * Ly + int_bz2), rel=1e-13)
    assert d["rho_min"] == 1.0 and d["p_min"] == pytest.approx(p, rel=1e-14)
    # B_max is taken at the DG nodes: the largest B_z there is at x = Lx for
    # m >= 1, and the constant of the last element for m = 0
    bz_max = 0.2 + 0.3 * Lx if pm[1] else 0.2 + 0.3 * XZ.max()
    assert d["B_max"] == pytest.approx(math.sqrt(0.4 ** 2 + 0.1 ** 2 + bz_max ** 2), rel=1e-13)


def test_velocity_oe_identities_through_diagnostics():
    """The velocity OE (eq. magnetic-oe-map) keeps every element momentum,
    moves kinetic energy into internal energy one for one and does not
    decrease the entropy (eqs. magnetic-oe-energy-balance and
    magnetic-oe-entropy), seen through the diagnostics of the maps' input and
    output states."""
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 8, 6, 3, 3)
    o.set_params(oe_vel=1, s_M=0.5)
    U, Bx, By, Bz = o.get_state()
    rho = U[0]
    u = U[1:4] / rho
    e = (U[4] - 0.5 * rho * (u ** 2).sum(axis=0)) / rho
    rng = np.random.default_rng(3)
    u = u * (1.0 + 0.3 * rng.uniform(-1, 1, u.shape))  # rough: the filter acts
    U1 = U.copy()
    U1[1:4] = rho * u
    U1[4] = rho * e + 0.5 * rho * (u ** 2).sum(axis=0)
    o.set_state(U1, Bx, By, Bz)
    d0 = o.diagnostics()
    e2, u2 = o.vel_oe(rho, e, u, Bx, By, Bz, 0.05)
    U2 = U1.copy()
    U2[1:4] = rho * u2
    U2[4] = rho * e2 + 0.5 * rho * (u2 ** 2).sum(axis=0)
    o.set_state(U2, Bx, By, Bz)
    d1 = o.diagnostics()
    assert d1["E_kin"] < d0["E_kin"] * (1 - 1e-4)  # the filter acted
    scale = d0["E_kin"] + d0["E_int"]
    assert abs((d1["E_kin"] + d1["E_int"]) - (d0["E_kin"] + d0["E_int"])) <= 1e-13 * scale
    mscale = math.sqrt(d0["mass"] * 2 * d0["E_kin"])
    for key in ("mom_x", "mom_y", "mom_z"):
        assert abs(d1[key] - d0[key]) <= 1e-13 * mscale
    assert d1["entropy"] >= d0["entropy"] - 1e-13 * abs(d0["entropy"])
    assert d1["mass"] == d0["mass"]
