"""Pins of the oracle's magnetic stage (§3.3, eq. magnetic-dae, Theorems 3-4, Table 1).

* Theorem (semidiscrete energy balance): sum M rho u.du + (B, dB)_B + sum M rho de = 0
  on random states, ideal and resistive; a wrong transpose or sign in J_h,
  E_h, the Lorentz load or the curl breaks it.
* Theorem (divergence preservation): the in-plane increment is divergence-free.
* Ideal stage: de = 0.
* Table 1: the reduced Alfven-wave errors at N = 16 for (p, m) = (1,0), (1,1),
  (2,2), (3,3), including the current stagnation of the odd (1,1) pair.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads
from tests.test_oracle_hydro import mass_matrix
from tests.util import oracle_state


def random_mag_state(o, rng):
    N = o.K * o.n2
    rho = rng.uniform(0.5, 2.0, N)
    e = rng.uniform(0.5, 2.0, N)
    u = rng.uniform(-1, 1, (3, N))
    Bx = rng.uniform(-1, 1, o.G)
    By = rng.uniform(-1, 1, o.G)
    Bz = rng.uniform(-1, 1, o.Z)
    return rho, e, u, Bx, By, Bz


@pytest.mark.parametrize("p,m", [(1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 4)])
@pytest.mark.parametrize("resistive", [False, True])
def test_energy_balance(p, m, resistive):
    rng = np.random.default_rng(10 * p + m)
    o = Oracle(3, 2, p, m, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    eta = rng.uniform(0.0, 0.3, o.K) if resistive else np.zeros(o.K)
    r = o.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    M = mass_matrix(o)
    kin = (M * rho * (u * r["du"]).sum(axis=0)).sum()
    mag = o.mag_product((Bx, By, Bz), (r["dBx"], r["dBy"], r["dBz"]))
    heat = (M * rho * r["de"]).sum()
    scale = (M * rho * np.abs(u * r["du"]).sum(axis=0)).sum() + abs(mag) + abs(heat)
    assert abs(kin + mag + heat) <= 1e-13 * scale
    if resistive:
        assert heat > 0
        assert kin + mag < 0
    else:
        assert np.abs(r["de"]).max() == 0.0
        assert abs(kin) > 1e-3 * scale  # the exchange itself is not trivially zero


@pytest.mark.parametrize("p,m", [(2, 2), (3, 2), (3, 3)])
def test_divergence_free_increment(p, m):
    rng = np.random.default_rng(7)
    o = Oracle(3, 3, p, m, 5 / 3, (0.0, 1.0, 0.0, 1.0))
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    r = o.mag_rhs(rho, e, u, Bx, By, Bz, rng.uniform(0, 0.2, o.K))
    o.set_state(np.ones((5, o.K * o.n2)), r["dBx"], r["dBy"], r["dBz"])
    assert o.div_metric() <= 1e-12 * max(np.abs(r["dBx"]).max(), np.abs(r["dBy"]).max())
    o.set_state(np.ones((5, o.K * o.n2)), Bx, By, Bz)
    assert o.div_metric() > 1e-3  # random B itself is not divergence-free


def table1_errors(p, m, N, dt):
    wl = workloads.alfven_diagonal()
    o = oracle_state(wl, N, N, p, m)
    steps = int(round(1.0 / dt))
    for _ in range(steps):
        o.substep("M", dt)
    nq = max(p, m) + 3
    ex = lambda X, Y: wl["exact"](X, Y, t=1.0)
    err = {}
    for name, comps in [("u", ("ux", "uy", "uz")), ("B", ("Bx", "By", "Bz")), ("E", ("Ex", "Ey", "Ez")),
                        ("J", ("Jx", "Jy", "Jz"))]:
        tot = 0.0
        for ci, c in enumerate(comps):
            v, X, Y, W = o.sample(c, nq)
            q = ex(X, Y)
            if name in ("u", "B"):
                ref = q[c]
            elif name == "E":  # E = -u x B
                ux, uy, uz, Bx, By, Bz = (q[k] for k in ("ux", "uy", "uz", "Bx", "By", "Bz"))
                ref = [-(uy * Bz - uz * By), -(uz * Bx - ux * Bz), -(ux * By - uy * Bx)][ci]
            else:  # J = curl B, from the closed form of the wave
                th = X + Y - wl["omega"] * 1.0
                eps = 0.1
                ref = [eps * np.cos(th), -eps * np.cos(th), -math.sqrt(2) * eps * np.sin(th)][ci]
            tot += np.sum(W * (v - ref) ** 2)
        err[name] = math.sqrt(tot)
    return err


# Table 1 (reduced Alfven wave, N = 16): e_u, e_B, e_E, e_J
TABLE1_N16 = {
    (1, 0): (5.367e-2, 8.803e-2, 5.782e-2, 8.042e-2),
    (1, 1): (7.512e-2, 7.792e-2, 4.259e-2, 6.176e-1),
    (2, 2): (6.337e-4, 9.094e-4, 4.242e-4, 1.654e-2),
    (3, 3): (7.826e-5, 1.028e-4, 4.782e-5, 1.856e-3),
}


# The error quadrature and the initial interpolation of the paper are not
# stated; the oracle reproduces the odd pairs within 6 % and (2,2) within 12 %.
@pytest.mark.parametrize("pm,dt,rel", [((1, 0), 1e-2, 0.06), ((1, 1), 1e-2, 0.06), ((2, 2), 5e-3, 0.12),
                                       ((3, 3), 4e-3, 0.03)])
def test_table1_alfven_magnetic_stage(pm, dt, rel):
    err = table1_errors(*pm, 16, dt)
    ref = dict(zip("uBEJ", TABLE1_N16[pm]))
    for k in "uBEJ":
        assert err[k] == pytest.approx(ref[k], rel=rel), (pm, k, err[k], ref[k])
