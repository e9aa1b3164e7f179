"""Pins of the oracle's magnetic stage (§3.3, eq. magnetic-dae, Theorems 3-4, Table 1).

* Theorem (semidiscrete energy balance): sum M rho u.du + (B, dB)_B + sum M rho de = 0
  on random states, ideal and resistive; a wrong transpose or sign in J_h,
  E_h, the Lorentz load or the curl breaks it.
* Theorem (divergence preservation): the in-plane increment is divergence-free.
* Ideal stage: de = 0.
* Table 1: the reduced Alfven-wave errors at N = 16 for (p, m) = (1,0), (1,1),
  (2,1), (2,2), (3,3) to the four printed digits, including the current
  stagnation of the odd (1,1) pair; the initial B_z is the L2 projection onto
  V_h^m (reading R10), the nodal interpolant misses (2,1) by 19x in e_u.
* Initial B_z projection: reproduces Q^m data, leaves a residual orthogonal to
  V_h^m (checked with an independent numpy quadrature) and is the best
  approximation, below the nodal interpolant's error.
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


def alfven_table1_state(p, m, N, nq=8):
    """Oracle with the reduced Alfven wave of Table 1: nodal u, in-plane B from
    the potential, B_z the L2 projection onto V_h^m (reading R10)."""
    wl = workloads.alfven_diagonal()
    o = oracle_state(wl, N, N, p, m)
    X, Y = o.quad_coords(nq)
    o.project_Bz(wl["fields"](X, Y)[5], nq)
    return o, wl


def table1_errors(p, m, N, dt, project_bz=True):
    if project_bz:
        o, wl = alfven_table1_state(p, m, N)
    else:
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
    (2, 1): (5.901e-4, 4.549e-3, 2.583e-3, 8.284e-3),
    (2, 2): (6.337e-4, 9.094e-4, 4.242e-4, 1.654e-2),
    (3, 3): (7.826e-5, 1.028e-4, 4.782e-5, 1.856e-3),
}


# Delta t = 2e-3 instead of the paper's 1e-4: the SSP-RK(3,3) error is then
# below 1e-5 of every entry (the same five digits as at 1e-3).
@pytest.mark.parametrize("pm", [(1, 0), (1, 1), (2, 1), (2, 2), (3, 3)])
def test_table1_alfven_magnetic_stage(pm):
    err = table1_errors(*pm, 16, 2e-3)
    ref = dict(zip("uBEJ", TABLE1_N16[pm]))
    for k in "uBEJ":  # four printed digits: rounding <= 5e-4 relative
        assert err[k] == pytest.approx(ref[k], rel=6e-4), (pm, k, err[k], ref[k])


def test_table1_needs_projected_bz():
    """With the nodal B_z interpolant the (2,1) pair is far from Table 1: its
    O(h^2) error is out of Alfvenic balance with the O(h^3) velocity and turns
    into velocity error as the wave evolves."""
    err = table1_errors(2, 1, 16, 4e-3, project_bz=False)
    assert err["u"] > 10 * TABLE1_N16[(2, 1)][0]


def _gll(m):
    if m == 0:
        return np.array([0.0])
    inner = np.sort(np.polynomial.legendre.Legendre.basis(m).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
def test_bz_projection(m):
    rng = np.random.default_rng(900 + m)
    p = max(m, 1)
    nq = m + 3
    o = Oracle(3, 2, p, m, 5 / 3, (0.0, 1.2, -0.5, 0.3))
    X, Y = o.quad_coords(nq)
    XZ, YZ = o.coords("bz")
    zero = np.zeros(5 * o.K * o.n2)
    o.set_state(zero.reshape(5, -1), np.zeros(o.G), np.zeros(o.G), np.zeros(o.Z))
    # Q^m data are reproduced: the projection equals the nodal values
    cx, cy = rng.standard_normal(m + 1), rng.standard_normal(m + 1)
    q = lambda x, y: np.polynomial.polynomial.polyval(x, cx) * np.polynomial.polynomial.polyval(y, cy)
    o.project_Bz(q(X, Y), nq)
    ref = q(XZ, YZ)
    assert np.abs(o.get_state()[3] - ref).max() <= 1e-12 * np.abs(ref).max()
    # total degree m+2: the nq-point rule is exact for (f - Pf) phi_a, so the
    # residual is orthogonal to V_h^m; checked with numpy's 20-point rule and
    # numpy-built Lagrange polynomials on element (0, 0) = [0, 0.4] x [-0.5, -0.1]
    c2 = rng.standard_normal((m + 3, m + 3))
    c2[np.add.outer(np.arange(m + 3), np.arange(m + 3)) > m + 2] = 0.0
    f = lambda x, y: np.polynomial.polynomial.polyval2d(x, y, c2)
    o.project_Bz(f(X, Y), nq)
    C = o.get_state()[3].reshape(o.K, m + 1, m + 1)[0]  # [b (y), a (x)]
    xm = _gll(m)

    def lagr(j, t):
        v = np.ones_like(t)
        for k_, xk in enumerate(xm):
            if k_ != j:
                v = v * (t - xk) / (xm[j] - xk)
        return v

    zq, wq = np.polynomial.legendre.leggauss(20)
    XX, YY = np.meshgrid(0.2 + 0.2 * zq, -0.3 + 0.2 * zq)  # [y, x]
    L = np.stack([lagr(a, zq) for a in range(m + 1)])  # [a, point]
    interp = lambda Cb: np.einsum("ba,by,ax->yx", Cb, L, L)
    r = f(XX, YY) - interp(C)
    scale = np.sqrt(np.einsum("y,x,yx->", wq, wq, f(XX, YY) ** 2))
    for a in range(m + 1):
        for b in range(m + 1):
            assert abs(np.einsum("y,x,yx,y,x->", wq, wq, r, L[b], L[a])) <= 1e-12 * scale
    # best approximation: below the nodal interpolant's error
    if m >= 1:
        g = lambda x, y: np.sin(3.0 * x + 1.0) * np.cos(2.0 * y)
        o.project_Bz(g(X, Y), nq)
        P = o.get_state()[3].reshape(o.K, m + 1, m + 1)[0]
        I = g(XZ, YZ).reshape(o.K, m + 1, m + 1)[0]
        e = lambda Cb: np.einsum("y,x,yx->", wq, wq, (g(XX, YY) - interp(Cb)) ** 2)
        assert e(P) < e(I)
