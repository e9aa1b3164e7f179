"""Pins of the oracle's stage stabilisation (§3.2.2 and §3.3.3).

* Hydro OE (eq. euler-oe-map): keeps every conservative element average; is the
  identity for s_H = 0 and on piecewise-constant states; leaves a smooth state
  nearly unchanged while it damps an oscillatory one.
* OE sensor: a roundoff-constant component contributes zero (reading R8).
* PP limiter (eqs. euler-pp-*): keeps the averages and enforces the nodal
  floors rho >= 64 eps, p >= eps_p.
* Velocity OE (Proposition, eq. magnetic-oe-energy-balance): element momentum is
  kept, the kinetic loss equals the internal gain, e does not decrease, and the
  discrete entropy does not decrease (Theorem, eq. magnetic-oe-entropy).
* A.R. coefficient: zero for a constant field, non-negative, and bounded by
  C_eta max(h a/(2p+1)).
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads
from tests.test_oracle_hydro import mass_matrix, smooth_random_state
from tests.util import oracle_state, prim_from_cons

EPS = np.finfo(float).eps


def elem_avg(o, U):
    M = mass_matrix(o)
    return (U * M).reshape(U.shape[0], o.K, o.n2).sum(axis=2) / (M.reshape(o.K, o.n2).sum(axis=1))


def rough_state(o, rng):
    U = smooth_random_state(o, rng)
    U[0] *= 1 + 0.2 * rng.uniform(-1, 1, U.shape[1])
    return U


@pytest.mark.parametrize("p", [2, 3])
def test_hydro_oe_keeps_averages_and_identities(p):
    rng = np.random.default_rng(p)
    o = Oracle(4, 3, p, p, 1.4, (0.0, 1.0, 0.0, 0.75))
    o.set_params(oe_hydro=1, s_H=0.02)
    U = rough_state(o, rng)
    V = o.hydro_stage_map(U, 0.01)
    np.testing.assert_allclose(elem_avg(o, V), elem_avg(o, U), rtol=1e-13, atol=1e-14)
    assert np.abs(V - U).max() > 1e-6  # it does damp
    o.set_params(oe_hydro=1, s_H=0.0)
    np.testing.assert_allclose(o.hydro_stage_map(U, 0.01), U, rtol=1e-13, atol=1e-13)
    o.set_params(oe_hydro=1, s_H=0.02)
    Pc = np.repeat(elem_avg(o, U), o.n2, axis=1)
    np.testing.assert_allclose(o.hydro_stage_map(Pc, 0.01), Pc, rtol=1e-14, atol=1e-14)


def test_hydro_oe_smooth_vs_rough():
    rng = np.random.default_rng(5)
    o = Oracle(8, 8, 3, 3, 1.4)
    o.set_params(oe_hydro=1, s_H=0.02)
    Us = smooth_random_state(o, rng, amp=0.1)
    Ur = rough_state(o, rng)
    ds = np.abs(o.hydro_stage_map(Us, 0.002) - Us).max() / np.abs(Us).max()
    dr = np.abs(o.hydro_stage_map(Ur, 0.002) - Ur).max() / np.abs(Ur).max()
    assert dr > 10 * ds


def test_sensor_roundoff_constant_component():
    o = Oracle(4, 4, 3, 3, 1.4)
    rng = np.random.default_rng(0)
    f = np.stack([np.full(o.K * o.n2, 2.5), rng.uniform(-1, 1, o.K * o.n2)])
    s_both = o.oe_sensor(f)
    s_one = o.oe_sensor(f[1:])
    assert np.all(o.oe_sensor(f[:1]) == 0.0)
    np.testing.assert_allclose(s_both, s_one, rtol=1e-15)
    assert s_one.max() > 0


def test_pp_limiter_floors_and_averages():
    rng = np.random.default_rng(9)
    o = Oracle(4, 4, 3, 3, 1.4)
    o.set_params(pp=1)
    U = smooth_random_state(o, rng)
    # push some nodes below zero density / pressure, keeping admissible averages
    idx = rng.choice(U.shape[1], 20, replace=False)
    U[0, idx] = -0.05
    idx2 = rng.choice(U.shape[1], 20, replace=False)
    U[4, idx2] = 0.5 * (U[1, idx2] ** 2 + U[2, idx2] ** 2 + U[3, idx2] ** 2) / np.abs(U[0, idx2]) - 0.3
    a = elem_avg(o, U)
    pa = 0.4 * (a[4] - 0.5 * (a[1] ** 2 + a[2] ** 2 + a[3] ** 2) / a[0])
    assert a[0].min() > 0 and pa.min() > 0
    V = o.hydro_stage_map(U, 0.01)
    np.testing.assert_allclose(elem_avg(o, V), a, rtol=1e-12, atol=1e-13)
    rho = V[0]
    p = 0.4 * (V[4] - 0.5 * (V[1] ** 2 + V[2] ** 2 + V[3] ** 2) / rho)
    assert rho.min() >= 64 * EPS * (1 - 1e-12)
    assert p.min() > 0
    # an admissible state is left unchanged
    Us = smooth_random_state(o, rng)
    np.testing.assert_array_equal(o.hydro_stage_map(Us, 0.01), Us)


def test_velocity_oe_identities():
    rng = np.random.default_rng(11)
    o = Oracle(4, 4, 3, 3, 5 / 3)
    o.set_params(oe_vel=1, s_M=0.02)
    N = o.K * o.n2
    rho = rng.uniform(0.5, 2.0, N)
    e = rng.uniform(0.5, 2.0, N)
    u = rng.uniform(-1, 1, (3, N))
    Bx, By, Bz = rng.uniform(-1, 1, o.G), rng.uniform(-1, 1, o.G), rng.uniform(-1, 1, o.Z)
    e2, u2 = o.vel_oe(rho, e, u, Bx, By, Bz, 0.05)
    M = mass_matrix(o)
    W = (M * rho).reshape(o.K, o.n2)
    mom0 = (W[None] * u.reshape(3, o.K, o.n2)).sum(axis=2)
    mom1 = (W[None] * u2.reshape(3, o.K, o.n2)).sum(axis=2)
    np.testing.assert_allclose(mom1, mom0, rtol=1e-12, atol=1e-13)
    kin0 = 0.5 * (W * (u ** 2).sum(axis=0).reshape(o.K, o.n2)).sum(axis=1)
    kin1 = 0.5 * (W * (u2 ** 2).sum(axis=0).reshape(o.K, o.n2)).sum(axis=1)
    heat = (W * (e2 - e).reshape(o.K, o.n2)).sum(axis=1)
    np.testing.assert_allclose(kin0 - kin1, heat, rtol=1e-10, atol=1e-14)
    assert np.all(e2 >= e)
    assert np.all(heat > 0)
    # entropy of the map: sum M rho log(e+/e-) >= 0
    assert (M * rho * np.log(e2 / e)).sum() > 0
    o.set_params(oe_vel=1, s_M=0.0)
    e3, u3 = o.vel_oe(rho, e, u, Bx, By, Bz, 0.05)
    np.testing.assert_allclose(u3, u, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(e3, e)


def test_ar_coefficient_bounds():
    rng = np.random.default_rng(12)
    o = Oracle(4, 4, 2, 2, 5 / 3)
    o.set_params(ar=1, C_eta=0.2, C_s=5.0)
    N = o.K * o.n2
    rho = rng.uniform(0.5, 2.0, N)
    u = rng.uniform(-1, 1, (3, N))
    const = o.ar_coefficient(rho, u, np.full(o.G, 0.7), np.full(o.G, -0.3), np.full(o.Z, 0.2))
    assert np.all(const == 0.0)
    Bx, By, Bz = rng.uniform(-1, 1, o.G), rng.uniform(-1, 1, o.G), rng.uniform(-1, 1, o.Z)
    eta = o.ar_coefficient(rho, u, Bx, By, Bz)
    assert np.all(eta >= 0) and eta.max() > 0
    # |u_I| + |B|/sqrt(rho) <= 1 + sqrt(3)/sqrt(0.5) is a crude upper bound of a_{I,K}
    amax = 1 + 1.5 * np.sqrt(3) / np.sqrt(0.5)
    assert eta.max() <= 0.2 * (1.0 / 4) / 5 * amax * 1.0001


def test_stabilised_vortex_ar_coefficient_table4():
    """Table 4 / §4.2.3: with OE + PP + A.R. (s_H = s_M = 0.02, C_eta = 0.2,
    C_s = 5) on the smooth vortex, p = m = 2, N = 16 on [-10,10]^2, the
    maximum A.R. coefficient of the final magnetic substep at t = 1 is
    6.46e-2.  The paper uses dt = 1e-4; the value is converged in dt already
    at dt = 0.025 (0.06315 vs 0.06311 at dt = 0.0125), so that is used here."""
    wl = workloads.balsara_vortex(L=10.0)
    o = oracle_state(wl, 16, 16, 2, 2)
    o.set_params(oe_hydro=1, oe_vel=1, pp=1, ar=1, C_eta=0.2, C_s=5.0, s_H=0.02, s_M=0.02)
    for _ in range(40):
        assert o.strang_step(0.025)[0] == 0
    assert o.eta().max() == pytest.approx(6.46e-2, rel=0.05)


def _uniform_state(o, rho=1.0, u=(0.2, -0.1, 0.05), p=1.0, g=1.4):
    U = np.zeros((5, o.K * o.n2))
    U[0] = rho
    for d in range(3):
        U[1 + d] = rho * u[d]
    U[4] = p / (g - 1.0) + 0.5 * rho * sum(v * v for v in u)
    return U


def test_pp_collapses_a_vacuum_element_to_its_average():
    """Reading R9: an element whose average density is at most 64 eps is
    replaced by its average in every component (the scaling has nothing to
    scale towards)."""
    rng = np.random.default_rng(41)
    o = Oracle(3, 2, 2, 2, 1.4)
    o.set_params(pp=1)
    U = _uniform_state(o)
    k = 4
    sl = slice(k * o.n2, (k + 1) * o.n2)
    U[:, sl] *= 1e-17  # average density 1e-17 < 64 eps
    U[0, sl] *= 1.0 + 0.5 * rng.uniform(-1, 1, o.n2)
    a = elem_avg(o, U)[:, k]
    V = o.hydro_stage_map(U, 0.0)
    for c in range(5):
        assert np.all(V[c, sl] == V[c, sl][0])
        assert abs(V[c, sl][0] - a[c]) <= 1e-12 * max(abs(a[c]), 1e-300)
    other = np.ones(U.shape[1], bool)
    other[sl] = False
    np.testing.assert_array_equal(V[:, other], U[:, other])


def test_pp_density_scaling_lands_on_the_floor():
    """The density scaling (eq. euler-pp-density) is the largest one that keeps
    every node at or above eps_rho = 64 eps: afterwards the smallest nodal
    density of a limited element equals the floor (to rounding), the average is
    kept, and the nodes keep their order."""
    o = Oracle(2, 2, 3, 3, 1.4)
    o.set_params(pp=1)
    U = _uniform_state(o)
    k = 1
    sl = slice(k * o.n2, (k + 1) * o.n2)
    rho = np.linspace(1.5, 0.5, o.n2)
    rho[3] = -0.2  # one negative node, positive average
    U[0, sl] = rho
    U[1:4, sl] = 0.0
    U[4, sl] = 5.0
    a = elem_avg(o, U)[:, k]
    V = o.hydro_stage_map(U, 0.0)
    eps_rho = 64 * EPS
    assert abs(V[0, sl].min() - eps_rho) <= 1e-12
    assert abs(elem_avg(o, V)[0, k] - a[0]) <= 1e-14
    assert np.array_equal(np.argsort(V[0, sl], kind="stable"), np.argsort(rho, kind="stable"))


def test_inadmissible_average_is_rejected_and_restored():
    """Reading R9 with R3: a negative element-average density makes every
    halving of the step inadmissible; the step reports it and restores the
    state."""
    from oracle import INADMISSIBLE
    o = Oracle(3, 3, 2, 2, 1.4)
    o.set_params(pp=1, max_halvings=3)
    U = _uniform_state(o)
    U[0, 2 * o.n2:3 * o.n2] = -0.5
    z = np.zeros(o.G)
    o.set_state(U, z, z, np.zeros(o.Z))
    before = [a.copy() for a in o.get_state()]
    st, _, nrej = o.strang_step(1e-3)
    assert st == INADMISSIBLE and nrej == 4
    for a, b in zip(o.get_state(), before):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("C_s", [5.0, 2.0])
def test_ar_coefficient_unsaturated_staircase(C_s):
    """The A.R. coefficient (eqs. magnetic-ar-sensor, magnetic-ar-coefficient)
    worked out by hand on a state where the sensor response is below 1.

    Mesh 21 x 1 on [0, 2.1] x [0, 0.5] (h_x = 0.1, h_y = 0.5), rho = 2,
    u = (0.3, -0.1, 0), in-plane B = 0 and B_z = b + c e_x constant on element
    e_x (V_h^m is discontinuous).  Then Delta_Omega(B_z) = c (N - 1)/2 and the
    only tangential jumps are those of B_z across x-faces: c on each face of an
    inner element, so J_0 = 2c and sigma^B_x = 2/(N - 1); the y-direction
    jumps vanish (one element row, periodic).  With
    a_x = |u_x| + |B_z|/sqrt(rho) the inner elements get
    eta_K = C_eta h_x/(2p + 1) a_x min(C_s 2/(N - 1), 1), and the two
    elements beside the periodic seam (jump c (N - 1)) are saturated, R = 1.
    A factor in sigma, C_s, h or 2p + 1 fails this."""
    N, p, b, c, rho0, ux = 21, 2, 0.3, 0.05, 2.0, 0.3
    o = Oracle(N, 1, p, p, 5 / 3, (0.0, 2.1, 0.0, 0.5))
    o.set_params(ar=1, C_eta=0.2, C_s=C_s)
    rho = np.full(o.K * o.n2, rho0)
    u = np.zeros((3, o.K * o.n2))
    u[0], u[1] = ux, -0.1
    Bx, By = o.b_from_potential(np.zeros(o.G))
    bz_el = b + c * np.arange(N)
    Bz = np.repeat(bz_el, o.mm * o.mm)
    eta = o.ar_coefficient(rho, u, Bx, By, Bz)
    a_x = ux + bz_el / np.sqrt(rho0)
    R = np.full(N, min(C_s * 2.0 / (N - 1), 1.0))
    R[0] = R[-1] = 1.0
    want = 0.2 * 0.1 / (2 * p + 1) * a_x * R
    assert R[1] < 1.0
    np.testing.assert_allclose(eta, want, rtol=1e-13)
