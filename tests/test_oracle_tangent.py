"""Pins of the oracle's forward-mode tangent build (dual numbers).

The tangent build is the reference J dx for the adjoint's J^T lam.  It is
pinned against something other than itself: its values must be those of the
plain oracle bit for bit, and its tangents must agree with central finite
differences of the plain oracle to O(eps^2) + roundoff (on states chosen away from the kinks of |u| and max in the LLF flux).
"""
import numpy as np
import pytest

from oracle import Oracle, Tangent
from tests.test_oracle_hydro import smooth_random_state
from tests.test_oracle_magnetic import random_mag_state


def generic_state(o, rng):
    """A state away from the kinks of the LLF flux: a mean flow keeps u_x, u_y
    away from 0, and 5% nodal noise gives O(1e-2) trace jumps so that the two
    wave-speed estimates of a face are far from a tie."""
    U = smooth_random_state(o, rng)
    U[1] += 0.4 * U[0]
    U[2] += 0.3 * U[0]
    return U * (1.0 + 0.05 * rng.standard_normal(U.shape))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hydro_rhs_tangent(p):
    rng = np.random.default_rng(700 + p)
    o = Oracle(4, 3, p, p, 1.4, (0.0, 1.0, 0.0, 0.8))
    t = Tangent(4, 3, p, p, 1.4, (0.0, 1.0, 0.0, 0.8))
    U = generic_state(o, rng)
    dU = rng.standard_normal(U.shape) * 1e-3 * np.abs(U).max(axis=1, keepdims=True)
    L, dL = t.hydro_rhs_tangent(U, dU)
    assert np.array_equal(L, o.hydro_rhs(U))
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (o.hydro_rhs(U + eps * dU) - o.hydro_rhs(U - eps * dU)) / (2 * eps)
        errs.append(np.abs(fd - dL).max() / np.abs(dL).max())
    # a wrong or missing term gives an O(1) relative error at every eps; the
    # central difference itself is accurate to O(eps^2) + roundoff
    assert np.isfinite(errs).all() and max(errs) < 1e-7, errs


@pytest.mark.parametrize("pk", [(1, 0), (2, 2), (3, 3), (4, 3)])
@pytest.mark.parametrize("resistive", [False, True])
def test_mag_rhs_tangent(pk, resistive):
    p, k = pk
    rng = np.random.default_rng(720 + 10 * p + k)
    o = Oracle(3, 2, p, k, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    t = Tangent(3, 2, p, k, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    eta = rng.uniform(0.0, 0.3, o.K) if resistive else np.zeros(o.K)
    state = dict(rho=rho, e=e, u=u, Bx=Bx, By=By, Bz=Bz)
    tang = {k_: rng.standard_normal(np.shape(v)) for k_, v in state.items()}
    r, dr = t.mag_rhs_tangent(state, tang, eta)
    ro = o.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    for key in ("de", "du", "dBx", "dBy", "dBz"):
        assert np.array_equal(r[key], ro[key]), key
    eps = 1e-5  # the map is polynomial in (u, B) and rational in rho
    plus = o.mag_rhs(*(state[k_] + eps * tang[k_] for k_ in ("rho", "e", "u", "Bx", "By", "Bz")), eta)
    minus = o.mag_rhs(*(state[k_] - eps * tang[k_] for k_ in ("rho", "e", "u", "Bx", "By", "Bz")), eta)
    for key in ("de", "du", "dBx", "dBy", "dBz"):
        fd = (plus[key] - minus[key]) / (2 * eps)
        scale = max(np.abs(dr[key]).max(), 1e-300)
        if np.abs(dr[key]).max() == 0.0:
            assert np.abs(fd).max() == 0.0
            continue
        assert np.abs(fd - dr[key]).max() <= 1e-7 * scale, key


def test_strang_step_tangent():
    rng = np.random.default_rng(731)
    p = k = 3
    dom = (0.0, 1.0, 0.0, 1.0)
    o = Oracle(4, 4, p, k, 5 / 3, dom)
    t = Tangent(4, 4, p, k, 5 / 3, dom)
    U = generic_state(o, rng)
    Bx, By = rng.uniform(-0.5, 0.5, o.G), rng.uniform(-0.5, 0.5, o.G)
    Bz = rng.uniform(-0.5, 0.5, o.Z)
    x = [U, Bx, By, Bz]
    dx = [rng.standard_normal(np.shape(a)) * 1e-3 * np.abs(a).max() for a in x]
    dt = 2e-3
    t.set_state(*x)
    t.set_tangent(*dx)
    assert t.strang_step(dt)[0] == 0
    vals = t.get_state()
    tan = t.get_tangent()
    o.set_state(*x)
    o.strang_step(dt)
    for a, b in zip(vals, o.get_state()):
        assert np.array_equal(a, b)

    def step(sign, eps):
        o.set_state(*(a + sign * eps * d for a, d in zip(x, dx)))
        assert o.strang_step(dt)[0] == 0
        return o.get_state()

    errs = []
    for eps in (1e-2, 1e-3):
        P, M = step(1, eps), step(-1, eps)
        errs.append(max(np.abs((a - b) / (2 * eps) - d).max() / max(np.abs(d).max(), 1e-300)
                        for a, b, d in zip(P, M, tan)))
    assert np.isfinite(errs).all() and max(errs) < 1e-7, errs
