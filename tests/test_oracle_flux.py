"""Pins of the oracle's two-point fluxes (§3.2.1, eqs. euler-chandrashekar-flux, euler-lf-flux).

* The log mean against a 50-digit mpmath reference (reading R1).
* Consistency and symmetry of the EC flux.
* Tadmor's identity (V_R - V_L).F_ec = psi_R - psi_L, psi_d = rho u_d, with the
  Euler entropy variables written out here from eta = -rho s/(g-1): any dropped
  term or wrong sign in the flux breaks it.
* LLF consistency and Tadmor's entropy inequality for the LLF flux.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle

G = 5.0 / 3.0


def rand_state(rng, g=G):
    rho = rng.uniform(0.2, 3.0)
    u = rng.uniform(-2.0, 2.0, 3)
    p = rng.uniform(0.1, 5.0)
    return np.array([rho, *(rho * u), p / (g - 1) + 0.5 * rho * u @ u])


def entropy_vars(U, g=G):
    rho = U[0]
    u = U[1:4] / rho
    p = (g - 1) * (U[4] - 0.5 * rho * u @ u)
    s = math.log(p) - g * math.log(rho)
    return np.array([(g - s) / (g - 1) - rho * (u @ u) / (2 * p), *(rho * u / p), -rho / p])


def test_log_mean_against_mpmath():
    rng = np.random.default_rng(1)
    mpmath.mp.dps = 50
    for _ in range(400):
        a = rng.uniform(0.01, 10.0)
        b = a * (1 + 10.0 ** rng.uniform(-12, 0.5) * rng.choice([-1, 1]))
        if b <= 0:
            continue
        ref = (mpmath.mpf(a) - mpmath.mpf(b)) / (mpmath.log(a) - mpmath.log(b))
        assert abs(oracle.log_mean(a, b) - float(ref)) <= 4e-15 * float(ref)
    assert oracle.log_mean(2.5, 2.5) == pytest.approx(2.5, rel=1e-16)


def test_ec_consistency_and_symmetry():
    rng = np.random.default_rng(2)
    for _ in range(200):
        UL, UR = rand_state(rng), rand_state(rng)
        for d in (0, 1):
            np.testing.assert_allclose(oracle.ec_flux(d, UL, UL, G), oracle.phys_flux(d, UL, G),
                                       rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(oracle.ec_flux(d, UL, UR, G), oracle.ec_flux(d, UR, UL, G),
                                       rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("scale", [1.0, 1e-2, 1e-5])
def test_tadmor_identity(scale):
    rng = np.random.default_rng(3)
    for _ in range(300):
        UL = rand_state(rng)
        UR = UL + scale * (rand_state(rng) - UL)
        VL, VR = entropy_vars(UL), entropy_vars(UR)
        for d in (0, 1):
            F = oracle.ec_flux(d, UL, UR, G)
            lhs = (VR - VL) @ F
            rhs = UR[1 + d] - UL[1 + d]
            mag = np.abs(VR - VL) @ np.abs(F) + abs(UR[1 + d]) + abs(UL[1 + d])
            assert abs(lhs - rhs) <= 5e-14 * mag


def test_llf_consistency_and_entropy_inequality():
    rng = np.random.default_rng(4)
    for _ in range(300):
        Um, Up = rand_state(rng), rand_state(rng)
        for d in (0, 1):
            np.testing.assert_allclose(oracle.llf_flux(d, Um, Um, G), oracle.phys_flux(d, Um, G),
                                       rtol=1e-14, atol=1e-14)
            F = oracle.llf_flux(d, Um, Up, G)
            Vm, Vp = entropy_vars(Um), entropy_vars(Up)
            prod = (Vp - Vm) @ F - (Up[1 + d] - Um[1 + d])
            assert prod <= 1e-12 * (np.abs(Vp - Vm) @ np.abs(F) + 1.0)
