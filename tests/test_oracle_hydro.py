"""Pins of the oracle's hydro stage (§3.2, eq. euler-nodal-index, Theorem 1, Algorithm 1).

* Free stream: a constant state has a zero residual.
* Theorem 1: sum_K sum_ij M L_E = 0 for all five components (conservation).
* Theorem 1: with the EC flux on faces the entropy rate sum M V.L_E vanishes;
  with LLF it is non-positive.
* Accuracy: an advected density wave (closed form) converges at order > p + 0.4
  (collocated DGSEM with LLF; the paper reports about p + 1/2 for p = 2).
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads
from tests.util import oracle_state

G = 1.4


def smooth_random_state(o, rng, amp=0.3):
    X, Y = o.coords("dg")
    x0, x1, y0, y1 = o.domain
    kx = 2 * np.pi / (x1 - x0)
    ky = 2 * np.pi / (y1 - y0)
    f = lambda: sum(rng.uniform(-1, 1) * np.sin(a * kx * X + b * ky * Y + rng.uniform(0, 6.3))
                    for a, b in [(1, 0), (0, 1), (1, 1), (2, -1)])
    rho = 1.0 + amp * f() / 4
    u = np.stack([0.5 * f(), 0.5 * f(), 0.5 * f()])
    p = 1.0 + amp * f() / 4
    U = np.zeros((5, X.size))
    U[0] = rho
    U[1:4] = rho * u
    U[4] = p / (o.gamma - 1) + 0.5 * rho * (u ** 2).sum(axis=0)
    return U


def mass_matrix(o):
    from oracle import rule
    _, w = rule("gll", o.p)
    hx = (o.domain[1] - o.domain[0]) / o.nx
    hy = (o.domain[3] - o.domain[2]) / o.ny
    return np.tile(np.outer(w, w).ravel() * hx * hy / 4, o.K)


def entropy_vars(U, g):
    rho = U[0]
    u = U[1:4] / rho
    p = (g - 1) * (U[4] - 0.5 * rho * (u ** 2).sum(axis=0))
    s = np.log(p) - g * np.log(rho)
    return np.stack([(g - s) / (g - 1) - rho * (u ** 2).sum(axis=0) / (2 * p), *(rho * u / p), -rho / p])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_free_stream(p):
    o = Oracle(3, 4, p, p, G, (0.0, 1.0, 0.0, 2.0))
    U = np.zeros((5, o.K * o.n2))
    U[0], U[1], U[2], U[3], U[4] = 1.3, 0.4, -0.7, 0.2, 3.1
    L = o.hydro_rhs(U)
    assert np.abs(L).max() < 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_conservation_and_entropy(p):
    rng = np.random.default_rng(p)
    o = Oracle(5, 4, p, p, G, (0.0, 1.0, 0.0, 0.8))
    U = smooth_random_state(o, rng)
    M = mass_matrix(o)
    L = o.hydro_rhs(U)
    scale = (M * np.abs(L)).sum(axis=1)
    assert np.all(np.abs((M * L).sum(axis=1)) <= 1e-13 * scale)
    V = entropy_vars(U, G)
    rate_llf = (M * (V * L).sum(axis=0)).sum()
    o.set_params(ec_faces=1)
    Lec = o.hydro_rhs(U)
    rate_ec = (M * (V * Lec).sum(axis=0)).sum()
    ref = (M * np.abs(V * Lec).sum(axis=0)).sum()
    assert abs(rate_ec) <= 1e-12 * ref
    assert rate_llf < 0.0
    # a wrong sign anywhere in the surface term would break conservation or entropy balance
    assert np.all(np.abs((M * Lec).sum(axis=1)) <= 1e-13 * (M * np.abs(Lec)).sum(axis=1))


def density_wave_error(N, p, tf=0.1, steps=40):
    wl = workloads.density_wave()
    o = oracle_state(wl, N, N, p, p)
    tau = tf / steps
    for _ in range(steps):
        assert o.substep("H", tau) == 0
    v, X, Y, W = o.sample("rho", p + 3)
    exact = wl["fields"](X, Y, t=tf)[0]
    return math.sqrt(np.sum(W * (v - exact) ** 2))


@pytest.mark.parametrize("p", [2, 3])
def test_density_wave_convergence(p):
    e = [density_wave_error(N, p) for N in (4, 8, 16)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert rates[-1] > p + 0.4, (e, rates)
