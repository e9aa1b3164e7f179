"""Seeded synthetic initial states of the benchmark workloads.

This module holds no arithmetic of the numerical method: it only evaluates the
analytic initial fields of the paper's test problems at coordinates that the
caller supplies (each side computes its own node coordinates), plus the
splitmix64 stream used for seeded variants.  Both the CUDA path and the CPU
oracle take their inputs from here.

Each workload returns a dict with

* ``fields(x, y) -> (rho, ux, uy, uz, p, Bz)`` nodal primitive fields,
* ``Az(x, y)`` a periodic potential whose rotated gradient is the varying part
  of the in-plane field (the field itself is built by each side from the
  potential's nodal interpolant, so that it is discretely divergence-free),
* ``B0 = (Bx0, By0)`` the constant part of the in-plane field,
* ``domain = (x0, x1, y0, y1)``, ``gamma``.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
SEED = 20260910


def splitmix64(state: int):
    """One step of splitmix64 (Steele, Lea & Flood 2014): returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Rng:
    """Uniform doubles in [0,1) from the top 53 bits of splitmix64."""

    def __init__(self, seed: int = SEED):
        self.state = seed & MASK64

    def uniform(self, lo=0.0, hi=1.0):
        self.state, z = splitmix64(self.state)
        return lo + (hi - lo) * ((z >> 11) * (1.0 / (1 << 53)))


def alfven_rotated(alpha=math.pi / 6, amp=0.1, rho0=1.0, p0=0.1, Bpar=1.0, gamma=5.0 / 3.0):
    """Circularly polarised Alfven wave along x_par = x cos a + y sin a on
    [0, 1/cos a] x [0, 1/sin a]: v_perp = B_perp = amp sin(2 pi x_par),
    v_z = B_z = amp cos(2 pi x_par).  With v = +dB/sqrt(rho) it travels towards
    -x_par at speed Bpar/sqrt(rho): q(x, t) = q0(x_par + t Bpar/sqrt(rho))."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    c = Bpar / math.sqrt(rho0)

    def xpar(x, y, t=0.0):
        return x * ca + y * sa + c * t

    def fields(x, y, t=0.0):
        s = xpar(x, y, t)
        vperp = amp * np.sin(2 * np.pi * s)
        vz = amp * np.cos(2 * np.pi * s)
        ux, uy = -sa * vperp, ca * vperp
        one = np.ones_like(s)
        return rho0 * one, ux, uy, vz, p0 * one, vz.copy()

    def Az(x, y, t=0.0):
        # grad^perp A = A'(x_par) (-sin a, cos a) = B_perp t  =>  A' = amp sin(2 pi x_par)
        return -amp * np.cos(2 * np.pi * xpar(x, y, t)) / (2 * np.pi)

    def exact_B(x, y, t=0.0):
        s = xpar(x, y, t)
        bperp = amp * np.sin(2 * np.pi * s)
        return Bpar * ca - sa * bperp, Bpar * sa + ca * bperp, amp * np.cos(2 * np.pi * s)

    return dict(name="alfven", fields=fields, Az=Az, B0=(Bpar * ca, Bpar * sa),
                domain=(0.0, 1.0 / ca, 0.0, 1.0 / sa), gamma=gamma, exact_B=exact_B)


def alfven_diagonal(eps=0.1, rho0=1.0, p0=1.0, B0=1.0, gamma=5.0 / 3.0):
    """Reduced magnetic-stage test of §4.1: wave along n = (1,1)/sqrt2 on
    [0, 2 pi]^2, theta = x + y - omega t, omega = sqrt2 B0/sqrt(rho0),
    B = B0 n + eps (t cos theta + e_z sin theta), u = -eps/sqrt(rho0)(...)."""
    k = math.sqrt(2.0)
    om = k * B0 / math.sqrt(rho0)
    r2 = 1.0 / math.sqrt(2.0)

    def th(x, y, t):
        return x + y - om * t

    def exact(x, y, t=0.0):
        c, s = np.cos(th(x, y, t)), np.sin(th(x, y, t))
        Bx = B0 * r2 - eps * r2 * c
        By = B0 * r2 + eps * r2 * c
        Bz = eps * s
        a = -eps / math.sqrt(rho0)
        ux, uy, uz = -a * r2 * c, a * r2 * c, a * s
        return dict(Bx=Bx, By=By, Bz=Bz, ux=ux, uy=uy, uz=uz)

    def fields(x, y, t=0.0):
        q = exact(x, y, t)
        one = np.ones_like(x)
        return rho0 * one, q["ux"], q["uy"], q["uz"], p0 * one, q["Bz"]

    def Az(x, y, t=0.0):
        # eps t cos(theta) = grad^perp A with A = eps sin(theta)/sqrt2
        return eps * r2 * np.sin(th(x, y, t))

    return dict(name="alfven_diag", fields=fields, Az=Az, B0=(B0 * r2, B0 * r2),
                domain=(0.0, 2 * math.pi, 0.0, 2 * math.pi), gamma=gamma, exact=exact, omega=om)


def orszag_tang(a_v=1.0, a_B=1.0, phi=(0.0, 0.0, 0.0), gamma=5.0 / 3.0):
    """Orszag-Tang vortex on [0,1]^2 (scaled variant): rho = 25/(36 pi),
    p = 5/(12 pi), v = a_v(-sin(2 pi y + phi1), sin(2 pi x + phi2), 0),
    B = a_B(-sin(2 pi y + phi1), sin(4 pi x + phi3), 0)/sqrt(4 pi)."""
    f1, f2, f3 = phi
    s4 = 1.0 / math.sqrt(4 * math.pi)

    def fields(x, y):
        one = np.ones_like(x)
        return (25.0 / (36.0 * math.pi) * one, -a_v * np.sin(2 * np.pi * y + f1),
                a_v * np.sin(2 * np.pi * x + f2), 0.0 * one, 5.0 / (12.0 * math.pi) * one, 0.0 * one)

    def Az(x, y):
        return -a_B * s4 * (np.cos(2 * np.pi * y + f1) / (2 * np.pi) + np.cos(4 * np.pi * x + f3) / (4 * np.pi))

    return dict(name="orszag_tang", fields=fields, Az=Az, B0=(0.0, 0.0), domain=(0.0, 1.0, 0.0, 1.0),
                gamma=gamma)


def orszag_tang_variant(i: int, seed: int = SEED):
    """Seeded Orszag-Tang variant number i: amplitudes U(0.8,1.2), phases U(0, 2 pi)."""
    r = Rng(seed + i)
    a_v = r.uniform(0.8, 1.2)
    a_B = r.uniform(0.8, 1.2)
    phi = (r.uniform(0, 2 * math.pi), r.uniform(0, 2 * math.pi), r.uniform(0, 2 * math.pi))
    return orszag_tang(a_v, a_B, phi)


def blast(gamma=1.4, p_in=1000.0, p_out=0.1, r0=0.1, B=100.0):
    """MHD blast wave on [-1/2,1/2]^2: rho = 1, v = 0, p = p_in for r < r0,
    B = (B/sqrt(4 pi)) (1/sqrt2, 1/sqrt2, 0)."""
    b = B / math.sqrt(4 * math.pi) / math.sqrt(2.0)

    def fields(x, y):
        one = np.ones_like(x)
        r = np.sqrt(x * x + y * y)
        p = np.where(r < r0, p_in, p_out)
        return one, 0.0 * one, 0.0 * one, 0.0 * one, p, 0.0 * one

    def Az(x, y):
        return 0.0 * x

    return dict(name="blast", fields=fields, Az=Az, B0=(b, b), domain=(-0.5, 0.5, -0.5, 0.5), gamma=gamma)


def orszag_tang_2pi(gamma=5.0 / 3.0):
    """Orszag-Tang vortex of §4.4 on the periodic [0, 2 pi]^2: rho = gamma^2,
    p = gamma, u = (-sin y, sin x, 0), B = (-sin y, sin 2x, 0) = curl(A e_z)
    with A = cos y + cos(2x)/2; ``Az`` is the potential of the library's
    grad-perp convention B = (-dAz/dy, dAz/dx), i.e. Az = -A."""
    def fields(x, y):
        one = np.ones_like(x)
        return gamma * gamma * one, -np.sin(y), np.sin(x), 0.0 * one, gamma * one, 0.0 * one

    def Az(x, y):
        return -(np.cos(y) + 0.5 * np.cos(2.0 * x))

    return dict(name="orszag_tang_2pi", fields=fields, Az=Az, B0=(0.0, 0.0),
                domain=(0.0, 2 * math.pi, 0.0, 2 * math.pi), gamma=gamma)


def blast_oblique(gamma=5.0 / 3.0, p_in=10.0, p_out=0.1, r0=0.1):
    """Oblique MHD blast wave of §4.6 on the periodic [0, 1]^2: rho = 1, u = 0,
    B = (cos pi/4, sin pi/4, 0), p = p_in in the disk of radius r0 about
    (1/2, 1/2) and p_out outside it."""
    def fields(x, y):
        one = np.ones_like(x)
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
        return one, 0.0 * one, 0.0 * one, 0.0 * one, np.where(r < r0, p_in, p_out), 0.0 * one

    def Az(x, y):
        return 0.0 * x

    c = math.cos(math.pi / 4)
    return dict(name="blast_oblique", fields=fields, Az=Az, B0=(c, c), domain=(0.0, 1.0, 0.0, 1.0), gamma=gamma)


def rotor(r0=0.1, r1=0.115, rho_in=10.0, u0=1.0, p0=0.5, gamma=5.0 / 3.0):
    """MHD rotor of §4.5 on [0,1]^2 with mirror walls: a dense core (rho = 10
    for r < r0 about (1/2, 1/2)) in rigid rotation with unit tangential speed at
    r0; over r0 <= r < r1 density and tangential speed taper linearly to the
    ambient rho = 1, u = 0; p = 1/2 everywhere; B = (2.5/sqrt(4 pi), 0, 0).
    Walls in x and y (walls = 3): the field crosses the x-walls, so they are
    symmetry planes for B, and lies along the y-walls, which are conducting
    (conducting = 2) - the wall parities that keep the uniform field."""
    b = 2.5 / math.sqrt(4 * math.pi)

    def fields(x, y):
        dx, dy = x - 0.5, y - 0.5
        r = np.sqrt(dx * dx + dy * dy)
        f = np.clip((r1 - r) / (r1 - r0), 0.0, 1.0)
        rho = 1.0 + (rho_in - 1.0) * f
        speed = np.where(r < r0, u0 * r / r0, u0 * f)
        inv = np.where(r > 0, 1.0 / np.maximum(r, 1e-300), 0.0)
        one = np.ones_like(x)
        return rho, -speed * dy * inv, speed * dx * inv, 0.0 * one, p0 * one, 0.0 * one

    def Az(x, y):
        return 0.0 * x

    return dict(name="rotor", fields=fields, Az=Az, B0=(b, 0.0), domain=(0.0, 1.0, 0.0, 1.0), gamma=gamma,
                walls=3, conducting=2)


def field_loop(A0=1e-3, R=0.3, u=(2.0, 1.0), gamma=5.0 / 3.0):
    """Weak-field loop of §4.3 on the periodic [-1, 1] x [-1/2, 1/2]: rho = p = 1,
    u = (2, 1, 0), B = curl(A e_z) with A = A0 max(R - r, 0) (``Az`` = -A in
    the library's convention B = (-dAz/dy, dAz/dx)).  ``exact_B`` is the loop
    translated by u t (periodically): |B| = A0 inside r < R."""
    Lx, Ly = 2.0, 1.0

    def fields(x, y):
        one = np.ones_like(x)
        return one, u[0] * one, u[1] * one, 0.0 * one, one, 0.0 * one

    def Az(x, y):
        return -A0 * np.maximum(R - np.sqrt(x * x + y * y), 0.0)

    def exact_B(x, y, t=0.0):
        xd = x - u[0] * t
        yd = y - u[1] * t
        xd = xd - Lx * np.round(xd / Lx)
        yd = yd - Ly * np.round(yd / Ly)
        r = np.sqrt(xd * xd + yd * yd)
        inside = (r < R) & (r > 0)
        rs = np.where(r > 0, r, 1.0)
        return np.where(inside, -A0 * yd / rs, 0.0), np.where(inside, A0 * xd / rs, 0.0), 0.0 * x

    return dict(name="field_loop", fields=fields, Az=Az, B0=(0.0, 0.0), domain=(-1.0, 1.0, -0.5, 0.5),
                gamma=gamma, exact_B=exact_B, A0=A0)


def balsara_vortex(L=5.0, gamma=5.0 / 3.0, ubar=(1.0, 1.0)):
    """Isodensity MHD vortex (§4.2) on the periodic box [-L, L]^2 with
    minimum-image displacement: rho = 1, u = ubar + g/(2 pi)(-y, x),
    p = 1 - r^2 g^2/(8 pi^2), B = g/(2 pi)(-y, x), g = exp((1 - r^2)/2)."""
    P = 2 * L

    def disp(x, y, t):
        X = x - ubar[0] * t
        Y = y - ubar[1] * t
        X = X - P * np.round(X / P)
        Y = Y - P * np.round(Y / P)
        return X, Y

    def fields(x, y, t=0.0):
        X, Y = disp(x, y, t)
        r2 = X * X + Y * Y
        gg = np.exp(0.5 * (1 - r2))
        one = np.ones_like(x)
        return (one, ubar[0] - gg / (2 * np.pi) * Y, ubar[1] + gg / (2 * np.pi) * X, 0.0 * one,
                1.0 - r2 * gg * gg / (8 * np.pi ** 2), 0.0 * one)

    def Az(x, y, t=0.0):
        # grad^perp A = (-dA/dy, dA/dx) = g/(2 pi) (-Y, X)  =>  A = -g/(2 pi)
        X, Y = disp(x, y, t)
        return -np.exp(0.5 * (1 - (X * X + Y * Y))) / (2 * np.pi)

    def exact_B(x, y, t=0.0):
        X, Y = disp(x, y, t)
        gg = np.exp(0.5 * (1 - (X * X + Y * Y)))
        return -gg / (2 * np.pi) * Y, gg / (2 * np.pi) * X, 0.0 * X

    return dict(name="vortex", fields=fields, Az=Az, B0=(0.0, 0.0), domain=(-L, L, -L, L), gamma=gamma,
                exact_B=exact_B)


def density_wave(amp=0.2, u=(1.0, 0.5, 0.3), p0=1.0, gamma=1.4):
    """Smooth advected density wave on [0,1]^2 (pure Euler, B = 0):
    rho = 1 + amp sin(2 pi (x + y)), constant u and p; exact solution
    rho(x - u_x t, y - u_y t)."""

    def fields(x, y, t=0.0):
        one = np.ones_like(x)
        rho = 1.0 + amp * np.sin(2 * np.pi * ((x - u[0] * t) + (y - u[1] * t)))
        return rho, u[0] * one, u[1] * one, u[2] * one, p0 * one, 0.0 * one

    def Az(x, y, t=0.0):
        return 0.0 * x

    return dict(name="density_wave", fields=fields, Az=Az, B0=(0.0, 0.0), domain=(0.0, 1.0, 0.0, 1.0),
                gamma=gamma)


def vortex_target_density(X, Y, seed: int = SEED):
    """Seeded perturbed initial density of the adjoint workload (a target run
    starts from it): rho* = 1 + 0.01 sum_{k=1..4} a_k sin(2 pi (kx_k x + ky_k y)/10
    + phi_k), a_k ~ U(-1, 1), kx_k, ky_k in {1, 2}, phi_k ~ U(0, 2 pi)."""
    r = Rng(seed + 5)
    out = np.ones_like(X)
    for _ in range(4):
        a = r.uniform(-1, 1)
        kx = 1 + min(int(r.uniform() * 2), 1)
        ky = 1 + min(int(r.uniform() * 2), 1)
        ph = r.uniform(0, 2 * math.pi)
        out = out + 0.01 * a * np.sin(2 * np.pi * (kx * X + ky * Y) / 10 + ph)
    return out


BATCH_MESHES = (32, 48, 64, 96, 128, 192, 256)
BATCH_DEGREES = (2, 3, 4)


def batch_specs(nruns: int, seed: int = SEED):
    """Seeded (N, p) of the batched workload: N from BATCH_MESHES (an N x N
    mesh), p = k from BATCH_DEGREES, drawn uniformly; run i is the Orszag-Tang
    variant orszag_tang_variant(i)."""
    r = Rng(seed ^ 0xB47C4)
    out = []
    for _ in range(nruns):
        N = BATCH_MESHES[min(int(r.uniform() * len(BATCH_MESHES)), len(BATCH_MESHES) - 1)]
        p = BATCH_DEGREES[min(int(r.uniform() * len(BATCH_DEGREES)), len(BATCH_DEGREES) - 1)]
        out.append((N, p))
    return out


WORKLOADS = {
    "alfven": alfven_rotated,
    "alfven_diag": alfven_diagonal,
    "orszag_tang": orszag_tang,
    "blast": blast,
    "vortex": balsara_vortex,
    "density_wave": density_wave,
    "rotor": rotor,
}
