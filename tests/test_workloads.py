"""The synthetic workloads' potentials produce the magnetic fields their
docstrings state, in the library's convention B = (B0x - dAz/dy, B0y + dAz/dx)
(checked by central differences at random points), and the fields that are
meant to vanish do.  The sign of a potential is easy to get wrong and would
silently turn a test problem into another one."""
import math

import numpy as np
import pytest

from paper_2609_10849_b300 import workloads


def curl_B(wl, x, y, h=1e-6, **kw):
    Az = wl["Az"]
    bx = wl["B0"][0] - (Az(x, y + h, **kw) - Az(x, y - h, **kw)) / (2 * h)
    by = wl["B0"][1] + (Az(x + h, y, **kw) - Az(x - h, y, **kw)) / (2 * h)
    return bx, by


def points(wl, rng, n=64):
    x0, x1, y0, y1 = wl["domain"]
    return rng.uniform(x0, x1, n), rng.uniform(y0, y1, n)


def test_orszag_tang_2pi_field():
    wl = workloads.orszag_tang_2pi()
    x, y = points(wl, np.random.default_rng(1))
    bx, by = curl_B(wl, x, y)
    assert np.allclose(bx, -np.sin(y), atol=1e-8) and np.allclose(by, np.sin(2 * x), atol=1e-8)
    rho, ux, uy, uz, p, bz = wl["fields"](x, y)
    g = wl["gamma"]
    assert np.allclose(rho, g * g) and np.allclose(p, g) and not np.any(uz) and not np.any(bz)
    assert np.allclose(ux, -np.sin(y)) and np.allclose(uy, np.sin(x))


def test_orszag_tang_scaled_field():
    wl = workloads.orszag_tang()
    x, y = points(wl, np.random.default_rng(2))
    bx, by = curl_B(wl, x, y)
    s4 = 1.0 / math.sqrt(4 * math.pi)
    assert np.allclose(bx, -s4 * np.sin(2 * np.pi * y), atol=1e-8)
    assert np.allclose(by, s4 * np.sin(4 * np.pi * x), atol=1e-8)


def test_field_loop_field():
    wl = workloads.field_loop()
    x, y = points(wl, np.random.default_rng(3), 400)
    r = np.hypot(x, y)
    keep = (np.abs(r - 0.3) > 1e-4) & (r > 1e-4)  # away from the kinks of A
    bx, by = curl_B(wl, x[keep], y[keep])
    ex = wl["exact_B"](x[keep], y[keep])
    assert np.allclose(bx, ex[0], atol=1e-9) and np.allclose(by, ex[1], atol=1e-9)
    inside = r[keep] < 0.3
    assert np.allclose(np.hypot(bx, by)[inside], wl["A0"]) and np.allclose(np.hypot(bx, by)[~inside], 0.0)
    # one traversal (u = (2, 1), box 2 x 1) brings the loop back
    assert np.allclose(wl["exact_B"](x, y, 1.0)[0], wl["exact_B"](x, y, 0.0)[0])


@pytest.mark.parametrize("t", [0.0, 0.7])
def test_vortex_field(t):
    wl = workloads.balsara_vortex(L=10.0)
    x, y = points(wl, np.random.default_rng(4))
    bx, by = curl_B(wl, x, y, t=t)
    ex = wl["exact_B"](x, y, t=t)
    assert np.allclose(bx, ex[0], atol=1e-8) and np.allclose(by, ex[1], atol=1e-8)


def test_alfven_diagonal_field():
    wl = workloads.alfven_diagonal()
    x, y = points(wl, np.random.default_rng(5))
    bx, by = curl_B(wl, x, y, t=0.3)
    ex = wl["exact"](x, y, t=0.3)
    assert np.allclose(bx, ex["Bx"], atol=1e-8) and np.allclose(by, ex["By"], atol=1e-8)
    # the exact wave is divergence-free and Alfvenic: u = -(B - B0 n)/sqrt(rho0)
    n = np.array([1.0, 1.0]) / math.sqrt(2.0)
    assert np.allclose(ex["ux"], -(ex["Bx"] - n[0])) and np.allclose(ex["uy"], -(ex["By"] - n[1]))


def test_blast_oblique_state():
    wl = workloads.blast_oblique()
    x, y = points(wl, np.random.default_rng(6), 2000)
    rho, ux, uy, uz, p, bz = wl["fields"](x, y)
    r = np.hypot(x - 0.5, y - 0.5)
    assert np.all(p[r < 0.1] == 10.0) and np.all(p[r >= 0.1] == 0.1)
    bx, by = curl_B(wl, x, y)
    assert np.allclose(bx, math.cos(math.pi / 4)) and np.allclose(by, math.sin(math.pi / 4))
    assert not np.any(ux) and not np.any(uy) and not np.any(uz) and not np.any(bz)
