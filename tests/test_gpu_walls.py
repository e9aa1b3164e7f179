"""Reflecting walls by the method of images (reading R24) on the GPU, through
the C ABI: mhd_create_walled holds the periodic domain doubled across the
walls, mhd_mirror_fill writes the images, and the step kernels are those of
the periodic path.

* mirror_fill against an independent numpy construction of the images
  (bit for bit: copies and sign flips only), for x, y and both wall pairs,
  conducting and symmetry-plane parities;
* stabilised Strang steps against the oracle on the doubled periodic mesh
  (1e-12 per step); the GPU's images stay images (1e-13); the diagnostics
  report the physical part, whose mass is conserved (nothing crosses a wall);
* the MHD rotor of §4.5 (p = m = 2, 256^2, mirror walls, t = 0.295, CFL 0.8 of
  the reading R2): the magnetic-pressure maxima the paper quotes (0.7051
  without A.R., 0.7038 with it) within 0.5 % (measured +0.12 %, +0.11 %), the
  final A.R. maximum (8.63e-5 quoted) within 20 %, mass conserved and the
  divergence metric at 1e-12.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads
from tests.test_gpu_parity import rel
from tests.test_oracle_hydro import mass_matrix, smooth_random_state
from tests.util import mirror_images, physical_part

pytestmark = pytest.mark.gpu

STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def walled_pair(pnx, pny, p, k, walls, cond, seed):
    """A GPU walled solver and the oracle on its doubled periodic mesh, both
    with the same mirror-symmetric random state."""
    from paper_2609_10849_b300.mhd import Solver
    s = Solver(pnx, pny, p, k, 5 / 3, (0.0, 0.7, 0.0, 0.5), walls=walls, conducting=cond)
    o = Oracle(s.nx, s.ny, p, k, 5 / 3, s.domain)
    rng = np.random.default_rng(seed)
    U = smooth_random_state(o, rng)
    XW, YW = o.coords("w")
    # a potential vanishing on conducting walls (B_n = -dAz/dy or dAz/dx = 0 there),
    # periodic on the doubled domain
    fx = np.sin(np.pi * XW / 0.7) if cond & 1 else np.sin(2 * np.pi * XW / 0.7 + 0.3)
    fy = np.sin(np.pi * YW / 0.5) if cond & 2 else np.cos(2 * np.pi * YW / 0.5)
    Bx, By = o.b_from_potential(0.05 * fx * fy, 0.0 if cond & 1 else 0.3, 0.0 if cond & 2 else 0.2)
    Bz = 0.1 * rng.standard_normal(o.Z)
    return s, o, (U, Bx, By, Bz)


@pytest.mark.parametrize("walls,cond", [(1, 0), (1, 1), (2, 0), (2, 2), (3, 2), (3, 1), (3, 3), (3, 0)])
@pytest.mark.parametrize("pk", [(1, 0), (2, 2), (3, 2)])
def test_mirror_fill_matches_numpy_images(walls, cond, pk):
    s, o, state = walled_pair(3, 2, *pk, walls, cond, seed=walls * 7 + cond)
    s.set_state(*state)
    s.mirror_fill()
    got = s.get_state()
    want = mirror_images(*state, 3, 2, *pk, walls, cond)
    for a, b in zip(got, want):
        assert np.array_equal(np.asarray(a).ravel(), np.asarray(b).ravel())


@pytest.mark.parametrize("walls,cond", [(1, 0), (2, 2), (3, 2)])
@pytest.mark.parametrize("pk", [(2, 2), (3, 3)])
def test_walled_strang_steps_match_the_oracle(walls, cond, pk):
    p, k = pk
    pnx, pny = 5, 4
    s, o, state = walled_pair(pnx, pny, p, k, walls, cond, seed=3 + walls + p)
    mirrored = mirror_images(*state, pnx, pny, p, k, walls, cond)
    o.set_state(*mirrored)
    o.set_params(cfl=0.4, **STAB)
    s.set_params(cfl=0.4, **STAB)
    s.set_state(*state)
    s.mirror_fill()
    M = mass_matrix(o).reshape(s.ny, s.nx, p + 1, p + 1)[:pny, :pnx]
    m_phys0 = (M * physical_part(*mirrored, s.nx, s.ny, pnx, pny, p, k)[0][0]).sum()
    assert s.diagnostics()["mass"] == pytest.approx(m_phys0, rel=1e-13)
    for _ in range(2):
        dt = o.cfl_dt()
        assert abs(s.compute_dt() / dt - 1.0) <= 1e-13
        assert o.strang_step(dt)[0] == 0
        assert s.strang_step(dt)[0] == 0
        Uo, Bxo, Byo, Bzo = o.get_state()
        Ug, Bxg, Byg, Bzg = s.get_state()
        bscale = max(np.abs(Bxo).max(), np.abs(Byo).max(), np.abs(Bzo).max())
        assert rel(Ug, Uo) <= 1e-12
        for a, b in ((Bxg, Bxo), (Byg, Byo), (Bzg, Bzo)):
            assert rel(a, b, bscale) <= 1e-12
        imaged = mirror_images(Ug, Bxg, Byg, Bzg, pnx, pny, p, k, walls, cond)
        for a, b in zip((Ug, Bxg, Byg, Bzg), imaged):
            assert np.abs(np.asarray(a).ravel() - np.asarray(b).ravel()).max() <= 1e-13 * max(np.abs(b).max(), 1.0)
        d = s.diagnostics()
        assert abs(d["mass"] - m_phys0) <= 1e-13 * m_phys0
        assert d["div_B"] <= 1e-12 * d["B_max"]


def test_mirror_fill_refuses_a_periodic_context():
    from paper_2609_10849_b300.mhd import MhdError, Solver
    s = Solver(4, 4, 2, 2, 5 / 3)
    with pytest.raises(MhdError, match="walled"):
        s.mirror_fill()


def run_to(s, tf):
    t = 0.0
    while t < tf * (1.0 - 1e-14):
        st, taken = s.strang_step(min(s.compute_dt(), tf - t))
        assert st == 0
        t += taken


def test_rotor_with_mirror_walls():
    """§4.5: p = m = 2 on 256^2, mirror walls, t = 0.295, without and with A.R.
    The paper quotes the magnetic-pressure maxima 0.7051 and 0.7038, the
    final-step maximum A.R. coefficient 8.63e-5 and an L2 divergence of 4.6e-12."""
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.rotor()
    pm, eta = {}, {}
    for ar in (0, 1):
        s = Solver(256, 256, 2, 2, wl["gamma"], wl["domain"], walls=wl["walls"], conducting=wl["conducting"])
        X, Y = s.coords("dg")
        rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
        s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
        XW, YW = s.coords("w")
        s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], np.zeros(s.Z))
        s.mirror_fill()
        s.set_params(oe_hydro=1, oe_vel=1, pp=1, s_H=0.02, s_M=0.02, C_s=5.0, cfl=0.8, ar=ar,
                     C_eta=0.2 if ar else 0.0)
        m0 = s.diagnostics()["mass"]
        run_to(s, 0.295)
        d = s.diagnostics()
        pm[ar] = 0.5 * d["B_max"] ** 2
        eta[ar] = d["eta_max"]
        assert abs(d["mass"] - m0) <= 1e-12 * m0
        assert d["div_B"] <= 1e-12 * d["B_max"]
    # measured 0.70596 and 0.70460 (+0.12 %, +0.11 %); A.R. lowers the maximum slightly, as printed
    assert abs(pm[0] / 0.7051 - 1.0) <= 5e-3 and abs(pm[1] / 0.7038 - 1.0) <= 5e-3, pm
    assert pm[1] < pm[0]
    # final-step A.R. maximum: measured 9.90e-5 against the quoted 8.63e-5 (reading R23: the paper's
    # quoted maxima come from a diagnostic of its own; the oblique blast matches to 3 %)
    assert eta[0] == 0.0 and abs(eta[1] / 8.63e-5 - 1.0) <= 0.2, eta
