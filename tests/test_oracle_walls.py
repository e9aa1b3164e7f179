"""Reflecting walls by the method of images (reading R24), pinned on the oracle.

A wall problem is the periodic problem on the domain doubled across the walls
with mirror-image data: normal velocity odd, the other fluid fields even, B
with the parity of a conducting wall or of a symmetry plane.  That is exact
only if the discrete step is reflection-equivariant; the oracle's is (its
rules, nodes and operators are symmetric), so one stabilised Strang step of a
mirror-symmetric state is mirror-symmetric again to rounding, no mass crosses
the mirror planes, and a conducting wall keeps B_n = 0 on it."""
import numpy as np
import pytest

from oracle import Oracle
from tests.test_oracle_hydro import mass_matrix, smooth_random_state
from tests.util import mirror_images, physical_part

STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def walled_oracle(pnx, pny, p, m, walls, cond, seed):
    rng = np.random.default_rng(seed)
    nx = pnx * (2 if walls & 1 else 1)
    ny = pny * (2 if walls & 2 else 1)
    o = Oracle(nx, ny, p, m, 5 / 3, (0.0, 0.7 * nx / pnx, 0.0, 0.5 * ny / pny))
    U = smooth_random_state(o, rng)
    XW, YW = o.coords("w")
    # a potential vanishing on conducting walls, periodic on the doubled domain
    fx = np.sin(np.pi * XW / 0.7) if cond & 1 else np.sin(2 * np.pi * XW / 0.7 + 0.3)
    fy = np.sin(np.pi * YW / 0.5) if cond & 2 else np.cos(2 * np.pi * YW / 0.5)
    Bx, By = o.b_from_potential(0.05 * fx * fy, 0.3 if not (cond & 1) else 0.0, 0.2 if not (cond & 2) else 0.0)
    Bz = 0.1 * rng.standard_normal(o.Z)
    o.set_state(*mirror_images(U, Bx, By, Bz, pnx, pny, p, m, walls, cond))
    o.set_params(cfl=0.4, **STAB)
    assert o.div_metric() <= 1e-12 * max(np.abs(Bx).max(), np.abs(By).max())  # the images keep div B = 0
    return o, nx, ny


@pytest.mark.parametrize("walls,cond", [(1, 0), (2, 2), (3, 2), (3, 3)])
@pytest.mark.parametrize("pm", [(2, 2), (3, 2)])
def test_images_stay_images(walls, cond, pm):
    p, m = pm
    pnx, pny = 4, 3
    o, nx, ny = walled_oracle(pnx, pny, p, m, walls, cond, seed=walls * 10 + cond + p)
    m0 = o.diagnostics()["mass"]
    U0, Bx0, By0, Bz0 = o.get_state()
    phys0 = physical_part(U0, Bx0, By0, Bz0, nx, ny, pnx, pny, p, m)
    dt = o.cfl_dt()
    assert o.strang_step(dt)[0] == 0
    U, Bx, By, Bz = o.get_state()
    mirrored = mirror_images(U, Bx, By, Bz, pnx, pny, p, m, walls, cond)
    for a, b in zip((U, Bx, By, Bz), mirrored):
        scale = max(np.abs(b).max(), 1e-300)
        assert np.abs(a - b).max() <= 1e-13 * scale
    # the physical part moved (the test is not vacuous), the total mass is kept,
    # and so is the physical part's own mass: nothing crosses a wall
    phys1 = physical_part(U, Bx, By, Bz, nx, ny, pnx, pny, p, m)
    assert np.abs(phys1[0] - phys0[0]).max() > 1e-6
    assert abs(o.diagnostics()["mass"] - m0) <= 1e-13 * m0
    M = mass_matrix(o).reshape(ny, nx, p + 1, p + 1)[:pny, :pnx]
    mp0, mp1 = (M * phys0[0][0]).sum(), (M * phys1[0][0]).sum()
    assert abs(mp1 - mp0) <= 1e-13 * mp0
    if walls & 2 and cond & 2:  # conducting y-walls: B_y stays 0 on them (to rounding: E_z is odd there)
        bs = max(np.abs(Bx).max(), np.abs(By).max())
        assert np.abs(phys1[2][0]).max() <= 1e-13 * bs and np.abs(phys1[2][-1]).max() <= 1e-13 * bs
